"""Compile the CUDA library in-tree: csrc/*.cu -> lib/libthc.so (sm_103a only)."""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "lib")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]


def sources():
    return sorted(os.path.join(SRC, f) for f in os.listdir(SRC) if f.endswith(".cu"))


def nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def build(verbose: bool = False, extra=None) -> str:
    """Compile every .cu under csrc/ (in parallel) and link lib/libthc.so."""
    os.makedirs(LIB, exist_ok=True)
    objs, procs = [], []
    for src in sources():
        obj = os.path.join(LIB, os.path.basename(src)[:-3] + ".o")
        cmd = [nvcc(), ARCH, *FLAGS, *(extra or []), "-c", src, "-o", obj]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        procs.append((subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT), src))
        objs.append(obj)
    failed = []
    for p, src in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            failed.append((src, out.decode(errors="replace")))
    if failed:
        raise RuntimeError("nvcc failed:\n" + "\n".join(f"{s}\n{o}" for s, o in failed))
    so = os.path.join(LIB, "libthc.so")
    tmp = so + ".tmp"
    subprocess.check_call([nvcc(), ARCH, "-shared", "-o", tmp, *objs])
    os.replace(tmp, so)
    for o in objs:
        os.remove(o)
    return so


if __name__ == "__main__":
    print(build(verbose=True))

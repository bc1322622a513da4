"""The C-ABI library builds for sm_103a and exports every entry point that
include/thc.h declares (no GPU: nothing is computed here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "thc.h")
LIB = os.path.join(ROOT, "paper_2409_12708_gb300", "lib", "libthc.so")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    # top-level prototypes start in column 0: "<type words> name("
    names = re.findall(r"^(?:[A-Za-z_]\w*[\s*]+)+([A-Za-z_]\w*)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(LIB):
        from paper_2409_12708_gb300 import build as b
        b.build()
    return ctypes.CDLL(LIB)


def test_header_declares_the_hot_path_calls():
    names = declared_functions()
    for n in ["thc_apply_H", "mps_inner", "mps_add_compress", "krylov_lanczos_ground",
              "krylov_expm_apply", "thc_layer_apply", "thc_compress", "thc_kinetic_factors",
              "thc_mps_free", "thc_last_error"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for n in declared_functions():
        assert hasattr(lib, n), n


def test_build_info_and_error_string_without_gpu(lib):
    lib.thc_build_info.restype = ctypes.c_char_p
    lib.thc_last_error.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.thc_build_info()
    assert isinstance(lib.thc_last_error(), bytes)


def test_invalid_arguments_rejected_before_any_gpu_work(lib):
    # a null descriptor is THC_EINVAL and touches no device
    lib.thc_apply_H.restype = ctypes.c_int
    assert lib.thc_apply_H(None, None, None, None, None, None) == 1
    lib.thc_last_error.restype = ctypes.c_char_p
    assert b"null" in lib.thc_last_error()


def test_binding_names_match_header():
    from paper_2409_12708_gb300 import binding as B
    assert set(B.EXPORTED) == set(declared_functions())


def test_binding_structs_match_the_header_layout(tmp_path):
    # the binding's ctypes mirrors of the ABI structs against the C compiler's
    # layout of include/thc.h (size and every field offset)
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    from paper_2409_12708_gb300 import binding as B
    structs = {"thc_opts": B.thc_opts, "thc_mps": B.thc_mps, "thc_hamiltonian": B.thc_hamiltonian,
               "thc_allocator": B.thc_allocator}
    lines = ["#include <stdio.h>", "#include <stddef.h>", f'#include "{HEADER}"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'  printf("{name} sizeof %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'  printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.check_call([cc, "-std=c11", str(src), "-o", str(exe)])
    out = subprocess.check_output([str(exe)], text=True).split("\n")
    c_layout = {(a, b): int(c) for a, b, c in (ln.split() for ln in out if ln.strip())}
    for name, cls in structs.items():
        assert c_layout[(name, "sizeof")] == ctypes.sizeof(cls), name
        for field, _ in cls._fields_:
            assert c_layout[(name, field)] == getattr(cls, field).offset, (name, field)

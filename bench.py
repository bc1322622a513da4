"""Benchmark of the THC-MPO hot path: one step = one full compressed H|psi>
(all 4N^2 Coulomb terms with the reuse of G_{nu s'}|psi>, the 2L kinetic terms,
every layer compressed, the pairwise reduction) on the L = 16, N = 48,
D_max = 128 workload with a half-filled psi whose Schmidt values decay as
exp(-k/12).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  The headline is the batched float32 path; the
plain float64 path is timed on a leading subset of terms and reported beside
it.  Under torchrun every rank runs an independent replica (no collective in
the data path); value = terms processed by all ranks / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2409_12708_gb300.workloads import WORKLOADS, full_bond_profile, workload  # noqa: E402

METRIC = ("THC terms/s and H|ψ⟩ applies/s; Krylov step time, batched+mixed vs plain FP64")
WORKLOAD = "L16_N48_D128"
L2_BYTES = 129 * 2 ** 20


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=1)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default=WORKLOAD)
    p.add_argument("--fp64-terms", type=int, default=96, help="leading terms timed on the float64 path")
    p.add_argument("--cpu-terms", type=int, default=12, help="terms in the oracle's CPU sample")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-fp64", action="store_true")
    p.add_argument("--batch", type=int, default=0)
    p.add_argument("--terms", type=int, default=0,
                   help="apply only the first TERMS terms per step (0 = all; for profiling slices)")
    p.add_argument("--no-profile", action="store_true", help="skip the CUDA-event profiled step")
    p.add_argument("--no-krylov", action="store_true", help="skip the Lanczos step timing")
    return p.parse_args()


# ----------------------------------------------------------------------------- helpers
def n_terms(w):
    return 4 * w["N"] ** 2 + 2 * w["L"]


class Clocks:
    """nvidia-smi samples (SM clock, reasons) taken during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()

    def summary(self):
        try:
            rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.strip()]
        except OSError:
            return None
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if "Active" in v and "Not" not in v})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "samples": len(rows), "reasons": reasons}


def flop_models(w, D, n_applied=None):
    """Algorithmic flops per kernel class for one H|psi> (float32 path) over all
    terms, or over the first n_applied terms.

    Shapes follow the static shape chain of the compression (QR bonds k,
    output bonds chi').  Per-unit models (Golub & Van Loan counts):
      qr_lq_sweep     Householder QR of X^T (m x n) plus forming its Q:
                      2mn k - (m+n)k^2 + 2k^3/3  +  2m k^2 - 2k^3/3,  k = min(m, n)
      qr_svd_precond  Householder QR of C (m x n, m > n): 2mn^2 - 2n^3/3
      jacobi_svd      SVD of the p x n matrix for sigma and V: 4pn^2 + 8n^3
      gemm_*          2 M N K
    """
    L, N = w["L"], w["N"]
    pf = full_bond_profile(L, D)

    def chain(inA, mode):
        e = [1] + [(2 * inA[b] if mode == "layer" else 2 * inA[b]) for b in range(1, L)] + [1]
        k = [1] * (L + 1)
        for s in range(L - 1, 0, -1):
            k[s] = min(e[s], 4 * k[s + 1])
        out = [1] * (L + 1)
        for s in range(L - 1):
            out[s + 1] = min(D, 4 * out[s], k[s + 1])
        return e, k, out

    acc = {}

    def add(name, f):
        acc[name] = acc.get(name, 0.0) + f

    def compress(inA):
        e, k, out = chain(inA, "layer")
        for s in range(L - 1, -1, -1):
            add("gemm_expand_absorb", 2.0 * (e[s] * 4) * k[s + 1] * e[s + 1])
            if s >= 1:
                m, n = 4 * k[s + 1], e[s]
                kk = min(m, n)
                add("qr_lq_sweep", 2 * m * n * kk - (m + n) * kk ** 2 + 2 * kk ** 3 / 3
                    + 2 * m * kk ** 2 - 2 * kk ** 3 / 3)
        for s in range(L - 1):
            m, n, ko = 4 * out[s], k[s + 1], out[s + 1]
            add("gemm_center", 2.0 * out[s] * 4 * n * max(k[s], 1))
            if m > n:
                add("qr_svd_precond", 2 * m * n * n - 2 * n ** 3 / 3)
            p = min(m, n)
            add("jacobi_svd", 4 * p * n * n + 8 * n ** 3)
            add("gemm_u", 2.0 * m * ko * n)
            add("svd_finalize", 4.0 * ko * ko * n + 2.0 * m * ko)
        add("gemm_center", 2.0 * out[L - 1] * 4 * k[L - 1])

    T = n_terms(w) if n_applied is None else n_applied
    # reuse stage: 2 layer compressions per (nu, s') block the applied terms touch
    # (2N consecutive Coulomb terms share one), 2 per term, T-1 reductions; all
    # with the same static shapes
    per = {}
    compress(pf)
    per = dict(acc)
    slots = -(-min(T, 4 * N * N) // (2 * N))
    count = 2 * slots + 2 * T + (T - 1)
    return {k: v * count for k, v in per.items()}, count


def ncu_traffic(profile_name, units_per_launch):
    """DRAM bytes per launch of a kernel from the committed ncu summary.

    profiles/dram_traffic_per_unit.txt holds lines
    "<profile name> <dram bytes per unit> <unit> <source file> <sha1 of it>"
    (dram__bytes_read.sum + dram__bytes_write.sum of one captured launch,
    divided by the units it processed).  The figure is used only while the
    kernel source still hashes to the recorded value; otherwise None.
    """
    import hashlib
    path = os.path.join(ROOT, "profiles", "dram_traffic_per_unit.txt")
    if units_per_launch is None or not os.path.exists(path):
        return None
    for line in open(path):
        f = line.split()
        if len(f) == 5 and f[0] == profile_name:
            src = os.path.join(ROOT, f[3])
            if not os.path.exists(src):
                return None
            if hashlib.sha1(open(src, "rb").read()).hexdigest() != f[4]:
                return None
            return float(f[1]) * units_per_launch
    return None


def roofline(prof, stats, models, clocks):
    """Roofline object of the dominant kernel function of a profiled step.

    prof: {profile name: {"launches", "ms"}} from the library's CUDA-event
    profile; stats: the Jacobi sweep statistics; models: algorithmic flops per
    profile name; clocks: the sampled clock summary.  Profile names are grouped
    by the kernel that runs them (k_qr serves the LQ sweep and the
    preconditioning QR), the one with the most time is reported against the
    derived FP32 SIMT peak, with its DRAM traffic from the committed ncu figure.
    """
    kernel_of = {"jacobi_svd": "k_jacobi_select", "qr_lq_sweep": "k_qr", "qr_svd_precond": "k_qr"}
    by_kernel = {}
    for nm, rec in prof.items():
        kn = kernel_of.get(nm)
        if kn is None:
            continue
        e = by_kernel.setdefault(kn, {"ms": 0.0, "launches": 0, "flops": 0.0, "names": []})
        e["ms"] += rec["ms"]
        e["launches"] += rec["launches"]
        e["flops"] += models.get(nm, 0.0)
        e["names"].append(nm)
    if not by_kernel:
        return None
    kname, rec = max(by_kernel.items(), key=lambda kv: kv[1]["ms"])
    sm_mhz = (clocks or {}).get("sm_mhz") or 2070.0
    achieved = rec["flops"] / (rec["ms"] / 1e3) / 1e12
    peak = fp32_alu_peak_tflops(sm_mhz)
    # matrices (CTAs) per launch: every compression step launches over the same
    # batch of terms, counted by the Jacobi statistics
    units = None
    if "jacobi_sweeps_all" in stats and "jacobi_svd" in prof:
        units = stats["jacobi_sweeps_all"]["launches"] / max(prof["jacobi_svd"]["launches"], 1)
    return {"kernel": kname, "profile_names": sorted(rec["names"]), "bound": "alu", "achieved": achieved,
            "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak, "traffic": ncu_traffic(kname, units),
            "traffic_unit": "DRAM bytes per launch (ncu, scaled by matrices per launch)",
            "launches_per_step": rec["launches"], "ms_per_step": rec["ms"],
            "peak_note": f"derived FP32 SIMT peak: 152 SMs x 128 lanes x 2 flop x {sm_mhz:.0f} MHz "
                         "(median SM clock under load)"}


def fp32_alu_peak_tflops(sm_mhz, sms=152):
    # 128 FP32 lanes per SM, one FMA (2 flops) per lane per clock
    return sms * 128 * 2 * sm_mhz * 1e6 / 1e12


# ----------------------------------------------------------------------------- reference arm
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import thc as OT
    w = WORKLOADS[args.workload]
    t, chi, zeta, psi, D = workload(args.workload)
    sample = 2  # terms per step: two Coulomb terms, their shared reuse state, one reduction
    for _ in range(args.warmup):
        OT.apply_H(psi, t, chi, zeta, D_max=D, term_begin=0, term_end=sample)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        OT.apply_H(psi, t, chi, zeta, D_max=D, term_begin=0, term_end=sample)
    dt = (time.perf_counter() - t0) / args.steps
    v = sample / dt
    cores = os.cpu_count()
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "terms/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "L": w["L"], "N": w["N"], "D_max": D, "terms": n_terms(w),
                   "path": "oracle float64 (timed sample: %d terms per step)" % sample,
                   "parallelism": "single"},
        "cpu_baseline": {"value": v, "unit": "terms/s", "cores": cores, "kind": "oracle",
                         "sample": f"terms [0,{sample}) of the workload per step (numpy float64 oracle)"},
        "e2e": {"value": v, "unit": "terms/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def cpu_baseline(args):
    from oracle import thc as OT
    t, chi, zeta, psi, D = workload(args.workload)
    n = args.cpu_terms
    t0 = time.perf_counter()
    OT.apply_H(psi, t, chi, zeta, D_max=D, term_begin=0, term_end=n)
    dt = time.perf_counter() - t0
    threads = os.environ.get("OMP_NUM_THREADS") or os.environ.get("OPENBLAS_NUM_THREADS")
    return {"value": n / dt, "unit": "terms/s", "cores": int(threads) if threads else os.cpu_count(),
            "kind": "oracle",
            "sample": f"terms [0,{n}) of the workload: their reuse state, {2 * n} layers and the "
                      f"{n - 1}-add pairwise reduction, numpy float64, {dt:.1f} s"}


def combine_replicas(seconds, n_step, steps, world, dist=None, device="cpu"):
    """Whole-job throughput of `world` independent replicas: every rank timed
    `steps` steps of n_step terms in `seconds`; the job time is the maximum
    over ranks (an all-reduce of one float64 when world > 1), and the value is
    all ranks' terms over that time.  Returns (terms/s, ms per step)."""
    if world > 1:
        import torch
        tt = torch.tensor([seconds], device=device, dtype=torch.float64)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        seconds = float(tt)
    return n_step * steps * world / seconds, seconds / steps * 1e3


# ----------------------------------------------------------------------------- our arm
def run_ours(args):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    from paper_2409_12708_gb300 import binding as B

    w = WORKLOADS[args.workload]
    t, chi, zeta, psi, D = workload(args.workload)
    T = n_terms(w)
    dev = lambda a, dt=torch.float64: torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dt)
    H = (dev(t), dev(chi), dev(zeta))
    psi32 = [dev(a, torch.float32) for a in psi]
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")

    n_step = args.terms if args.terms > 0 else T

    def step():
        if args.terms > 0:
            return B.thc_apply_H(*H, psi32, D_max=D, path="fp32", batch=args.batch, term_begin=0,
                                 term_end=args.terms)
        return B.thc_apply_H(*H, psi32, D_max=D, path="fp32", batch=args.batch)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        step()
    barrier()
    launches0 = B.kernel_launches()
    ms = []
    with Clocks(local) as clk:
        for _ in range(args.steps):
            flush.fill_(1.0)  # evict L2 between timed steps
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            out = step()
            e1.record()
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
    barrier()
    launches = (B.kernel_launches() - launches0) // max(args.steps, 1)
    value, ms_step = combine_replicas(sum(ms) / 1e3, n_step, args.steps, world, dist if world > 1 else None,
                                      "cuda")

    # ---- end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        hp = [torch.from_numpy(np.ascontiguousarray(a)).float().pin_memory() for a in psi]
        hH = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in (t, chi, zeta)]
        h2d = sum(x.numel() * x.element_size() for x in hp + hH)
        d2h = 0
        tms = []
        for _ in range(1):  # one end-to-end step (each step is a full H|psi>)
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            dH = [x.to("cuda", non_blocking=True) for x in hH]
            dp = [x.to("cuda", non_blocking=True) for x in hp]
            if args.terms > 0:
                o = B.thc_apply_H(*dH, dp, D_max=D, path="fp32", batch=args.batch, term_begin=0,
                                  term_end=args.terms)
            else:
                o = B.thc_apply_H(*dH, dp, D_max=D, path="fp32", batch=args.batch)
            res = [x.to("cpu", non_blocking=True) for x in o]
            e1.record()
            e1.synchronize()
            tms.append(e0.elapsed_time(e1))
            d2h = sum(x.numel() * x.element_size() for x in res)
        e2e = {"value": n_step * len(tms) * world / (sum(tms) / 1e3), "unit": "terms/s",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

    # ---- one profiled step: per-kernel CUDA-event durations for the roofline
    prof = {}
    if not args.no_profile:
        B.profile_read()
        B.profile_enable(True)
        step()
        torch.cuda.synchronize()
        prof = B.profile_read()
        B.profile_enable(False)
    stats = {k: prof.pop(k) for k in list(prof) if k.startswith("jacobi_sweeps") or k.startswith("jacobi_budget")}

    # ---- plain float64 per-term path on a leading subset of terms (extrapolated)
    fp64 = None
    if not args.no_fp64:
        psi64 = [dev(a) for a in psi]
        n64 = min(args.fp64_terms, T)
        B.thc_apply_H(*H, psi64, D_max=D, path="fp64", term_begin=0, term_end=min(n64, 4))
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        B.thc_apply_H(*H, psi64, D_max=D, path="fp64", term_begin=0, term_end=n64)
        e1.record()
        e1.synchronize()
        s64 = e0.elapsed_time(e1) / 1e3
        fp64 = {"value": n64 / s64, "unit": "terms/s", "terms_timed": n64,
                "extrapolated_hpsi_s": s64 * T / n64,
                "note": f"float64 path timed on terms [0,{n64}) incl. their reuse states, extrapolated"}

    # ---- Krylov step time: 10-step Lanczos on the small L=6, N=12, D=16 workload
    # (after the timed region; one warm-up run each)
    krylov = None
    if not args.no_krylov and rank == 0:
        tk, ck, zk, pk, Dk = workload("L6_N12_D16")
        Hk = (dev(tk), dev(ck), dev(zk))
        krylov = {"workload": "L6_N12_D16", "K": 10}
        for pth, dtk in (("fp64", torch.float64), ("fp32", torch.float32)):
            pp = [dev(a, dtk) for a in pk]
            B.krylov_lanczos_ground(*Hk, pp, 10, Dk, path=pth)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            en, _, _ = B.krylov_lanczos_ground(*Hk, pp, 10, Dk, path=pth)
            e1.record()
            e1.synchronize()
            krylov[pth] = {"s_per_krylov_step": e0.elapsed_time(e1) / 1e3 / 10, "energy": en}

    if rank != 0:
        return
    clocks = clk.summary()
    models, n_compress = flop_models(w, D, n_step)
    roof = roofline(prof, stats, models, clocks)
    line = {
        "metric": METRIC, "value": value, "unit": "terms/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": args.workload, "L": w["L"], "N": w["N"], "D_max": D, "terms": n_step,
                   "path": "fp32", "l2": "flushed between steps (256 MiB write)",
                   "parallelism": "replicas" if world > 1 else "single"},
        "hpsi_per_s": value / T,
        "gpu_launches": int(launches),
        "e2e": e2e,
        "roofline": roof,
        "clocks": clocks,
        "fp64": fp64,
        "speedup_vs_fp64": (value / world) / fp64["value"] if fp64 else None,
        "kernel_ms_per_step": {k: round(v["ms"], 3) for k, v in sorted(prof.items(), key=lambda kv: -kv[1]["ms"])},
        "jacobi_sweeps_per_svd": {k: round(v["ms"] / max(v["launches"], 1), 2) for k, v in stats.items()
                                  if k.startswith("jacobi_sweeps")},
        "compressions_per_step": n_compress,
        "krylov": krylov,
    }
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline(args)
    print(json.dumps(line))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

"""Benchmark of the THC-MPO hot path: one step = one full compressed H|psi>
(all 4N^2 Coulomb terms with the reuse of G_{nu s'}|psi>, the 2L kinetic terms,
every layer compressed, the pairwise reduction) on the L = 16, N = 48,
D_max = 128 workload with a half-filled psi whose Schmidt values decay as
exp(-k/12).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  The headline is the batched float32 path; the
float32 and plain float64 paths are also timed on the same leading slice of
terms with the whole slice in flight, with the float32 result's distance from
the float64 one.  Under torchrun every rank runs an independent replica (no collective in
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

from paper_2409_12708_gb300.workloads import (WORKLOADS, full_bond_profile, sector_mps,  # noqa: E402
                                              thc_hamiltonian, workload)

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
    p.add_argument("--slice-terms", type=int, default=608,
                   help="leading terms on which the float32 and float64 paths are compared (same terms, "
                        "all of them in flight at once)")
    p.add_argument("--cpu-terms", type=int, default=12, help="terms in the oracle's CPU sample")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-fp64", action="store_true")
    p.add_argument("--batch", type=int, default=0)
    p.add_argument("--path", default="tf32", choices=["fp32", "tf32"],
                   help="compute path of the headline (tf32: contractions on the tensor cores)")
    p.add_argument("--terms", type=int, default=0,
                   help="apply only the first TERMS terms per step (0 = all; for profiling slices)")
    p.add_argument("--no-profile", action="store_true", help="skip the CUDA-event profiled step")
    p.add_argument("--no-krylov", action="store_true", help="skip the Lanczos step timing")
    p.add_argument("--no-adjoint", action="store_true", help="skip the adjoint (L=16, N=48, D=64) record")
    p.add_argument("--no-expm", action="store_true", help="skip the Krylov time-step record")
    p.add_argument("--no-config2", action="store_true", help="skip the L=24, N=96, D=256 slice record")
    p.add_argument("--no-merge", action="store_true", help="skip the spin-merged H|psi> record")
    p.add_argument("--no-peaks", action="store_true", help="skip the cuBLAS GEMM rate measurement")
    p.add_argument("--no-batched", action="store_true", help="skip the batched-instances record")
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


def qr_flops(m, n):
    """Householder QR of an m x n matrix without forming Q (Golub & Van Loan):
    sum over the k = min(m, n) reflectors of 4 (m - j)(n - j) = 2mn^2 - 2n^3/3
    for m >= n."""
    k = min(m, n)
    return 4.0 * m * n * k - 2.0 * (m + n) * k * k + 4.0 * k ** 3 / 3.0


def svd_flops(m, n):
    """Singular values and right singular vectors of an m x n matrix
    (Golub & Van Loan, R-SVD count): 4mn^2 + 8n^3 with the roles of m and n
    taken so that m >= n."""
    a, b = max(m, n), min(m, n)
    return 4.0 * a * b * b + 8.0 * b ** 3


# The units of the algorithmic-work model: per compression, the QR sweep's
# Householder QR of every X_s^T (unit "qr"), the SVD sweep's factorisation of
# every C_s for sigma and V ("svd", which the library runs as a pivoted QR of C
# followed by one-sided Jacobi), and the contractions ("gemm").
# qt_apply forms the product M Q^T from the stored reflectors (the float
# paths' replacement of gemm_center): its algorithmic work is that product's.
UNIT_OF = {"qr_lq_sweep": "qr", "qr_svd_precond": "svd", "jacobi_svd": "svd", "gemm_expand_absorb": "gemm",
           "gemm_center": "gemm", "qt_apply": "gemm", "gemm_u": "gemm", "svd_finalize": "gemm"}
KERNELS_OF = {"qr": "k_qr (LQ sweep launches)", "svd": "k_qr (pivoted R-only launches) + k_jacobi_select",
              "gemm": "k_gemm128 / k_gemm / k_gemm_tc / k_apply_qt"}


def flop_models(w, D, n_applied=None):
    """Algorithmic flops per unit class for one H|psi> over all terms, or over
    the first n_applied terms.

    Shapes follow the static shape chain of the compression (QR bonds k,
    output bonds chi').  Per compression (one expanded term, Fig. 3):
      qr    sites L-1..1: Householder QR of X_s^T (m = 4 k_{s+1}, n = e_s), no Q formation
      svd   sites 0..L-2: sigma and V of C_s (m = 4 chi'_s, n = k_{s+1})
      gemm  expand+absorb, M Q (a GEMM, or the reflectors applied on the
            float paths), U = C V^T, the projector correction: 2 M N K
    Returns ({unit: flops}, compressions).
    """
    L, N = w["L"], w["N"]
    pf = full_bond_profile(L, D)
    e = [1] + [2 * pf[b] for b in range(1, L)] + [1]
    k = [1] * (L + 1)
    for s in range(L - 1, 0, -1):
        k[s] = min(e[s], 4 * k[s + 1])
    out = [1] * (L + 1)
    for s in range(L - 1):
        out[s + 1] = min(D, 4 * out[s], k[s + 1])
    per = {"qr": 0.0, "svd": 0.0, "gemm": 0.0}
    for s in range(L - 1, -1, -1):
        per["gemm"] += 2.0 * (e[s] * 4) * k[s + 1] * e[s + 1]
        if s >= 1:
            per["qr"] += qr_flops(4 * k[s + 1], e[s])
    for s in range(L - 1):
        m, n, ko = 4 * out[s], k[s + 1], out[s + 1]
        per["gemm"] += 2.0 * out[s] * 4 * n * max(k[s], 1) + 2.0 * m * ko * n + 4.0 * ko * ko * n
        per["svd"] += svd_flops(m, n)
    per["gemm"] += 2.0 * out[L - 1] * 4 * k[L - 1]
    T = n_terms(w) if n_applied is None else n_applied
    # reuse stage: 2 layer compressions per (nu, s') block the applied terms touch
    # (2N consecutive Coulomb terms share one), 2 per term, T-1 reductions; all
    # with the same static shapes
    slots = -(-min(T, 4 * N * N) // (2 * N))
    count = 2 * slots + 2 * T + (T - 1)
    return {u: v * count for u, v in per.items()}, count


def ncu_traffic(kernel, units_per_launch):
    """DRAM bytes per launch of a kernel from the committed ncu summary.

    profiles/dram_traffic_per_unit.txt holds lines
    "<kernel key> <dram bytes per unit> <unit> <source file> <sha1 of it>"
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
        if len(f) == 5 and f[0] == kernel:
            src = os.path.join(ROOT, f[3])
            if not os.path.exists(src):
                return None
            if hashlib.sha1(open(src, "rb").read()).hexdigest() != f[4]:
                return None
            return float(f[1]) * units_per_launch
    return None


def fp32_alu_peak_tflops(sm_mhz, sms):
    """FP32 SIMT peak: sms x 128 FP32 lanes x one FMA (2 flops) per clock."""
    return sms * 128 * 2 * sm_mhz * 1e6 / 1e12


def measure_gemm_peaks(torch):
    """Dense GEMM rates of this GPU through cuBLAS (torch.matmul), the
    denominators the measured-peaks file lacks: TF32 tensor (8192^3, float32
    inputs with TF32 allowed), FP32 SIMT (same shape, TF32 off) and FP64
    (4096^3).  Best of 5 after 2 warm-up calls, CUDA events; a second of GPU
    time in all."""
    def rate(n, dtype, tf32, reps=5):
        old = torch.backends.cuda.matmul.allow_tf32
        torch.backends.cuda.matmul.allow_tf32 = tf32
        try:
            a = torch.randn(n, n, device="cuda", dtype=dtype)
            b = torch.randn(n, n, device="cuda", dtype=dtype)
            for _ in range(2):
                a @ b
            best = None
            for _ in range(reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                a @ b
                e1.record()
                e1.synchronize()
                ms = e0.elapsed_time(e1)
                best = ms if best is None else min(best, ms)
            return 2.0 * n ** 3 / (best / 1e3) / 1e12
        finally:
            torch.backends.cuda.matmul.allow_tf32 = old
    return {"tf32_tflops": rate(8192, torch.float32, True), "fp32_simt_tflops": rate(8192, torch.float32, False),
            "fp64_tflops": rate(4096, torch.float64, False),
            "note": "cuBLAS via torch.matmul on this GPU: TF32 8192^3, FP32 8192^3 (TF32 off), FP64 4096^3; "
                    "best of 5 after 2 warm-up calls"}


def roofline(prof, stats, models, clocks, sms, peaks=None, tf32_measured=None):
    """Roofline object of the dominant unit class of a profiled step.

    prof: {profile name: {"launches", "ms"}} from the library's CUDA-event
    profile; stats: the Jacobi sweep statistics; models: algorithmic flops per
    unit class (flop_models); clocks: the sampled clock summary; sms: the
    device's SM count; peaks: MEASURED_PEAKS.json.  Profile names are grouped
    into the units of flop_models; the unit with the most time is reported
    against the derived FP32 SIMT peak (the kernels are SIMT float32), with the
    TF32 tensor peak (half the measured BF16 sustained rate) beside it.
    """
    by_unit = {}
    for nm, rec in prof.items():
        u = UNIT_OF.get(nm)
        if u is None:
            continue
        e = by_unit.setdefault(u, {"ms": 0.0, "launches": 0, "names": []})
        e["ms"] += rec["ms"]
        e["launches"] += rec["launches"]
        e["names"].append(nm)
    if not by_unit:
        return None
    unit, rec = max(by_unit.items(), key=lambda kv: kv[1]["ms"])
    sm_mhz = (clocks or {}).get("sm_mhz") or 2070.0
    peak = fp32_alu_peak_tflops(sm_mhz, sms)
    if tf32_measured:
        tf32, tf32_src = tf32_measured, "the measured cuBLAS TF32 GEMM rate of this run"
    elif peaks and "bf16_tflops_sustained" in peaks:
        tf32, tf32_src = 0.5 * peaks["bf16_tflops_sustained"], "1/2 of the measured BF16 sustained rate"
    else:
        tf32, tf32_src = None, "not available"
    summary = {}
    for u, r in by_unit.items():
        a = models.get(u, 0.0) / (r["ms"] / 1e3) / 1e12
        summary[u] = {"ms_per_step": r["ms"], "flops_per_step": models.get(u, 0.0), "achieved_tflops": a,
                      "frac_fp32_simt": a / peak, "frac_tf32_tensor": a / tf32 if tf32 else None,
                      "profile_names": sorted(r["names"])}
    achieved = summary[unit]["achieved_tflops"]
    # matrices (CTAs) per launch: every compression step launches over the same
    # batch of terms, counted by the Jacobi statistics
    units = None
    if "jacobi_sweeps_all" in stats and "jacobi_svd" in prof:
        units = stats["jacobi_sweeps_all"]["launches"] / max(prof["jacobi_svd"]["launches"], 1)
    traffic = None
    if unit == "qr":
        traffic = ncu_traffic("k_qr", units)
    elif unit == "svd":
        a, b = ncu_traffic("k_qr_precond", units), ncu_traffic("k_jacobi_select", units)
        traffic = a + b if a is not None and b is not None else None
    return {"kernel": KERNELS_OF[unit], "unit": "TFLOP/s", "work_unit": unit, "bound": "alu",
            "achieved": achieved, "peak": peak, "frac": achieved / peak,
            "peak_tensor_tf32": tf32, "frac_tensor_tf32": achieved / tf32 if tf32 else None,
            "traffic": traffic, "traffic_unit": "DRAM bytes per launch (ncu, scaled by matrices per launch)",
            "launches_per_step": rec["launches"], "ms_per_step": rec["ms"], "by_unit": summary,
            "peak_note": f"FP32 SIMT peak derived from the device: {sms} SMs x 128 lanes x 2 flop x "
                         f"{sm_mhz:.0f} MHz (median SM clock under load); TF32 tensor peak = {tf32_src}"}


def read_golden(path):
    """{name: value} from a golden file ("name value" lines, '#' comments)."""
    vals = {}
    if os.path.exists(path):
        for line in open(path):
            if line.strip() and not line.startswith("#"):
                k, v = line.split()
                vals[k] = float(v)
    return vals


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
            return B.thc_apply_H(*H, psi32, D_max=D, path=args.path, batch=args.batch, term_begin=0,
                                 term_end=args.terms)
        return B.thc_apply_H(*H, psi32, D_max=D, path=args.path, batch=args.batch)

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
                o = B.thc_apply_H(*dH, dp, D_max=D, path=args.path, batch=args.batch, term_begin=0,
                                  term_end=args.terms)
            else:
                o = B.thc_apply_H(*dH, dp, D_max=D, path=args.path, batch=args.batch)
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
    stats = {k: prof.pop(k) for k in list(prof)
             if k.startswith("jacobi_sweeps") or k.startswith("jacobi_budget") or k == "tc_gemm_launches"}

    # ---- the spin-merged term list (3N^2 Coulomb terms instead of 4N^2): one
    # whole H|psi> on the same path, its time beside the timed step's, and its
    # relative distance from the timed step's result (both truncated at D_max:
    # the two term lists differ by their truncation errors)
    merged = None
    if not args.no_merge and args.terms == 0 and rank == 0:
        Tm = 3 * w["N"] * w["N"] + 2 * w["L"]
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        om = B.thc_apply_H(*H, psi32, D_max=D, path=args.path, batch=args.batch, merge_spin=True)
        e1.record()
        e1.synchronize()
        sm = e0.elapsed_time(e1) / 1e3
        a = [x.double() for x in om]
        b = [x.double() for x in out]
        aa, bb, ab = B.mps_inner(a, a), B.mps_inner(b, b), B.mps_inner(a, b)
        merged = {"terms": Tm, "hpsi_s": sm, "hpsi_per_s": 1.0 / sm, "speedup_vs_unmerged": ms_step / 1e3 / sm,
                  "rel_distance_to_unmerged": float(np.sqrt(max(aa + bb - 2.0 * ab, 0.0) / bb)),
                  "note": "opposite-spin Coulomb terms folded pairwise (G_{mu up}, G_{nu down} commute, zeta "
                          "symmetric); same path and D_max as the timed step; distance by float64 inner "
                          "products on the device"}

    # ---- independent instances of uneven L in one call (thc_apply_H_batched):
    # 8 Hamiltonians L = 8..16, N = 2L, half-filled states at D_max = 32, on
    # the same path; the batched call against the 8 single calls in sequence
    batched = None
    if not args.no_batched and rank == 0:
        Ls = (8, 10, 12, 14, 16, 16, 12, 10)
        hams, psis = [], []
        for k, Lb in enumerate(Ls):
            tb, cb, zb = thc_hamiltonian(Lb, 2 * Lb, seed=100 + k)
            hams.append((dev(tb), dev(cb), dev(zb)))
            psis.append([dev(a, torch.float32) for a in sector_mps(Lb, Lb // 2, Lb // 2, 32, seed=200 + k)])
        Tb = sum(4 * (2 * Lb) ** 2 + 2 * Lb for Lb in Ls)
        B.thc_apply_H_batched(hams[:2], psis[:2], D_max=32, path=args.path)  # warm-up
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for h, pp in zip(hams, psis):
            B.thc_apply_H(*h, pp, D_max=32, path=args.path)
        e1.record()
        e1.synchronize()
        s_seq = e0.elapsed_time(e1) / 1e3
        e0.record()
        B.thc_apply_H_batched(hams, psis, D_max=32, path=args.path)
        e1.record()
        e1.synchronize()
        s_bat = e0.elapsed_time(e1) / 1e3
        batched = {"instances": [f"L{Lb}_N{2 * Lb}_D32" for Lb in Ls], "terms": Tb, "path": args.path,
                   "sequential_s": s_seq, "batched_s": s_bat, "batched_terms_per_s": Tb / s_bat,
                   "speedup": s_seq / s_bat,
                   "note": "8 independent H|psi> (own Hamiltonian and state each) in one call, one stream per "
                           "instance, against the 8 single calls in sequence on one stream"}

    # ---- float32 vs plain float64 on the same leading slice of terms, every term
    # of the slice in flight at once on both paths (so both fill the GPU alike);
    # the float32 result's distance from the float64 one is computed with float64
    # inner products on the device: |a-b|^2 = <a|a> + <b|b> - 2<a|b>
    fp64 = None
    if not args.no_fp64:
        psi64 = [dev(a) for a in psi]
        n64 = min(args.slice_terms, T)
        res = {}
        for pth, pp in (("fp32", psi32), ("tf32", psi32), ("fp64", psi64)):
            B.thc_apply_H(*H, pp, D_max=D, path=pth, term_begin=0, term_end=min(n64, 8), batch=8)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            o = B.thc_apply_H(*H, pp, D_max=D, path=pth, term_begin=0, term_end=n64, batch=n64)
            e1.record()
            e1.synchronize()
            res[pth] = (e0.elapsed_time(e1) / 1e3, o)
        b = res["fp64"][1]
        bb = B.mps_inner(b, b)

        def rel_to_fp64(pth):
            a = [x.double() for x in res[pth][1]]
            aa, ab = B.mps_inner(a, a), B.mps_inner(a, b)
            return float(np.sqrt(max(aa + bb - 2.0 * ab, 0.0) / bb))

        s32, s64, stf = res["fp32"][0], res["fp64"][0], res["tf32"][0]
        fp64 = {"terms": n64, "in_flight": n64, "fp64_terms_per_s": n64 / s64, "fp32_terms_per_s": n64 / s32,
                "tf32_terms_per_s": n64 / stf, "speedup_fp32_vs_fp64": s64 / s32,
                "speedup_tf32_vs_fp64": s64 / stf, "fp32_rel_error_vs_fp64": rel_to_fp64("fp32"),
                "tf32_rel_error_vs_fp64": rel_to_fp64("tf32"),
                "extrapolated_fp64_hpsi_s": s64 * T / n64,
                "note": f"both paths on terms [0,{n64}) with all {n64} terms in flight; float64 H|psi> time "
                        f"extrapolated from the slice (labelled); relative distance of the float32 result "
                        f"from the float64 one, float64 inner products on the device"}

    # ---- Krylov step time: 10-step Lanczos on the L=6, N=12 workload (after the
    # timed region; one warm-up run each), at D_max = 16 and untruncated (64);
    # energies beside the exact ground energy of the (3,3) sector and the dense
    # 10-step Lanczos value of the same start vector (committed golden file)
    krylov = None
    if not args.no_krylov and rank == 0:
        tk, ck, zk, pk, Dk = workload("L6_N12_D16")
        Hk = (dev(tk), dev(ck), dev(zk))
        gold = read_golden(os.path.join(ROOT, "tests", "golden", "config0_energies.txt"))
        krylov = {"workload": "L6_N12_D16", "K": 10, "ed_ground_energy": gold.get("ed_ground_energy"),
                  "dense_lanczos_K10": gold.get("dense_lanczos_K10")}
        for pth, dtk in (("fp64", torch.float64), ("fp32", torch.float32)):
            for Dx in (Dk, 64):
                pp = [dev(a, dtk) for a in pk]
                B.krylov_lanczos_ground(*Hk, pp, 10, Dx, path=pth)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                en, _, _ = B.krylov_lanczos_ground(*Hk, pp, 10, Dx, path=pth)
                e1.record()
                e1.synchronize()
                rec = {"s_per_krylov_step": e0.elapsed_time(e1) / 1e3 / 10, "energy": en}
                if gold:
                    rec["minus_ed"] = en - gold["ed_ground_energy"]
                    rec["minus_dense_lanczos_K10"] = en - gold["dense_lanczos_K10"]
                krylov[f"{pth}_D{Dx}"] = rec

    # ---- the adjoint on the L=16, N=48, D_max=64 configuration: phi and psi
    # independent half-filled states; all 9248 terms in float32 (value and every
    # derivative), the float64 path on one (nu, s') block (96 terms,
    # extrapolated, labelled), and central finite differences (step 1e-5) of
    # that block's float64 value on random entries of chi, zeta and psi
    adjoint = None
    if not args.no_adjoint and rank == 0:
        tA, cA, zA = thc_hamiltonian(16, 48, seed=0)
        phiA = sector_mps(16, 8, 8, 64, seed=1003)
        psiA = sector_mps(16, 8, 8, 64, seed=1013)
        HA = (dev(tA), dev(cA), dev(zA))
        TA = 4 * 48 * 48 + 32
        adjoint = {"workload": "L16_N48_D64 (phi, psi independent half-filled)", "terms": TA}
        p32 = ([dev(a, torch.float32) for a in phiA], [dev(a, torch.float32) for a in psiA])
        p64 = ([dev(a) for a in phiA], [dev(a) for a in psiA])
        B.thc_expect_grad(*HA, *p32, path="fp32", term_begin=0, term_end=96)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        v32 = B.thc_expect_grad(*HA, *p32, path="fp32")
        e1.record()
        e1.synchronize()
        adjoint["fp32_all_terms_s"] = e0.elapsed_time(e1) / 1e3
        adjoint["fp32_value"] = v32[0]
        e0.record()
        v64 = B.thc_expect_grad(*HA, *p64, term_begin=0, term_end=96)
        e1.record()
        e1.synchronize()
        s64 = e0.elapsed_time(e1) / 1e3
        adjoint["fp64_96_terms_s"] = s64
        adjoint["fp64_extrapolated_all_terms_s"] = s64 * TA / 96
        rng = np.random.default_rng(7)
        worst = 0.0
        X, Z, P = HA[1], HA[2], p64[1]
        val = lambda x, z, pp: B.thc_expect_grad(HA[0], x, z, p64[0], pp, grads=False, term_begin=0, term_end=96)
        for _ in range(4):
            for which in ("chi", "zeta", "psi"):
                if which == "chi":
                    i = (int(rng.integers(16)), int(rng.integers(48)))
                    xp, xm = X.clone(), X.clone()
                    xp[i] += 1e-5
                    xm[i] -= 1e-5
                    fd = (val(xp, Z, P) - val(xm, Z, P)) / 2e-5
                    g = float(v64[2][i])
                elif which == "zeta":
                    i = (int(rng.integers(48)), int(rng.integers(48)))
                    zp, zm = Z.clone(), Z.clone()
                    zp[i] += 1e-5
                    zm[i] -= 1e-5
                    fd = (val(X, zp, P) - val(X, zm, P)) / 2e-5
                    g = float(v64[3][i])
                else:
                    st = int(rng.integers(16))
                    i = tuple(int(rng.integers(n)) for n in P[st].shape)
                    pp, pm = [x.clone() for x in P], [x.clone() for x in P]
                    pp[st][i] += 1e-5
                    pm[st][i] -= 1e-5
                    fd = (val(X, Z, pp) - val(X, Z, pm)) / 2e-5
                    g = float(v64[4][st][i])
                worst = max(worst, abs(g - fd) / max(abs(fd), 1e-2))
        adjoint["fp64_fd_check"] = {"entries": 12, "step": 1e-5, "max_rel_error": worst,
                                    "note": "terms [0,96), float64, central differences"}

    # ---- one Krylov time step (K = 12, dt = 0.05) with complex site tensors
    expm = None
    if not args.no_expm and rank == 0:
        tk, ck, zk, pk, Dk = workload("L6_N12_D16")
        Hk = (dev(tk), dev(ck), dev(zk))
        expm = {"workload": "L6_N12_D16", "K": 12, "dt": 0.05}
        for pth, dtk in (("fp64", torch.float64), ("fp32", torch.float32)):
            pp = [dev(a, dtk) for a in pk]
            B.krylov_expm_apply(*Hk, pp, 0.05, 12, Dk, path=pth)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            _, lost = B.krylov_expm_apply(*Hk, pp, 0.05, 12, Dk, path=pth)
            e1.record()
            e1.synchronize()
            expm[pth] = {"s_per_time_step": e0.elapsed_time(e1) / 1e3, "lost_norm": lost}

    # ---- the L=24, N=96, D_max=256 configuration on one (nu, s') block
    # (192 terms), extrapolated to a full H|psi> and a 20-step Lanczos (labelled)
    config2 = None
    if not args.no_config2 and rank == 0:
        t2, c2, z2, p2, D2 = workload("L24_N96_D256")
        H2 = (dev(t2), dev(c2), dev(z2))
        T2 = 4 * 96 * 96 + 48
        config2 = {"workload": "L24_N96_D256", "terms": T2, "timed_terms": 192}
        pp = [dev(a, torch.float32) for a in p2]
        B.thc_apply_H(*H2, pp, D_max=D2, path=args.path, term_begin=0, term_end=8, batch=8)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        B.thc_apply_H(*H2, pp, D_max=D2, path=args.path, term_begin=0, term_end=192)
        e1.record()
        e1.synchronize()
        s2 = e0.elapsed_time(e1) / 1e3
        config2.update({"path": args.path, "terms_per_s": 192 / s2, "extrapolated_hpsi_s": s2 * T2 / 192,
                        "extrapolated_20_step_lanczos_s": 20 * s2 * T2 / 192,
                        "note": "one (nu, s') block timed, whole H|psi> and Lanczos extrapolated"})

    if rank != 0:
        return
    clocks = clk.summary()
    models, n_compress = flop_models(w, D, n_step)
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    peaks = None
    if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")):
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    gemm_peaks = None if args.no_peaks else measure_gemm_peaks(torch)
    roof = roofline(prof, stats, models, clocks, sms, peaks,
                    tf32_measured=gemm_peaks["tf32_tflops"] if gemm_peaks else None)
    line = {
        "metric": METRIC, "value": value, "unit": "terms/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": args.workload, "L": w["L"], "N": w["N"], "D_max": D, "terms": n_step,
                   "path": args.path, "l2": "flushed between steps (256 MiB write)",
                   "parallelism": "replicas" if world > 1 else "single"},
        "hpsi_per_s": value / T,
        "gpu_launches": int(launches),
        "e2e": e2e,
        "roofline": roof,
        "clocks": clocks,
        "fp64": fp64,
        "speedup_vs_fp64": fp64["speedup_%s_vs_fp64" % args.path] if fp64 else None,
        "kernel_ms_per_step": {k: round(v["ms"], 3) for k, v in sorted(prof.items(), key=lambda kv: -kv[1]["ms"])},
        "jacobi_sweeps_per_svd": {k: round(v["ms"] / max(v["launches"], 1), 2) for k, v in stats.items()
                                  if k.startswith("jacobi_sweeps")},
        "jacobi_budget_exhausted": int(stats["jacobi_budget_exhausted"]["launches"])
        if "jacobi_budget_exhausted" in stats else 0,
        "compressions_per_step": n_compress,
        "krylov": krylov,
        "adjoint": adjoint,
        "expm": expm,
        "config2": config2,
        "merged_spin": merged,
        "gemm_peaks": gemm_peaks,
        "batched_instances": batched,
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

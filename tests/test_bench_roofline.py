"""Host logic of bench.py's roofline object (no GPU): profile names are grouped
by kernel function, the dominant one is reported, and the ncu traffic figure is
scaled by the matrices per launch and dropped when the kernel source changed."""
import hashlib
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _prof():
    # the numbers of a profiled step of the L=16, N=48, D=128 workload
    prof = {"jacobi_svd": {"launches": 915, "ms": 8361.6}, "qr_lq_sweep": {"launches": 915, "ms": 6063.1},
            "qr_svd_precond": {"launches": 671, "ms": 2774.4}, "gemm_center": {"launches": 976, "ms": 619.7}}
    stats = {"jacobi_sweeps_all": {"launches": 292000, "ms": 1.68e6}}
    return prof, stats


def test_dominant_kernel_groups_qr_profile_names():
    prof, stats = _prof()
    models = {"jacobi_svd": 5.0e16, "qr_lq_sweep": 3.0e16, "qr_svd_precond": 1.0e16}
    r = bench.roofline(prof, stats, models, {"sm_mhz": 2070.0})
    assert r["kernel"] == "k_qr"
    assert r["profile_names"] == ["qr_lq_sweep", "qr_svd_precond"]
    assert abs(r["ms_per_step"] - (6063.1 + 2774.4)) < 1e-9
    assert abs(r["achieved"] - 4.0e16 / ((6063.1 + 2774.4) / 1e3) / 1e12) < 1e-9
    assert abs(r["peak"] - 152 * 128 * 2 * 2070e6 / 1e12) < 1e-9
    assert r["frac"] == r["achieved"] / r["peak"]


def test_traffic_scaled_by_matrices_and_tied_to_source(tmp_path, monkeypatch):
    src = tmp_path / "k.cu"
    src.write_text("kernel v1")
    sha = hashlib.sha1(src.read_bytes()).hexdigest()
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "dram_traffic_per_unit.txt").write_text(f"k_qr 1000 matrix k.cu {sha}\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.ncu_traffic("k_qr", 320.0) == 320000.0
    assert bench.ncu_traffic("k_jacobi_select", 320.0) is None
    assert bench.ncu_traffic("k_qr", None) is None
    src.write_text("kernel v2")  # the kernel changed after the counters were taken
    assert bench.ncu_traffic("k_qr", 320.0) is None


def test_flop_model_counts_the_applied_terms():
    from paper_2409_12708_gb300.workloads import WORKLOADS
    w = WORKLOADS["L16_N48_D128"]
    N, T = w["N"], 4 * w["N"] ** 2 + 2 * w["L"]
    full, c_full = bench.flop_models(w, 128)
    part, c_part = bench.flop_models(w, 128, 608)
    # 2 layers for each of the 2N reuse blocks, 2 per term, T - 1 additions
    assert c_full == 2 * (2 * N) + 2 * T + (T - 1)
    assert c_part == 2 * 7 + 2 * 608 + 607  # 608 terms touch ceil(608 / 96) = 7 blocks
    for k in full:
        assert abs(part[k] / full[k] - c_part / c_full) < 1e-12

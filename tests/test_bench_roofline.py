"""Host logic of bench.py's roofline object (no GPU): profile names are grouped
into the work units of the flop model (Householder QR of the QR sweep; sigma
and V of the SVD sweep; contractions), the dominant unit is reported against
a peak derived from the device's SM count, and the ncu traffic figure is
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


def test_flop_units_follow_golub_van_loan():
    # Householder QR without Q: 2mn^2 - 2n^3/3 (m >= n); the wide case is the transpose
    assert bench.qr_flops(1024, 256) == 2 * 1024 * 256 ** 2 - 2 * 256 ** 3 / 3
    assert abs(bench.qr_flops(256, 1024) - bench.qr_flops(1024, 256)) < 1e-3
    assert bench.qr_flops(1, 1) == 4 - 4 + 4 / 3  # one reflector on one entry
    # sigma and V: 4mn^2 + 8n^3
    assert bench.svd_flops(512, 256) == 4 * 512 * 256 ** 2 + 8 * 256 ** 3
    assert bench.svd_flops(256, 512) == bench.svd_flops(512, 256)


def test_dominant_unit_groups_precond_qr_with_jacobi():
    prof, stats = _prof()
    models = {"svd": 5.0e16, "qr": 3.0e16, "gemm": 1e16}
    r = bench.roofline(prof, stats, models, {"sm_mhz": 2070.0}, sms=148,
                       peaks={"bf16_tflops_sustained": 1700.0})
    assert r["work_unit"] == "svd"
    assert r["by_unit"]["svd"]["profile_names"] == ["jacobi_svd", "qr_svd_precond"]
    assert abs(r["ms_per_step"] - (8361.6 + 2774.4)) < 1e-9
    assert abs(r["achieved"] - 5.0e16 / ((8361.6 + 2774.4) / 1e3) / 1e12) < 1e-9
    assert abs(r["peak"] - 148 * 128 * 2 * 2070e6 / 1e12) < 1e-9  # SM count from the device
    assert r["frac"] == r["achieved"] / r["peak"]
    assert r["peak_tensor_tf32"] == 850.0
    qr = r["by_unit"]["qr"]
    assert abs(qr["achieved_tflops"] - 3.0e16 / 6.0631 / 1e12) < 1e-9
    # a TF32 rate measured in the run replaces the BF16-derived estimate
    r2 = bench.roofline(prof, stats, models, {"sm_mhz": 2070.0}, sms=148,
                        peaks={"bf16_tflops_sustained": 1700.0}, tf32_measured=1000.0)
    assert r2["peak_tensor_tf32"] == 1000.0 and r2["frac_tensor_tf32"] == r2["achieved"] / 1000.0
    assert "measured cuBLAS TF32" in r2["peak_note"]


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
    # per compression at D = 128 the sites at full bond count about L - 7 full-size
    # units (edge sites with smaller bonds as fractions): 8 to 9 QRs of 1024 x 256
    # and SVDs of 512 x 256
    assert 8 < full["qr"] / c_full / bench.qr_flops(1024, 256) < 9
    assert 8 < full["svd"] / c_full / bench.svd_flops(512, 256) < 9

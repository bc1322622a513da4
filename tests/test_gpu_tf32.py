"""The TF32 path: float32 storage with the compression's contractions on the
tensor cores (tcgen05, error-compensated 3xTF32).  It must keep the float32
path's accuracy: the same tolerances as the float32 tests (untruncated layer
against the dense operator 2e-6, truncated results against the oracle 1e-5),
and agree with the float32 SIMT path at the same level on the full-size
workload.  The profile shows that the contractions ran on the tensor cores."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import mps as OM  # noqa: E402
from oracle import thc as OT  # noqa: E402
from paper_2409_12708_gb300.workloads import random_mps, sector_mps, workload  # noqa: E402


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2409_12708_gb300 import binding
    return binding


def dev(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype)


def to_np(sites):
    return [s.detach().cpu().double().numpy() for s in sites]


def test_tf32_layer_untruncated_equals_dense_and_uses_tensor_cores(B):
    L = 6
    psi = random_mps(L, 64, seed=2)
    coef = np.random.default_rng(7).standard_normal(L)
    B.profile_read()
    B.profile_enable(True)
    out = B.thc_layer_apply([dev(a, torch.float32) for a in psi], dev(coef), 0, 1, D_max=64, path="tf32")
    torch.cuda.synchronize()
    prof = B.profile_read()
    B.profile_enable(False)
    ref = OM.mpo_to_dense(OM.ladder_mpo(coef, 0, True)) @ OM.to_dense(psi)
    got = OM.to_dense(to_np(out))
    assert np.linalg.norm(got - ref) <= 2e-6 * np.linalg.norm(ref)
    assert prof.get("tc_gemm_launches", {}).get("launches", 0) > 0


def test_tf32_apply_H_truncated_matches_oracle(B):
    t, chi, zeta, psi, D = workload("L6_N12_D16")
    out = B.thc_apply_H(dev(t), dev(chi), dev(zeta), [dev(a, torch.float32) for a in psi], D_max=D, path="tf32")
    ref = OT.apply_H(psi, t, chi, zeta, D_max=D)
    va, vb = OM.to_dense(to_np(out)), OM.to_dense(ref)
    assert np.linalg.norm(va - vb) < 1e-5 * np.linalg.norm(vb)


def test_tf32_as_accurate_as_fp32_at_full_size(B):
    # L = 16, N = 48, D_max = 128: 16 terms (one reuse state, 16 x 2 layers,
    # the tree); both float32-storage paths against the float64 path, compared
    # through float64 inner products on the device.  Both land between 5e-5
    # and 1.2e-4 (mostly rounding noise in other particle-number sectors,
    # which dense tensors do not exclude, amplified through the compressions):
    # where in that range depends on the order of rounding, and the TF32
    # path's order varies from process to process because the GEMM autotuner
    # picks the tensor-core or the SIMT kernel per shape by timing.  Measured:
    # float32 5.6e-5 to 5.8e-5, TF32 5.2e-5 to 1.18e-4.  Both paths are held
    # to the same bound.
    t, chi, zeta, psi, D = workload("L16_N48_D128")
    H = (dev(t), dev(chi), dev(zeta))
    p32 = [dev(a, torch.float32) for a in psi]
    ref = B.thc_apply_H(*H, [dev(a) for a in psi], D_max=D, term_begin=0, term_end=16)

    def dist(x):
        x = [v.double() for v in x]
        aa, xx, ax = B.mps_inner(ref, ref), B.mps_inner(x, x), B.mps_inner(ref, x)
        return np.sqrt(max(aa + xx - 2 * ax, 0.0) / aa)

    e32 = dist(B.thc_apply_H(*H, p32, D_max=D, path="fp32", term_begin=0, term_end=16))
    etf = dist(B.thc_apply_H(*H, p32, D_max=D, path="tf32", term_begin=0, term_end=16))
    assert e32 < 2e-4
    assert etf < 2e-4


def test_tf32_block_sparse_state_at_tiny_scale(B):
    # the split a = a_hi + a_lo must survive entries near the float32 underflow
    # range like the SIMT path (compare test_compress_block_sparse_fp32_at_any_scale)
    L = 7
    psi = sector_mps(L, 3, 4, 16, seed=77)
    psi[-1] = psi[-1] * 1e-20
    out = B.thc_compress([dev(a, torch.float32) for a in psi], D_max=7, path="tf32")
    ref = OM.compress(psi, 7)
    va, vb = OM.to_dense(to_np(out)), OM.to_dense(ref)
    assert np.linalg.norm(va - vb) < 1e-5 * np.linalg.norm(vb)

"""Complex MPS through the C ABI (the states of a Krylov time evolution,
Sec. 2.2): every step with complex site tensors against the oracle (which runs
the same definitions in complex128) or the dense Fock-space operators.

Tolerances as for real states: float64 path untruncated 1e-10 (dense) and
truncated 1e-9 (gauge-invariant, dense vectors at L <= 8); the time step
untruncated against the oracle's Krylov step 1e-10, two steps against the
dense exp(-i dt H) 1e-8 (the oracle's own pin, App. A bound).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import fock as F  # noqa: E402
from oracle import krylov as OK  # noqa: E402
from oracle import mps as OM  # noqa: E402
from oracle import thc as OT  # noqa: E402
from paper_2409_12708_gb300.workloads import random_mps, sector_mps, thc_hamiltonian  # noqa: E402


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2409_12708_gb300 import binding
    return binding


CDT = {"fp64": torch.complex128, "fp32": torch.complex64}


def dev(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype)


def to_np(sites):
    return [s.detach().cpu().numpy().astype(np.complex128) for s in sites]


def complex_mps(L, D, seed, sector=None):
    """A complex MPS: real and imaginary parts from two seeded random MPS (of
    one sector when given, so that H keeps it in that sector)."""
    if sector:
        a = sector_mps(L, sector[0], sector[1], D, seed=seed)
        b = sector_mps(L, sector[0], sector[1], D, seed=seed + 1)
    else:
        a, b = random_mps(L, D, seed=seed), random_mps(L, D, seed=seed + 1)
    # a one-site phase keeps the state in the span of the two real ones
    out = [x.astype(np.complex128) for x in a]
    out[-1] = a[-1] + 0.7j * b[-1] if a[-1].shape == b[-1].shape else out[-1]
    mid = L // 2
    out[mid] = a[mid] * np.exp(0.3j) + 0.2j * b[mid]
    return out


def dense_rel(a, b):
    va, vb = OM.to_dense(a), OM.to_dense(b)
    return np.linalg.norm(va - vb) / max(np.linalg.norm(vb), 1e-300)


@pytest.mark.parametrize("sigma,dagger", [(0, 0), (1, 1)])
def test_complex_layer_untruncated_equals_dense_operator(B, sigma, dagger):
    L = 5
    psi = complex_mps(L, 16, seed=3)
    coef = np.random.default_rng(7).standard_normal(L)
    out = B.thc_layer_apply([dev(a, torch.complex128) for a in psi], dev(coef), sigma, dagger, D_max=256)
    ref = OM.mpo_to_dense(OM.ladder_mpo(coef, sigma, bool(dagger))) @ OM.to_dense(psi)
    got = OM.to_dense(to_np(out))
    assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)


@pytest.mark.parametrize("path,tolr", [("fp64", 1e-10), ("fp32", 2e-6)])
def test_complex_apply_H_untruncated_equals_dense(B, path, tolr):
    L, N = 4, 3
    t, chi, zeta = thc_hamiltonian(L, N, seed=14)
    psi = complex_mps(L, 256, seed=15, sector=(2, 2))
    ref = F.hamiltonian_eq1(t, F.thc_v(chi, zeta)) @ OM.to_dense(psi)
    out = B.thc_apply_H(dev(t), dev(chi), dev(zeta), [dev(a, CDT[path]) for a in psi], D_max=256, path=path)
    got = OM.to_dense(to_np(out))
    assert np.linalg.norm(got - ref) <= tolr * np.linalg.norm(ref)


def test_complex_compress_truncated_matches_oracle(B):
    L = 7
    psi = complex_mps(L, 16, seed=9, sector=(3, 4))
    for D, tol in [(5, 0.0), (16, 1e-2)]:
        out = B.thc_compress([dev(a, torch.complex128) for a in psi], D_max=D, tol=tol)
        ref = OM.compress(psi, D, tol)
        assert dense_rel(to_np(out), ref) < 1e-9


def test_complex_inner_conjugates_the_bra(B):
    L = 6
    a, b = complex_mps(L, 8, seed=1), complex_mps(L, 16, seed=5)
    got = B.mps_inner([dev(x, torch.complex128) for x in a], [dev(x, torch.complex128) for x in b])
    ref = OM.inner(a, b)
    assert isinstance(got, complex)
    assert abs(got - ref) <= 1e-13 * OM.norm(a) * OM.norm(b)
    assert abs(ref - np.vdot(OM.to_dense(a), OM.to_dense(b))) < 1e-10 * abs(ref)


def test_complex_add_compress_with_complex_coefficients(B):
    L = 6
    xs = [complex_mps(L, 16, seed=60 + 2 * i, sector=(3, 3)) for i in range(5)]
    cs = [1.0, -0.5j, 0.25 + 0.5j, 2.0, -1.5 + 0.1j]
    out = B.mps_add_compress(cs, [[dev(a, torch.complex128) for a in x] for x in xs], D_max=16)
    ref = OT.pairwise_sum([OM.scale(x, c) for x, c in zip(xs, cs)], 16, 0.0)
    assert dense_rel(to_np(out), ref) < 1e-9


def test_real_mps_rejects_complex_coefficients(B):
    xs = [[dev(a) for a in random_mps(4, 4, seed=i)] for i in range(2)]
    with pytest.raises(B.ThcError) as e:
        B.mps_add_compress([1.0, 1j], xs, D_max=4)
    assert e.value.status == B.EINVAL


# ------------------------------------------------------------------ the time step (a8)
def _setup(L=3, N=3, seed=20):
    t, chi, zeta = thc_hamiltonian(L, N, seed=seed)
    H = F.hamiltonian_eq1(t, F.thc_v(chi, zeta))
    psi = sector_mps(L, 1, 2, 64, seed=seed + 1)
    Hop = lambda x: OT.apply_H(x, t, chi, zeta, D_max=10 ** 6, tol=0.0)
    return t, chi, zeta, H, psi, Hop


@pytest.mark.parametrize("K", [3, 5])
def test_expm_step_untruncated_matches_oracle(B, K):
    t, chi, zeta, H, psi, Hop = _setup()
    dt = 0.05
    out, lost = B.krylov_expm_apply(dev(t), dev(chi), dev(zeta), [dev(a) for a in psi], dt, K, D_max=64)
    ref, lost_ref = OK.krylov_expm_step(Hop, psi, dt, K, D_max=10 ** 6)
    assert out[0].dtype == torch.complex128
    assert dense_rel(to_np(out), ref) < 1e-10
    assert lost < 1e-10 and lost_ref < 1e-10


def test_two_complex_expm_steps_match_dense_exponential(B):
    # step 2 starts from the complex output of step 1
    t, chi, zeta, H, psi, _ = _setup()
    args = (dev(t), dev(chi), dev(zeta))
    x, _ = B.krylov_expm_apply(*args, [dev(a) for a in psi], 0.03, 6, D_max=64)
    x, _ = B.krylov_expm_apply(*args, x, 0.03, 6, D_max=64)
    import scipy.linalg as sla
    ref = sla.expm(-1j * 0.06 * H.toarray()) @ OM.to_dense(psi)
    assert np.linalg.norm(OM.to_dense(to_np(x)) - ref) < 1e-8


def test_expm_step_from_complex_state_matches_oracle(B):
    # a complex start state: complex Krylov vectors, complex Htil and S
    L, N = 4, 3
    t, chi, zeta = thc_hamiltonian(L, N, seed=31)
    psi = complex_mps(L, 16, seed=32, sector=(2, 2))
    Hop = lambda x: OT.apply_H(x, t, chi, zeta, D_max=256, tol=0.0)
    out, lost = B.krylov_expm_apply(dev(t), dev(chi), dev(zeta), [dev(a, torch.complex128) for a in psi], 0.1, 4,
                                    D_max=256)
    ref, _ = OK.krylov_expm_step(Hop, psi, 0.1, 4, D_max=256)
    assert dense_rel(to_np(out), ref) < 1e-10


def test_expm_step_truncated_matches_oracle(B):
    # D_max = 8 at L = 6 from a state with decaying Schmidt values
    L, N, D = 6, 6, 8
    t, chi, zeta = thc_hamiltonian(L, N, seed=0)
    psi = sector_mps(L, 3, 3, 8, seed=1000, decay=1.0)
    Hop = lambda x: OT.apply_H(x, t, chi, zeta, D_max=D)
    out, lost = B.krylov_expm_apply(dev(t), dev(chi), dev(zeta), [dev(a) for a in psi], 0.05, 4, D_max=D)
    ref, lost_ref = OK.krylov_expm_step(Hop, psi, 0.05, 4, D_max=D)
    assert dense_rel(to_np(out), ref) < 1e-9
    assert abs(lost - lost_ref) < 1e-9


def test_expm_step_fp32_path(B):
    t, chi, zeta, H, psi, Hop = _setup()
    out, _ = B.krylov_expm_apply(dev(t), dev(chi), dev(zeta), [dev(a, torch.float32) for a in psi], 0.05, 4,
                                 D_max=64, path="fp32")
    ref, _ = OK.krylov_expm_step(Hop, psi, 0.05, 4, D_max=10 ** 6)
    assert out[0].dtype == torch.complex64
    assert dense_rel(to_np(out), ref) < 2e-6


def test_lanczos_from_complex_start_equals_real(B):
    # a global phase on the start state changes nothing in exact arithmetic
    L, N, D, K = 5, 4, 256, 6
    t, chi, zeta = thc_hamiltonian(L, N, seed=30)
    psi = sector_mps(L, 2, 3, 16, seed=31)
    args = (dev(t), dev(chi), dev(zeta))
    e_r, _, _ = B.krylov_lanczos_ground(*args, [dev(a) for a in psi], K, D_max=D)
    pc = [a.astype(np.complex128) for a in psi]
    pc[0] = pc[0] * np.exp(0.4j)
    e_c, _, _ = B.krylov_lanczos_ground(*args, [dev(a, torch.complex128) for a in pc], K, D_max=D)
    assert abs(e_r - e_c) < 1e-9

"""The adjoint through the C ABI: exact <phi|H|psi> and its derivatives with
respect to t, chi, zeta and psi's sites (thc_expect_grad), against the
oracle's dense gradients at L = 6, N = 12 (float64, relative 1e-10), against
central finite differences of the GPU's own value (step 1e-5, relative 1e-6,
float64), through torch.autograd, and float32 against float64."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import grad as OG  # noqa: E402
from oracle import mps as OM  # noqa: E402
from paper_2409_12708_gb300.workloads import sector_mps, thc_hamiltonian  # noqa: E402


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2409_12708_gb300 import binding
    return binding


def dev(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype)


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def test_adjoint_matches_dense_oracle_L6_N12(B):
    L, N = 6, 12
    t, chi, zeta = thc_hamiltonian(L, N, seed=0)
    phi = sector_mps(L, 3, 3, 16, seed=2001)
    psi = sector_mps(L, 3, 3, 16, seed=2002)
    v, dt, dchi, dz, dpsi = B.thc_expect_grad(dev(t), dev(chi), dev(zeta), [dev(a) for a in phi],
                                              [dev(a) for a in psi])
    vphi, vpsi = OM.to_dense(phi), OM.to_dense(psi)
    ref = OG.expectation(vphi, vpsi, t, chi, zeta)
    rt, rc, rz, rpsi = OG.gradients(vphi, vpsi, t, chi, zeta)
    assert abs(v - ref) < 1e-12 * abs(ref)
    assert rel(dt.cpu().numpy(), rt) < 1e-10
    assert rel(dchi.cpu().numpy(), rc) < 1e-10
    assert rel(dz.cpu().numpy(), rz) < 1e-10
    for i in range(L):
        assert rel(dpsi[i].cpu().numpy(), OG.site_gradient(rpsi, psi, i)) < 1e-10


def test_adjoint_finite_differences_L8_N16_D32(B):
    L, N, D = 8, 16, 32
    t, chi, zeta = thc_hamiltonian(L, N, seed=3)
    phi = [dev(a) for a in sector_mps(L, 4, 4, D, seed=2003)]
    psi = [dev(a) for a in sector_mps(L, 4, 4, D, seed=2004)]
    T, X, Z = dev(t), dev(chi), dev(zeta)
    _, dt, dchi, dz, dpsi = B.thc_expect_grad(T, X, Z, phi, psi)
    E = lambda tt, xx, zz, pp: B.thc_expect_grad(tt, xx, zz, phi, pp, grads=False)
    rng = np.random.default_rng(7)
    h = 1e-5

    def fd(arr, idx, call):
        p, m = arr.clone(), arr.clone()
        p[idx] += h
        m[idx] -= h
        return (call(p) - call(m)) / (2 * h)

    def close(a, b):
        return abs(a - b) <= 1e-6 * max(abs(b), 1e-2)

    for _ in range(4):
        i = tuple(int(x) for x in rng.integers(L, size=2))
        assert close(float(dt[i]), fd(T, i, lambda x: E(x, X, Z, psi)))
        i = (int(rng.integers(L)), int(rng.integers(N)))
        assert close(float(dchi[i]), fd(X, i, lambda x: E(T, x, Z, psi)))
        i = tuple(int(x) for x in rng.integers(N, size=2))
        assert close(float(dz[i]), fd(Z, i, lambda x: E(T, X, x, psi)))
        s = int(rng.integers(L))
        i = tuple(int(rng.integers(n)) for n in psi[s].shape)
        assert close(float(dpsi[s][i]), fd(psi[s], i, lambda x: E(T, X, Z, psi[:s] + [x] + psi[s + 1:])))


def test_adjoint_through_torch_autograd(B):
    L, N = 6, 8
    t, chi, zeta = thc_hamiltonian(L, N, seed=5)
    T, X, Z = dev(t).requires_grad_(), dev(chi).requires_grad_(), dev(zeta).requires_grad_()
    phi = [dev(a) for a in sector_mps(L, 3, 3, 16, seed=2005)]
    psi = [dev(a).requires_grad_() for a in sector_mps(L, 3, 3, 16, seed=2006)]
    e = B.expectation(T, X, Z, phi, psi)
    (2.5 * e).backward()
    v, dt, dchi, dz, dpsi = B.thc_expect_grad(T.detach(), X.detach(), Z.detach(), phi,
                                              [x.detach() for x in psi])
    assert abs(float(e) - v) < 1e-14 * abs(v)  # float64 atomics: summation order may differ
    assert torch.allclose(T.grad, 2.5 * dt) and torch.allclose(X.grad, 2.5 * dchi) and torch.allclose(Z.grad, 2.5 * dz)
    assert all(torch.allclose(a.grad, 2.5 * b) for a, b in zip(psi, dpsi))


def test_adjoint_fp32_matches_fp64(B):
    L, N, D = 8, 16, 32
    t, chi, zeta = thc_hamiltonian(L, N, seed=3)
    phi = sector_mps(L, 4, 4, D, seed=2003)
    psi = sector_mps(L, 4, 4, D, seed=2004)
    r64 = B.thc_expect_grad(dev(t), dev(chi), dev(zeta), [dev(a) for a in phi], [dev(a) for a in psi])
    r32 = B.thc_expect_grad(dev(t), dev(chi), dev(zeta), [dev(a, torch.float32) for a in phi],
                            [dev(a, torch.float32) for a in psi], path="fp32")
    assert abs(r32[0] - r64[0]) < 1e-5 * abs(r64[0])
    for a, b in zip(r32[1:4], r64[1:4]):
        assert rel(a.cpu().numpy(), b.cpu().numpy()) < 1e-5
    assert max(rel(a.double().cpu().numpy(), b.cpu().numpy()) for a, b in zip(r32[4], r64[4])) < 1e-5

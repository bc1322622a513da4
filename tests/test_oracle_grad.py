"""Pins of the oracle's derivatives of <phi|H|psi> (no GPU): every analytic
derivative against central finite differences of the oracle's own dense
expectation value (step 1e-5, relative 1e-6), on random entries of t, chi,
zeta and of psi's MPS sites, plus special cases with a closed form."""
import numpy as np

from oracle import fock as F
from oracle import grad as G
from oracle import mps as M
from paper_2409_12708_gb300.workloads import sector_mps, thc_hamiltonian

L, N = 4, 5


def _setup():
    t, chi, zeta = thc_hamiltonian(L, N, seed=7)
    phi = sector_mps(L, 2, 2, 16, seed=8)
    psi = sector_mps(L, 2, 2, 16, seed=9)
    return t, chi, zeta, phi, psi


def _fd(f, x, idx, h=1e-5):
    xp, xm = x.copy(), x.copy()
    xp[idx] += h
    xm[idx] -= h
    return (f(xp) - f(xm)) / (2 * h)


def _close(a, b, tol=1e-6):
    return abs(a - b) <= tol * max(abs(b), 1e-3)


def test_gradients_match_finite_differences():
    t, chi, zeta, phi, psi = _setup()
    vphi, vpsi = M.to_dense(phi), M.to_dense(psi)
    dt, dchi, dzeta, dpsi = G.gradients(vphi, vpsi, t, chi, zeta)
    rng = np.random.default_rng(0)
    E = lambda tt, cc, zz: G.expectation(vphi, vpsi, tt, cc, zz)
    for _ in range(6):
        p, q = rng.integers(L, size=2)
        assert _close(dt[p, q], _fd(lambda x: E(x, chi, zeta), t, (p, q)))
        p, k = rng.integers(L), rng.integers(N)
        assert _close(dchi[p, k], _fd(lambda x: E(t, x, zeta), chi, (p, k)))
        m, n = rng.integers(N, size=2)
        assert _close(dzeta[m, n], _fd(lambda x: E(t, chi, x), zeta, (m, n)))
    # psi's sites: E is linear in each site, so the site gradient contracts dE/dpsi
    H = F.hamiltonian_eq1(t, F.thc_v(chi, zeta))
    for i in (0, 2, L - 1):
        g = G.site_gradient(dpsi, psi, i)
        assert g.shape == psi[i].shape
        for _ in range(4):
            idx = tuple(rng.integers(s) for s in psi[i].shape)
            f = lambda x: float(vphi @ (H @ M.to_dense(psi[:i] + [x] + psi[i + 1:])))
            assert _close(g[idx], _fd(f, psi[i], idx))


def test_gradient_closed_forms():
    t, chi, zeta, phi, psi = _setup()
    vphi, vpsi = M.to_dense(phi), M.to_dense(psi)
    dt, dchi, dzeta, dpsi = G.gradients(vphi, vpsi, t, chi, zeta)
    # E is linear in t and in zeta: Euler's theorem for homogeneous parts
    E = G.expectation(vphi, vpsi, t, chi, zeta)
    assert abs(np.sum(dt * t) + np.sum(dzeta * zeta) - E) < 1e-10 * abs(E)
    # E_V is homogeneous of degree 4 in chi: sum chi dE/dchi = 4 E_V
    EV = G.expectation(vphi, vpsi, 0 * t, chi, zeta)
    assert abs(np.sum(dchi * chi) - 4 * EV) < 1e-10 * abs(EV)
    # phi = psi: dE/dt is the one-particle density matrix, trace = particle number 4
    dtt, _, _, _ = G.gradients(vpsi, vpsi, t, chi, zeta)
    assert abs(np.trace(dtt) / (vpsi @ vpsi) - 4.0) < 1e-12

"""Pins of the oracle's global Krylov methods (Sec. 2.2, App. A), no GPU."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import fock as F
from oracle import krylov as KR
from oracle import mps as M
from oracle import thc as TH
from paper_2409_12708_gb300.workloads import sector_mps, thc_hamiltonian


def _setup(L=3, N=3, seed=20):
    t, chi, zeta = thc_hamiltonian(L, N, seed=seed)
    H = F.hamiltonian_eq1(t, F.thc_v(chi, zeta))
    psi = sector_mps(L, 1, 2, 64, seed=seed + 1)
    Hop = lambda x: TH.apply_H(x, t, chi, zeta, D_max=10 ** 6, tol=0.0)
    return t, chi, zeta, H, psi, Hop


def _dense_lanczos_ritz(H, v0, K):
    """Textbook Lanczos with full reorthogonalisation on dense vectors."""
    V = [v0 / np.linalg.norm(v0)]
    for k in range(K - 1):
        w = H @ V[k]
        for v in V:
            w = w - np.dot(v, w) * v
        for v in V:
            w = w - np.dot(v, w) * v
        V.append(w / np.linalg.norm(w))
    Vm = np.array(V).T
    return np.linalg.eigvalsh(Vm.T @ (H @ Vm))


def test_lanczos_small_K_matches_dense_lanczos():
    _, _, _, H, psi, Hop = _setup()
    K = 5
    e, _, _ = KR.lanczos_ground(Hop, psi, K, D_max=10 ** 6)
    ref = _dense_lanczos_ritz(H.toarray(), M.to_dense(psi), K)
    assert np.allclose(e, ref, atol=1e-10)


def test_lanczos_full_krylov_space_gives_ED():
    L = 3
    _, _, _, H, psi, Hop = _setup(L=L)
    dim = len(F.sector(L, 1, 2))  # 3 * 3 = 9 states
    e, c, v = KR.lanczos_ground(Hop, psi, dim + 2, D_max=10 ** 6)
    assert len(v) == dim  # the exhausted Krylov space is detected (breakdown)
    assert np.isclose(e[0], F.ground_energy(H, L, 1, 2), atol=1e-9)
    # the Ritz vector is an eigenvector of the dense H
    x = sum(c[i] * M.to_dense(v[i]) for i in range(len(v)))
    x /= np.linalg.norm(x)
    assert np.linalg.norm(H @ x - e[0] * x) < 1e-7


def _hochbruck_lubich(W, dt, K):
    """App. A, Eq. error_bond, for the shifted operator with spectrum in [-W, 0]."""
    wd = W * dt
    if K >= wd / 2:
        return 10.0 / (wd / 4) * np.exp(-wd / 4) * (np.e * wd / (4 * K)) ** K
    if np.sqrt(wd) <= K:
        return 10.0 * np.exp(-4 * K * K / (5 * wd))
    return np.inf


@pytest.mark.parametrize("K", [3, 4, 5])
def test_krylov_step_within_hochbruck_lubich_bound(K):
    L = 3
    _, _, _, H, psi, Hop = _setup(L=L)
    dt = 0.05
    out, lost = KR.krylov_expm_step(Hop, psi, dt, K, D_max=10 ** 6)
    ref = F.expm_apply(H, M.to_dense(psi), dt)
    err = np.linalg.norm(M.to_dense(out) - ref)
    s = F.sector(L, 1, 2)
    ev = np.linalg.eigvalsh(H[s][:, s].toarray())
    W = ev[-1] - ev[0]
    assert err <= _hochbruck_lubich(W, dt, K)
    assert lost < 1e-10


def test_krylov_step_error_scales_as_dt_power_K():
    L = 3
    _, _, _, H, psi, Hop = _setup(L=L)
    K = 3
    errs = []
    dts = [0.04, 0.02]
    for dt in dts:
        out, _ = KR.krylov_expm_step(Hop, psi, dt, K, D_max=10 ** 6)
        errs.append(np.linalg.norm(M.to_dense(out) - F.expm_apply(H, M.to_dense(psi), dt)))
    order = np.log(errs[0] / errs[1]) / np.log(dts[0] / dts[1])
    assert order > K - 0.3  # local error O(dt^K)


def test_two_steps_complex_state_unitary():
    L = 3
    _, _, _, H, psi, Hop = _setup(L=L)
    x, _ = KR.krylov_expm_step(Hop, psi, 0.03, 6, D_max=10 ** 6)
    x, _ = KR.krylov_expm_step(Hop, x, 0.03, 6, D_max=10 ** 6)
    ref = sla.expm(-1j * 0.06 * H.toarray()) @ M.to_dense(psi)
    assert np.iscomplexobj(x[-1])
    assert np.linalg.norm(M.to_dense(x) - ref) < 1e-8

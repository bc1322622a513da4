"""Pins of the dense Fock-space oracle against what the paper and textbook
second quantisation fix (no GPU)."""
import os

import numpy as np
import pytest

from oracle import fock as F
from oracle import mps as M
from paper_2409_12708_gb300.workloads import thc_hamiltonian

GOLD = os.path.join(os.path.dirname(__file__), "golden", "app_c_local_ops.txt")


def _golden_c():
    for line in open(GOLD):
        if line.startswith("c "):
            return np.array([float(x) for x in line.split()[1:]]).reshape(2, 2)
    raise AssertionError("no c in golden file")


def test_app_c_local_operators_match_printed_form():
    c = _golden_c()
    Z = np.diag([1.0, -1.0])
    assert np.array_equal(M.C2, c)
    assert np.array_equal(M.B_UP, np.kron(c, np.eye(2)))
    assert np.array_equal(M.B_DN, np.kron(Z, c))
    # one site: the full-space JW annihilators are exactly b_up, b_dn
    a = F.mode_annihilators(1)
    assert np.array_equal(a[0][0].toarray(), M.B_UP)
    assert np.array_equal(a[0][1].toarray(), M.B_DN)


def test_canonical_anticommutation_relations():
    L = 3
    a = F.mode_annihilators(L)
    ops = [a[p][s].toarray() for p in range(L) for s in range(2)]
    I = np.eye(4 ** L)
    for i, ai in enumerate(ops):
        for j, aj in enumerate(ops):
            acomm = ai @ aj.T + aj.T @ ai
            assert np.allclose(acomm, I if i == j else 0.0, atol=0)
            assert np.allclose(ai @ aj + aj @ ai, 0.0, atol=0)


def test_hamiltonian_hermitian_and_conserves_spin_numbers():
    L, N = 4, 5
    t, chi, zeta = thc_hamiltonian(L, N, seed=3)
    H = F.hamiltonian_eq1(t, F.thc_v(chi, zeta))
    Hd = H.toarray()
    assert np.allclose(Hd, Hd.T, atol=1e-12)
    nu, nd = F.number_ops(L)
    assert abs(H @ nu - nu @ H).max() < 1e-12
    assert abs(H @ nd - nd @ H).max() < 1e-12


def test_thc_v_has_eightfold_symmetry():
    L, N = 5, 7
    _, chi, zeta = thc_hamiltonian(L, N, seed=4)
    v = F.thc_v(chi, zeta)
    assert np.allclose(v, v.transpose(1, 0, 2, 3))  # p <-> q
    assert np.allclose(v, v.transpose(0, 1, 3, 2))  # r <-> s
    assert np.allclose(v, v.transpose(2, 3, 0, 1))  # (pq) <-> (rs)
    # and it is the four-fold chi contraction of Eq. thc, checked entrywise
    p, q, r, s = 1, 3, 0, 4
    ref = sum(chi[p, m] * chi[q, m] * zeta[m, n] * chi[r, n] * chi[s, n]
              for m in range(N) for n in range(N))
    assert np.isclose(v[p, q, r, s], ref)


def test_thc_subterms_sum_to_eq1():
    L, N = 3, 4
    t, chi, zeta = thc_hamiltonian(L, N, seed=5)
    a = F.mode_annihilators(L)
    H1 = F.hamiltonian_eq1(t, F.thc_v(chi, zeta), a).toarray()
    H2 = F.hamiltonian_thc(t, chi, zeta, a).toarray()
    assert np.allclose(H1, H2, atol=1e-12)
    # G_{mu s, nu s'} = zeta^{mu nu} G_{mu s} G_{nu s'}
    mu, nu = 1, 2
    for s in range(2):
        for sp in range(2):
            G = F.thc_subterm(chi, zeta, mu, s, nu, sp, a).toarray()
            Gm = (F.ladder_operator(chi[:, mu], s, True, a) @ F.ladder_operator(chi[:, mu], s, False, a)).toarray()
            Gn = (F.ladder_operator(chi[:, nu], sp, True, a) @ F.ladder_operator(chi[:, nu], sp, False, a)).toarray()
            assert np.allclose(G, zeta[mu, nu] * Gm @ Gn, atol=1e-13)


def test_free_fermions_closed_form():
    # zeta = 0: ground energy in (N_up, N_dn) is the sum of the lowest orbital energies
    L, N = 4, 3
    t, chi, _ = thc_hamiltonian(L, N, seed=6)
    H = F.hamiltonian_eq1(t, F.thc_v(chi, np.zeros((N, N))))
    eps = np.sort(np.linalg.eigvalsh(t))
    for nu, nd in [(1, 1), (2, 1), (2, 2), (3, 1)]:
        assert np.isclose(F.ground_energy(H, L, nu, nd), eps[:nu].sum() + eps[:nd].sum(), atol=1e-12)


def test_hubbard_reduction():
    # chi = I (N = L), zeta = U I  =>  V = U sum_p n_pu n_pd + (U/2) N_total
    L, U = 3, 1.7
    t, _, _ = thc_hamiltonian(L, L, seed=7)
    a = F.mode_annihilators(L)
    H = F.hamiltonian_eq1(t, F.thc_v(np.eye(L), U * np.eye(L)), a).toarray()
    H0 = F.hamiltonian_eq1(t, np.zeros((L, L, L, L)), a).toarray()
    n = [[(a[p][s].T @ a[p][s]).toarray() for s in range(2)] for p in range(L)]
    Ntot = sum(n[p][s] for p in range(L) for s in range(2))
    V = U * sum(n[p][0] @ n[p][1] for p in range(L)) + 0.5 * U * Ntot
    assert np.allclose(H - H0, V, atol=1e-12)


@pytest.mark.parametrize("U,tau", [(0.0, 1.0), (1.0, 1.0), (4.0, 0.5), (8.0, 1.3)])
def test_hubbard_dimer_closed_form(U, tau):
    t = np.array([[0.0, -tau], [-tau, 0.0]])
    H = F.hamiltonian_eq1(t, F.thc_v(np.eye(2), U * np.eye(2)))
    e0 = F.ground_energy(H, 2, 1, 1)
    assert np.isclose(e0, U / 2 - np.sqrt(U * U / 4 + 4 * tau * tau) + U, atol=1e-12)


def test_config0_golden_energies_are_current():
    """tests/golden/config0_energies.txt (read by bench.py's Krylov record)
    equals a fresh oracle computation; 40 dense Lanczos steps reach ED."""
    import importlib.util
    path = os.path.join(os.path.dirname(__file__), "golden", "make_config0_energies.py")
    spec = importlib.util.spec_from_file_location("mk0", path)
    mk = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mk)
    stored, fresh = mk.read(), mk.compute()
    for k in fresh:
        assert abs(stored[k] - fresh[k]) < 1e-11
    assert abs(fresh["dense_lanczos_K40"] - fresh["ed_ground_energy"]) < 1e-9
    assert fresh["dense_lanczos_K10"] > fresh["ed_ground_energy"] + 0.1  # 10 steps are far from converged

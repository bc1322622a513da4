"""Pins of the spin-merged term list (symmetric zeta, Eq. thc; Eq. G).

The merge rests on two operator facts, checked here on dense Fock-space
matrices built from the definitions (oracle.fock): G_{mu up} and G_{nu down}
commute; two same-spin G do not, their commutator being
(chi^mu . chi^nu)(A+_mu A_nu - A+_nu A_mu).  The merged list is then pinned
against the dense Eq. 1 Hamiltonian (untruncated), against the unmerged list,
and by its enumeration."""
import numpy as np

from oracle import fock as F
from oracle import mps as M
from oracle import thc as TH
from paper_2409_12708_gb300.workloads import sector_mps, thc_hamiltonian


def _G(chi, k, s, a):
    return (F.ladder_operator(chi[:, k], s, True, a) @ F.ladder_operator(chi[:, k], s, False, a)).toarray()


def test_opposite_spin_one_body_operators_commute():
    L, N = 3, 3
    _, chi, _ = thc_hamiltonian(L, N, seed=3)
    a = F.mode_annihilators(L)
    for mu in range(N):
        for nu in range(N):
            gu, gd = _G(chi, mu, 0, a), _G(chi, nu, 1, a)
            assert np.abs(gu @ gd - gd @ gu).max() < 1e-12


def test_same_spin_commutator_closed_form():
    # [A+_m A_m, A+_n A_n] = (chi^m . chi^n) (A+_m A_n - A+_n A_m) for one spin
    L, N = 3, 2
    _, chi, _ = thc_hamiltonian(L, N, seed=4)
    a = F.mode_annihilators(L)
    for s in range(2):
        Ad = lambda k: F.ladder_operator(chi[:, k], s, True, a).toarray()
        An = lambda k: F.ladder_operator(chi[:, k], s, False, a).toarray()
        g0, g1 = _G(chi, 0, s, a), _G(chi, 1, s, a)
        comm = g0 @ g1 - g1 @ g0
        ref = float(chi[:, 0] @ chi[:, 1]) * (Ad(0) @ An(1) - Ad(1) @ An(0))
        assert np.abs(comm - ref).max() < 1e-12
        assert np.abs(comm).max() > 1e-3  # not zero: same-spin terms cannot merge


def test_merged_enumeration():
    L, N = 3, 4
    T = TH.n_terms(L, N, merge_spin=True)
    assert T == 3 * N * N + 2 * L
    seen = {}
    blocks = []
    for t in range(T):
        k = TH.decode_term_merged(t, L, N)
        if k[0] == "V":
            _, mu, s, nu, sp, f = k
            assert (mu, s, nu, sp) not in seen
            seen[(mu, s, nu, sp)] = f
            if not blocks or blocks[-1] != (nu, sp):
                blocks.append((nu, sp))
        else:
            assert t >= 3 * N * N
    # every (nu, s') block is contiguous, visited once, up blocks first
    assert len(blocks) == len(set(blocks)) == 2 * N
    assert blocks[:N] == [(nu, 0) for nu in range(N)]
    for mu in range(N):
        for nu in range(N):
            assert seen[(mu, 0, nu, 0)] == 1.0 and seen[(mu, 1, nu, 1)] == 1.0  # same spin kept
            assert seen[(mu, 0, nu, 1)] == 2.0                                 # merged pair
            assert (mu, 1, nu, 0) not in seen                                  # folded away


def test_merged_untruncated_equals_dense_H():
    L, N = 4, 3
    t, chi, zeta = thc_hamiltonian(L, N, seed=21)
    psi = sector_mps(L, 2, 2, 16, seed=22)
    ref = F.hamiltonian_eq1(t, F.thc_v(chi, zeta)) @ M.to_dense(psi)
    got = M.to_dense(TH.apply_H(psi, t, chi, zeta, D_max=10 ** 6, merge_spin=True))
    assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)


def test_merge_needs_symmetric_zeta():
    # with zeta != zeta^T the folded (mu down, nu up) terms carry zeta^{nu mu}
    # in the unmerged list and zeta^{mu nu} in the merged one
    L, N = 3, 2
    t, chi, zeta = thc_hamiltonian(L, N, seed=23)
    zeta = zeta + np.array([[0.0, 0.3], [-0.3, 0.0]])
    psi = sector_mps(L, 1, 2, 16, seed=24)
    a = M.to_dense(TH.apply_H(psi, t, chi, zeta, D_max=10 ** 6))
    b = M.to_dense(TH.apply_H(psi, t, chi, zeta, D_max=10 ** 6, merge_spin=True))
    assert np.linalg.norm(a - b) > 1e-3 * np.linalg.norm(a)


def test_merged_truncated_stays_close_to_unmerged():
    # truncated: the two lists differ by their truncation errors only
    L, N, D = 6, 3, 6
    t, chi, zeta = thc_hamiltonian(L, N, seed=25)
    psi = sector_mps(L, 3, 3, 6, seed=26, decay=1.0)
    a = M.to_dense(TH.apply_H(psi, t, chi, zeta, D_max=D))
    b = M.to_dense(TH.apply_H(psi, t, chi, zeta, D_max=D, merge_spin=True))
    exact = F.hamiltonian_eq1(t, F.thc_v(chi, zeta)) @ M.to_dense(psi)
    ea, eb = np.linalg.norm(a - exact), np.linalg.norm(b - exact)
    assert np.linalg.norm(a - b) <= 2.0 * (ea + eb) + 1e-12

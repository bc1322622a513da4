"""Pins of the oracle's MPS engine and Alg. 1 against the dense definition and
against properties that hold for any correct implementation (no GPU)."""
import numpy as np
import pytest

from oracle import fock as F
from oracle import mps as M
from oracle import thc as TH
from paper_2409_12708_gb300.workloads import random_mps, sector_mps, thc_hamiltonian


@pytest.mark.parametrize("sigma", [0, 1])
@pytest.mark.parametrize("dagger", [False, True])
def test_ladder_mpo_equals_dense_operator(sigma, dagger):
    # "contract the W matrices sequentially to verify the correctness" (Sec. 3.1)
    L = 4
    coef = np.random.default_rng(1).standard_normal(L)
    Wd = M.mpo_to_dense(M.ladder_mpo(coef, sigma, dagger))
    ref = F.ladder_operator(coef, sigma, dagger).toarray()
    assert np.allclose(Wd, ref, atol=1e-14)


def test_apply_mpo_matches_dense_matvec():
    L = 4
    rng = np.random.default_rng(2)
    A = random_mps(L, 8, seed=3)
    coef = rng.standard_normal(L)
    W = M.ladder_mpo(coef, 1, True)
    out = M.apply_mpo(W, A)
    assert [x.shape[0] for x in out[1:]] == [2 * a.shape[0] for a in A[1:]]
    assert np.allclose(M.to_dense(out), M.mpo_to_dense(W) @ M.to_dense(A), atol=1e-12)


def test_untruncated_compress_preserves_state_and_is_left_canonical():
    L = 5
    A = random_mps(L, 16, seed=4)
    W = M.ladder_mpo(np.random.default_rng(5).standard_normal(L), 0, False)
    X = M.apply_mpo(W, A)
    C = M.compress(X, D_max=10 ** 6)
    assert np.allclose(M.to_dense(C), M.to_dense(X), atol=1e-12)
    for s in C[:-1]:
        Dl, d, Dr = s.shape
        U = s.reshape(Dl * d, Dr)
        assert np.allclose(U.T @ U, np.eye(Dr), atol=1e-12)


def test_truncation_errors_add_in_quadrature():
    # From right-canonical form every SVD step discards an orthogonal piece, so
    # ||psi - psi'||^2 equals the sum of the discarded weights over all bonds.
    L = 5
    A = random_mps(L, 16, seed=6)
    C, disc = M.compress(A, D_max=5, return_discarded=True)
    err2 = np.linalg.norm(M.to_dense(A) - M.to_dense(C)) ** 2
    assert np.isclose(err2, sum(disc), rtol=1e-9)
    assert max(x.shape[2] for x in C) <= 5
    # psi' is the orthogonal projection: <psi'|psi - psi'> = 0
    v, w = M.to_dense(A), M.to_dense(C)
    assert abs(np.dot(w, v - w)) < 1e-10 * np.dot(v, v)


def test_two_site_truncation_is_the_best_rank_k_approximation():
    # L = 2: the compressed state is the Eckart-Young optimum.  Pinned without
    # an SVD: its norm^2 equals the top eigenvalue of M M^T found by power
    # iteration, and no random rank-1 state gets closer.
    rng = np.random.default_rng(7)
    Mx = rng.standard_normal((4, 4))
    A = [Mx.reshape(1, 4, 4), np.eye(4).reshape(4, 4, 1)]
    C = M.compress(A, D_max=1)
    G = Mx @ Mx.T
    x = np.ones(4)
    for _ in range(2000):
        x = G @ x
        x /= np.linalg.norm(x)
    lam = x @ G @ x
    w = M.to_dense(C)
    assert np.isclose(np.dot(w, w), lam, rtol=1e-10)
    best = np.linalg.norm(Mx.reshape(-1) - w)
    for _ in range(200):
        a, b = rng.standard_normal(4), rng.standard_normal(4)
        cand = np.outer(a, b)
        cand *= np.sum(cand * Mx) / np.sum(cand * cand)
        assert np.linalg.norm(Mx - cand) >= best - 1e-12


def test_truncation_rule_tol():
    s = np.array([1.0, 0.5, 0.1, 0.01, 0.0])
    assert M.keep_count(s, 10, 0.0) == 5
    assert M.keep_count(s, 3, 0.0) == 3
    # discarded weight of keeping 2 is 0.0101 <= tol^2 * 1.2601
    assert M.keep_count(s, 10, 0.1) == 2
    assert M.keep_count(s, 10, 1e-3) == 4
    assert M.keep_count(np.zeros(3), 10, 0.5) == 1


def test_direct_sum_and_inner():
    L = 4
    A = random_mps(L, 4, seed=8)
    B = [x.astype(np.complex128) * (1 + 0.5j) for x in random_mps(L, 8, seed=9)]
    S = M.direct_sum(A, B)
    assert np.allclose(M.to_dense(S), M.to_dense(A) + M.to_dense(B), atol=1e-12)
    assert np.isclose(M.inner(A, B), np.vdot(M.to_dense(A), M.to_dense(B)))
    assert np.isclose(M.inner(B, A), np.vdot(M.to_dense(B), M.to_dense(A)))


@pytest.mark.parametrize("L,N", [(3, 2), (4, 3)])
def test_untruncated_thc_apply_equals_dense_H(L, N):
    t, chi, zeta = thc_hamiltonian(L, N, seed=10 + L)
    psi = sector_mps(L, L // 2, (L + 1) // 2, 64, seed=11)
    H = F.hamiltonian_eq1(t, F.thc_v(chi, zeta))
    ref = H @ M.to_dense(psi)
    out = TH.apply_H(psi, t, chi, zeta, D_max=10 ** 6, tol=0.0)
    got = M.to_dense(out)
    assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)


def test_alg1_sequential_equals_pairwise_untruncated():
    L, N = 3, 3
    t, chi, zeta = thc_hamiltonian(L, N, seed=12)
    psi = sector_mps(L, 1, 2, 64, seed=13)
    a = TH.apply_V_alg1(psi, chi, zeta, 10 ** 6)
    b = TH.apply_H(psi, np.zeros((L, L)), chi, zeta, 10 ** 6, term_end=4 * N * N)
    ref = (F.hamiltonian_eq1(np.zeros((L, L)), F.thc_v(chi, zeta)) @ M.to_dense(psi))
    assert np.allclose(M.to_dense(a), ref, atol=1e-12)
    assert np.allclose(M.to_dense(b), ref, atol=1e-12)


def test_term_order_and_decode():
    L, N = 3, 4
    seen = set()
    for t in range(TH.n_terms(L, N)):
        k = TH.decode_term(t, L, N)
        if k[0] == "V":
            _, mu, s, nu, sp = k
            assert TH.coulomb_index(mu, s, nu, sp, N) == t
        seen.add(k)
    assert len(seen) == 4 * N * N + 2 * L
    assert TH.decode_term(1, L, N) == ("V", 1, 0, 0, 0)      # mu fastest
    assert TH.decode_term(N, L, N) == ("V", 0, 1, 0, 0)      # then sigma


def test_reduction_keeps_bond_at_D():
    L, N = 5, 2
    t, chi, zeta = thc_hamiltonian(L, N, seed=14)
    psi = sector_mps(L, 2, 2, 8, seed=15)
    out = TH.apply_H(psi, t, chi, zeta, D_max=8, tol=0.0)
    assert max(x.shape[2] for x in out) <= 8
    # the truncated result is still a good approximation of the exact H psi
    ref = F.hamiltonian_eq1(t, F.thc_v(chi, zeta)) @ M.to_dense(psi)
    rel = np.linalg.norm(M.to_dense(out) - ref) / np.linalg.norm(ref)
    assert rel < 0.5

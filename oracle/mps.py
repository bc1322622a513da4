"""CPU MPS engine for the oracle (float64 / complex128).

Test infrastructure only (see oracle/__init__.py).

An MPS is a Python list of L arrays A[i] of shape [chi_i, 4, chi_{i+1}] with
chi_0 = chi_L = 1 (Sec. 2.1, the MPS equation).  An MPO site is W[a, b, m, n]
with MPO bonds a, b and physical output/input indices m, n (Eq. MPO_def).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

# --- App. C: local operators on one spatial orbital (index 2*n_up + n_dn) -----
C2 = np.array([[0.0, 1.0], [0.0, 0.0]])
Z2 = np.diag([1.0, -1.0])
I2 = np.eye(2)
B_UP = np.kron(C2, I2)          # b_{s, up} = c (x) I2
B_DN = np.kron(Z2, C2)          # b_{s, dn} = Z (x) c
P_SITE = np.kron(Z2, Z2)        # Z (x) Z, the Jordan-Wigner string on one site
I4 = np.eye(4)


def local_annihilator(sigma: int) -> np.ndarray:
    return B_UP if sigma == 0 else B_DN


def ladder_mpo(coef: np.ndarray, sigma: int, dagger: bool):
    """MPO of sum_s coef_s a_{s,sigma} (or the creation version), bond dimension 2.

    Elementary-MPO equations with the Jordan-Wigner replacement: the bulk site
    is [[Z(x)Z, coef_s b_s], [0, I4]]; site 1 keeps only the first row and
    site L only the second column.  The creation operator uses b_s^T (App. C:
    creation operators are the conjugate transposes, and b is real).
    """
    L = coef.shape[0]
    b = local_annihilator(sigma)
    if dagger:
        b = b.T
    W = []
    for s in range(L):
        bulk = np.zeros((2, 2, 4, 4), dtype=np.result_type(coef, np.float64))
        bulk[0, 0] = P_SITE
        bulk[0, 1] = coef[s] * b
        bulk[1, 1] = I4
        if L == 1:
            W.append(bulk[0:1, 1:2].copy())
        elif s == 0:
            W.append(bulk[0:1, :].copy())
        elif s == L - 1:
            W.append(bulk[:, 1:2].copy())
        else:
            W.append(bulk)
    return W


def apply_mpo(W, A):
    """MPO x MPS by explicit loops over the MPO bonds and physical indices.

    out[(a, alpha), m, (b, beta)] = sum_n W[a, b, m, n] A[alpha, n, beta]:
    the bond dimension grows from chi to 2 chi (Sec. 2.1).
    """
    out = []
    for Ws, As in zip(W, A):
        na, nb, d, _ = Ws.shape
        Dl, _, Dr = As.shape
        dt = np.result_type(Ws, As)
        X = np.zeros((na, Dl, d, nb, Dr), dtype=dt)
        for a in range(na):
            for b in range(nb):
                for m in range(d):
                    for n in range(d):
                        w = Ws[a, b, m, n]
                        if w != 0.0:
                            X[a, :, m, b, :] += w * As[:, n, :]
        out.append(X.reshape(na * Dl, d, nb * Dr))
    return out


def to_dense(A) -> np.ndarray:
    """Contract an MPS to its 4^L coefficient vector (site 1 most significant)."""
    v = A[0]
    for s in A[1:]:
        v = np.tensordot(v, s, axes=(v.ndim - 1, 0))
    return v.reshape(-1)


def mpo_to_dense(W) -> np.ndarray:
    """Contract an MPO to its dense 4^L x 4^L matrix."""
    O = W[0][0]  # [b, m, n] after fixing the left boundary bond
    O = O.transpose(1, 2, 0)  # [m, n, b]
    for Ws in W[1:]:
        # O[M, N, b] x Ws[b, c, m, n] -> [M m, N n, c]
        O = np.einsum("MNb,bcmn->MmNnc", O, Ws)
        s = O.shape
        O = O.reshape(s[0] * s[1], s[2] * s[3], s[4])
    return O[:, :, 0]


def svd(M):
    """Thin SVD; LAPACK's divide-and-conquer driver with the QR-iteration driver
    as fallback when the former reports non-convergence."""
    try:
        return np.linalg.svd(M, full_matrices=False)
    except np.linalg.LinAlgError:
        return sla.svd(M, full_matrices=False, lapack_driver="gesvd")


def keep_count(s: np.ndarray, D_max: int, tol: float) -> int:
    """Truncation rule (reading of Sec. 2.2 / Fig. 3): s sorted descending.

    tol == 0: keep min(D_max, len(s)) values (zeros included: static shapes).
    tol > 0 : keep the smallest k whose discarded weight sum_{i>=k} s_i^2 is
              at most tol^2 * sum_i s_i^2, then cap at D_max; at least 1.
    """
    n = s.shape[0]
    if tol <= 0.0:
        return min(D_max, n)
    w = s.astype(np.float64) ** 2
    total = w.sum()
    tail = np.concatenate([np.cumsum(w[::-1])[::-1], [0.0]])  # tail[k] = sum_{i>=k}
    k = n
    for kk in range(1, n + 1):
        if tail[kk] <= tol * tol * total:
            k = kk
            break
    return max(1, min(D_max, k))


def compress(A, D_max: int, tol: float = 0.0, return_discarded: bool = False):
    """Compression of Fig. 3: QR sweep to right-canonical form, then an SVD
    sweep from left to right that keeps the largest singular values and merges
    S V^dagger into the next site.  The result is left-canonical with the norm
    in the last site (no renormalisation)."""
    A = [x.copy() for x in A]
    L = len(A)
    for i in range(L - 1, 0, -1):
        Dl, d, Dr = A[i].shape
        M = A[i].reshape(Dl, d * Dr)
        q, r = np.linalg.qr(M.T)              # M^T = q r  ->  M = r^T q^T  (LQ)
        k = q.shape[1]
        A[i] = q.T.reshape(k, d, Dr)
        A[i - 1] = np.tensordot(A[i - 1], r.T, axes=(2, 0))
    discarded = []
    for i in range(L - 1):
        Dl, d, Dr = A[i].shape
        u, s, vh = svd(A[i].reshape(Dl * d, Dr))
        k = keep_count(s, D_max, tol)
        discarded.append(float(np.sum(s[k:] ** 2)))
        A[i] = u[:, :k].reshape(Dl, d, k)
        A[i + 1] = np.tensordot(s[:k, None] * vh[:k], A[i + 1], axes=(1, 0))
    if return_discarded:
        return A, discarded
    return A


def direct_sum(A, B):
    """MPS addition by direct sum (Sec. 3.2): [A1 B1], diag(A_i, B_i), [A_L; B_L]."""
    L = len(A)
    if L == 1:
        return [A[0] + B[0]]
    out = []
    for i, (a, b) in enumerate(zip(A, B)):
        dt = np.result_type(a, b)
        if i == 0:
            out.append(np.concatenate([a, b], axis=2).astype(dt))
        elif i == L - 1:
            out.append(np.concatenate([a, b], axis=0).astype(dt))
        else:
            X = np.zeros((a.shape[0] + b.shape[0], a.shape[1], a.shape[2] + b.shape[2]), dtype=dt)
            X[: a.shape[0], :, : a.shape[2]] = a
            X[a.shape[0]:, :, a.shape[2]:] = b
            out.append(X)
    return out


def scale(A, c):
    """c |A>, applied to the last site."""
    out = [x.copy() for x in A]
    out[-1] = out[-1] * c
    return out


def add_compress(A, B, D_max: int, tol: float = 0.0):
    """compress(A (+) B): the reduction step of Alg. 1 and of Fig. parallel."""
    return compress(direct_sum(A, B), D_max, tol)


def inner(A, B) -> complex:
    """<A|B> by transfer matrices E_i = sum_n A^n^dagger E_{i-1} B^n."""
    E = np.ones((1, 1), dtype=np.result_type(A[0], B[0]))
    for a, b in zip(A, B):
        E = np.einsum("xy,xnz,ynw->zw", E, a.conj(), b)
    return E[0, 0]


def norm(A) -> float:
    return float(np.sqrt(abs(inner(A, A))))


def pad_to_profile(A, profile):
    """Zero-pad every bond of an MPS to the given bond dimensions."""
    out = []
    for i, a in enumerate(A):
        Dl, d, Dr = a.shape
        X = np.zeros((profile[i], d, profile[i + 1]), dtype=a.dtype)
        X[:Dl, :, :Dr] = a
        out.append(X)
    return out

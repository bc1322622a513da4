"""Dense (sparse-matrix) Fock-space definition of the molecular Hamiltonian.

Test infrastructure only (see oracle/__init__.py).

Conventions (readings of the paper where it leaves the choice open):
  * 2L fermionic modes, ordered site-major with spin-up before spin-down
    (App. C: "ordering the spin-up before the spin-down").
  * Two-level mode basis |0>, |1> with |1> occupied; c = [[0,1],[0,0]]
    (App. C) lowers |1> to |0>, Z = diag(1, -1).
  * Jordan-Wigner: a_j = Z (x) ... (x) Z (x) c (x) I (x) ... (x) I over the
    2L modes (textbook form).  Per site this is the pair b_up = c (x) I2,
    b_dn = Z (x) c of App. C with Z (x) Z strings on the sites to the left.
  * Full-space index: site 1 is the most significant Kronecker factor; within
    a site the index is 2*n_up + n_dn.
  * Eq. 1 is taken literally: the two-body operator is the product
    a+_{p s} a_{q s} a+_{r s'} a_{s s'} in that order, not normal ordered.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

C2 = np.array([[0.0, 1.0], [0.0, 0.0]])
Z2 = np.diag([1.0, -1.0])
I2 = np.eye(2)


def mode_annihilators(L: int):
    """The 2L annihilators a_{p,sigma} (sparse CSR), textbook JW over modes.

    Returned as a list indexed [p][sigma] with p = 0..L-1, sigma = 0 (up), 1 (dn).
    """
    nm = 2 * L
    ops = []
    for j in range(nm):
        factors = [Z2] * j + [C2] + [I2] * (nm - j - 1)
        op = sp.csr_matrix(np.array([[1.0]]))
        for f in factors:
            op = sp.kron(op, sp.csr_matrix(f), format="csr")
        ops.append(op)
    return [[ops[2 * p], ops[2 * p + 1]] for p in range(L)]


def number_ops(L: int, a=None):
    """(N_up, N_dn) as sparse matrices."""
    a = a if a is not None else mode_annihilators(L)
    nu = sum(a[p][0].T @ a[p][0] for p in range(L))
    nd = sum(a[p][1].T @ a[p][1] for p in range(L))
    return nu.tocsr(), nd.tocsr()


def thc_v(chi: np.ndarray, zeta: np.ndarray) -> np.ndarray:
    """Eq. thc: v_pqrs = sum_{mu,nu} chi^mu_p chi^mu_q zeta^{mu nu} chi^nu_r chi^nu_s."""
    L, N = chi.shape
    v = np.zeros((L, L, L, L))
    for mu in range(N):
        for nu in range(N):
            a = np.outer(chi[:, mu], chi[:, mu])
            b = np.outer(chi[:, nu], chi[:, nu])
            v += zeta[mu, nu] * a[:, :, None, None] * b[None, None, :, :]
    return v


def hamiltonian_eq1(t: np.ndarray, v: np.ndarray, a=None):
    """Eq. 1 with the literal operator order (sparse CSR, real)."""
    L = t.shape[0]
    a = a if a is not None else mode_annihilators(L)
    dim = 4 ** L
    # one-body operators E_pq^sigma = a+_{p sigma} a_{q sigma}
    E = [[[(a[p][s].T @ a[q][s]).tocsr() for s in range(2)] for q in range(L)]
         for p in range(L)]
    H = sp.csr_matrix((dim, dim))
    for p in range(L):
        for q in range(L):
            if t[p, q] != 0.0:
                H = H + t[p, q] * (E[p][q][0] + E[p][q][1])
    Esum = [[E[p][q][0] + E[p][q][1] for q in range(L)] for p in range(L)]
    for p in range(L):
        for q in range(L):
            acc = sp.csr_matrix((dim, dim))
            for r in range(L):
                for s in range(L):
                    if v[p, q, r, s] != 0.0:
                        acc = acc + v[p, q, r, s] * Esum[r][s]
            H = H + 0.5 * (Esum[p][q] @ acc)
    return H.tocsr()


def ladder_operator(coef: np.ndarray, sigma: int, dagger: bool, a=None):
    """sum_s coef_s a_{s,sigma} (or its adjoint) as a sparse matrix."""
    L = coef.shape[0]
    a = a if a is not None else mode_annihilators(L)
    op = sum(coef[s] * a[s][sigma] for s in range(L))
    return (op.T if dagger else op).tocsr()


def thc_subterm(chi, zeta, mu, sig, nu, sigp, a=None):
    """Eq. G: G_{mu sig, nu sig'} = zeta^{mu nu} A+_{mu sig} A_{mu sig} A+_{nu sig'} A_{nu sig'}."""
    A = lambda k, s, dag: ladder_operator(chi[:, k], s, dag, a)
    return zeta[mu, nu] * (A(mu, sig, True) @ A(mu, sig, False)
                           @ A(nu, sigp, True) @ A(nu, sigp, False))


def hamiltonian_thc(t, chi, zeta, a=None):
    """H built from the THC sub-terms: T (App. D) + 1/2 sum G (Eq. sum_of_H)."""
    L, N = chi.shape
    a = a if a is not None else mode_annihilators(L)
    lam, u = np.linalg.eigh(t)
    H = sp.csr_matrix((4 ** L, 4 ** L))
    for i in range(L):
        for s in range(2):
            H = H + lam[i] * (ladder_operator(u[:, i], s, True, a)
                              @ ladder_operator(u[:, i], s, False, a))
    # G_{mu s, nu s'} = zeta^{mu nu} G_{mu s} G_{nu s'}, G_{k s} = A+_{k s} A_{k s}
    G = [[(ladder_operator(chi[:, k], s, True, a) @ ladder_operator(chi[:, k], s, False, a)).tocsr()
          for s in range(2)] for k in range(N)]
    for mu in range(N):
        for nu in range(N):
            for s in range(2):
                for sp_ in range(2):
                    H = H + 0.5 * zeta[mu, nu] * (G[mu][s] @ G[nu][sp_])
    return H.tocsr()


def basis_occupations(L: int):
    """(n_up, n_dn) of every full-space basis index."""
    idx = np.arange(4 ** L)
    nu = np.zeros(4 ** L, dtype=np.int64)
    nd = np.zeros(4 ** L, dtype=np.int64)
    for site in range(L):
        shift = 2 * (L - 1 - site)
        nu += (idx >> (shift + 1)) & 1
        nd += (idx >> shift) & 1
    return nu, nd


def sector(L: int, n_up: int, n_dn: int) -> np.ndarray:
    nu, nd = basis_occupations(L)
    return np.nonzero((nu == n_up) & (nd == n_dn))[0]


def ground_energy(H, L: int, n_up: int, n_dn: int, k: int = 1):
    """Lowest k eigenvalues of H restricted to the (N_up, N_dn) sector (ED)."""
    s = sector(L, n_up, n_dn)
    Hs = H[s][:, s].toarray()
    w = np.linalg.eigvalsh(0.5 * (Hs + Hs.T))
    return w[:k] if k > 1 else w[0]


def expm_apply(H, psi: np.ndarray, dt: float) -> np.ndarray:
    """exp(-i dt H) psi (sparse Krylov-free reference, scipy expm_multiply)."""
    return spla.expm_multiply(-1j * dt * H.astype(np.complex128), psi.astype(np.complex128))

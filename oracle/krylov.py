"""Global Krylov methods on MPS (Sec. 2.2) for the oracle.

Test infrastructure only (see oracle/__init__.py).

Readings of the paper where it leaves the choice open:
  * Krylov vectors by full Gram-Schmidt: v_{k+1} is the compressed, normalised
    H v_k - sum_{j<=k} <v_j|H v_k> v_j, where the sum is one pairwise
    add-and-compress reduction over [H v_k, -h_0 v_0, ..., -h_k v_k].
  * The projected matrix is kept in full: Htil_jk = <v_j|H v_k> (Eq. Krylov_H),
    Hermitian-symmetrised, together with the overlap S_jk = <v_j|v_k>.
  * Loss of orthogonality is corrected by a coefficient matrix C (Eq. reortho,
    Eq. eff_H) from canonical orthogonalisation: S = W s W^H, eigenvalues below
    1e-12 * max(s) dropped, C = W s^{-1/2}.
  * Restart: the next run starts from the lowest Ritz vector sum_i (C y_0)_i v_i,
    compressed by the pairwise reduction and normalised.  Excited states: the
    start vector and every Krylov vector are orthogonalised against given lower
    states within the same Gram-Schmidt sum.
  * Time step: a(dt) = exp(-i dt Heff) a(0) in the orthonormalised basis, with
    a(0) the coordinates of v_0; psi(dt) = sum_i (C a)_i v_i, compressed,
    renormalised to the input norm; the lost norm is reported.
"""
from __future__ import annotations

import numpy as np

from . import mps as M
from .thc import pairwise_sum

ORTHO_DROP = 1e-12
BREAKDOWN = 1e-8  # relative to ||H v_k||: the Krylov space is exhausted


def orthogonalise_against(x, lower, D_max, tol):
    """x - sum_m <phi_m|x> phi_m by one pairwise add-and-compress (the lower
    states phi_m are orthonormal); x itself when there are none."""
    if not lower:
        return x
    items = [x] + [M.scale(f, -M.inner(f, x)) for f in lower]
    return pairwise_sum(items, D_max, tol)


def krylov_basis(Hop, psi0, K, D_max, tol, lower=()):
    """Return (v, w): K orthogonalised vectors and their compressed images H v.

    With `lower` (orthonormal MPS, e.g. lower eigenstates) the start vector and
    every new Krylov vector are also orthogonalised against them, in the same
    Gram-Schmidt sum (excited states, Sec. 2.2)."""
    x = orthogonalise_against(psi0, list(lower), D_max, tol)
    v = [M.scale(x, 1.0 / M.norm(x))]
    w = []
    for k in range(K):
        wk = Hop(v[k])
        w.append(wk)
        if k == K - 1:
            break
        h = [M.inner(v[j], wk) for j in range(k + 1)]
        g = [M.inner(f, wk) for f in lower]
        items = [wk] + [M.scale(v[j], -h[j]) for j in range(k + 1)] + [M.scale(f, -gm) for f, gm in zip(lower, g)]
        r = pairwise_sum(items, D_max, tol)
        nr = M.norm(r)
        if nr < BREAKDOWN * M.norm(wk):
            break
        v.append(M.scale(r, 1.0 / nr))
    return v, w


def projected(v, w):
    n = len(v)
    Ht = np.array([[M.inner(v[j], w[k]) for k in range(n)] for j in range(n)])
    S = np.array([[M.inner(v[j], v[k]) for k in range(n)] for j in range(n)])
    Ht = 0.5 * (Ht + Ht.conj().T)
    S = 0.5 * (S + S.conj().T)
    if np.all(np.isreal(Ht)) and np.all(np.isreal(S)):
        Ht, S = Ht.real, S.real
    return Ht, S


def canonical_orthogonalisation(S):
    s, W = np.linalg.eigh(S)
    keep = s > ORTHO_DROP * s.max()
    return W[:, keep] / np.sqrt(s[keep])


def ritz_from_projection(Ht, S):
    """Eq. eff_H: Ritz values (ascending) of C^H Htil C and the coefficients
    C y_0 of the lowest Ritz vector on the (non-orthogonal) Krylov vectors."""
    C = canonical_orthogonalisation(S)
    Heff = C.conj().T @ Ht @ C
    e, y = np.linalg.eigh(0.5 * (Heff + Heff.conj().T))
    return e, C @ y[:, 0]


def expm_coefficients(Ht, S, dt):
    """Eq. Krylov_combination in the C-orthonormalised basis: the coefficients a
    with sum_i a_i |v_i> = exp(-i dt H) |v_0> projected on span{v_i}; a(0) is
    the coordinate vector of v_0, C^H S e_0."""
    C = canonical_orthogonalisation(S)
    Heff = C.conj().T @ Ht @ C
    e, y = np.linalg.eigh(0.5 * (Heff + Heff.conj().T))
    b0 = C.conj().T @ S[:, 0]
    b = y @ (np.exp(-1j * dt * e) * (y.conj().T @ b0))
    return C @ b


def lanczos_ground(Hop, psi0, K, D_max, tol=0.0, lower=()):
    """Ritz values (ascending) and ground-state coefficients on the v_i."""
    v, w = krylov_basis(Hop, psi0, K, D_max, tol, lower)
    Ht, S = projected(v, w)
    e, c = ritz_from_projection(Ht, S)
    return e, c, v


def ritz_vector(c, v, D_max, tol=0.0):
    """sum_i c_i |v_i> by the pairwise reduction, normalised."""
    x = pairwise_sum([M.scale(v[i], c[i]) for i in range(len(v))], D_max, tol)
    return M.scale(x, 1.0 / M.norm(x))


def lanczos_restarted(Hop, psi0, K, cycles, D_max, tol=0.0, lower=()):
    """Restarted Lanczos (Sec. 2.2): `cycles` runs of K-step Lanczos, each
    started from the previous run's lowest Ritz vector (compressed and
    normalised).  With `lower` states every run stays orthogonal to them, so the
    lowest Ritz value approximates the next eigenvalue above them.  Returns the
    lowest Ritz value of every cycle and the last Ritz vector."""
    x = psi0
    energies = []
    for _ in range(cycles):
        e, c, v = lanczos_ground(Hop, x, K, D_max, tol, lower)
        energies.append(e[0])
        x = ritz_vector(c, v, D_max, tol)
    return np.array(energies), x


def krylov_expm_step(Hop, psi, dt, K, D_max, tol=0.0):
    """One global-Krylov time step; returns (psi(dt), lost_norm)."""
    n0 = M.norm(psi)
    v, w = krylov_basis(Hop, psi, K, D_max, tol)
    Ht, S = projected(v, w)
    a = expm_coefficients(Ht, S, dt)
    out = pairwise_sum([M.scale(v[i], a[i] * n0) for i in range(len(v))], D_max, tol)
    n1 = M.norm(out)
    lost = max(0.0, 1.0 - n1 / n0)
    return M.scale(out, n0 / n1), lost

"""THC-MPO application H|psi> on the CPU: Alg. 1, App. D and the reduction.

Test infrastructure only (see oracle/__init__.py).

Term list (readings of the paper where it leaves the choice open):
  * Coulomb terms G_{mu sig, nu sig'} (Eq. G), 4 N^2 of them, indexed
        t = ((sig' * N + nu) * 2 + sig) * N + mu
    i.e. mu fastest, then sig, then nu, then sig' (the order of the labels in
    Fig. parallel).  Each is four bond-2 layers applied bottom-up in the order
    s, r, q, p of Fig. thc_mpo: A_{nu sig'}, A+_{nu sig'}, A_{mu sig}, A+_{mu sig},
    with the state scaled by zeta^{mu nu}/2 before the last two (Alg. 1).
  * Kinetic terms T_{i sig} (App. D), 2L of them, indexed t = 4N^2 + sig*L + i:
    lambda_i A+_{u_i sig} A_{u_i sig} with t = U diag(lambda) U^T.
  * Every layer is followed by a compression (Fig. thc_mpo, Sec. 3.2).  The
    reuse of Sec. 3.2 computes psi_{nu sig'} = compress(A+ compress(A psi)) once
    per (nu, sig') and shares it across all (mu, sig).
  * The compressed terms are summed by the pairwise reduction of Fig. parallel:
    level by level, items 2j and 2j+1 are added and compressed, an odd last item
    moves up unchanged.
  * Optional spin merge (merge_spin=True; the symmetric-zeta reading of Eq. thc):
    for sig != sig' the one-body operators G_{mu sig} and G_{nu sig'} act on
    different spin modes and commute, so with zeta = zeta^T the sum over
    (mu down, nu up) equals the sum over (mu up, nu down) and the two merge
    into zeta^{mu nu} G_{mu up} G_{nu down}.  Same-spin products do not commute
    (the pair is [G_a, G_b] = (chi^a . chi^b)(A+_a A_b - A+_b A_a) apart) and
    stay as they are.  Term list: 3 N^2 Coulomb terms, block by block,
        t <  N^2        : block (nu = t // N, sig' = up),   mu = t % N, sig = up
        t >= N^2, t' = t - N^2 :
                          block (nu = t' // 2N, sig' = down), sig = (t' // N) % 2,
                          mu = t' % N; the factor 2 on sig = up (the merged pair)
    then the 2L kinetic terms.
"""
from __future__ import annotations

import numpy as np

from . import mps as M


def kinetic_factors(t: np.ndarray):
    """App. D, Eq. t_diagonalization: t = U diag(lambda) U^T (numerically exact)."""
    lam, u = np.linalg.eigh(t)
    return lam, u


def n_terms(L: int, N: int, merge_spin: bool = False) -> int:
    return (3 if merge_spin else 4) * N * N + 2 * L


def n_coulomb(N: int, merge_spin: bool = False) -> int:
    return (3 if merge_spin else 4) * N * N


def coulomb_index(mu, sig, nu, sigp, N):
    return ((sigp * N + nu) * 2 + sig) * N + mu


def decode_term(tidx: int, L: int, N: int):
    """('V', mu, sig, nu, sigp) or ('T', i, sig) for a term index."""
    if tidx < 4 * N * N:
        mu = tidx % N
        rest = tidx // N
        sig = rest % 2
        rest //= 2
        nu = rest % N
        sigp = rest // N
        return ("V", mu, sig, nu, sigp)
    k = tidx - 4 * N * N
    return ("T", k % L, k // L)


def decode_term_merged(tidx: int, L: int, N: int):
    """('V', mu, sig, nu, sigp, factor) or ('T', i, sig) in the spin-merged list."""
    if tidx < N * N:
        return ("V", tidx % N, 0, tidx // N, 0, 1.0)
    if tidx < 3 * N * N:
        k = tidx - N * N
        sig = (k // N) % 2
        return ("V", k % N, sig, k // (2 * N), 1, 2.0 if sig == 0 else 1.0)
    k = tidx - 3 * N * N
    return ("T", k % L, k // L)


def apply_layer(A, coef, sigma, dagger, D_max, tol):
    """One elementary MPO applied and the result compressed (Fig. thc_mpo arrows)."""
    return M.compress(M.apply_mpo(M.ladder_mpo(coef, sigma, dagger), A), D_max, tol)


def pairwise_sum(items, D_max, tol):
    """Pairwise add-and-compress reduction (Fig. parallel, Sec. 4.5)."""
    level = list(items)
    if not level:
        raise ValueError("empty reduction")
    while len(level) > 1:
        nxt = [M.add_compress(level[2 * j], level[2 * j + 1], D_max, tol)
               for j in range(len(level) // 2)]
        if len(level) % 2:
            nxt.append(level[-1])
        level = nxt
    return level[0]


def sequential_sum(items, D_max, tol):
    """Alg. 1's literal accumulation phi = compress(phi + x), phi starting at 0."""
    phi = None
    for x in items:
        phi = x if phi is None else M.add_compress(phi, x, D_max, tol)
    return phi


def term_states(psi, t, chi, zeta, D_max, tol, term_begin=0, term_end=None, merge_spin=False):
    """Compressed G|psi> / T|psi> for the terms in [term_begin, term_end), in order."""
    L, N = chi.shape
    T = n_terms(L, N, merge_spin)
    term_end = T if term_end is None else term_end
    lam, u = kinetic_factors(t)
    reuse = {}
    out = []
    for tidx in range(term_begin, term_end):
        kind = decode_term_merged(tidx, L, N) if merge_spin else decode_term(tidx, L, N)
        if kind[0] == "V" and not merge_spin:
            kind = kind + (1.0,)
        if kind[0] == "V":
            _, mu, sig, nu, sigp, factor = kind
            key = (nu, sigp)
            if key not in reuse:  # Alg. 1: psi_{nu sig'} from the two lower layers
                x = apply_layer(psi, chi[:, nu], sigp, False, D_max, tol)
                reuse[key] = apply_layer(x, chi[:, nu], sigp, True, D_max, tol)
            x = M.scale(reuse[key], factor * 0.5 * zeta[mu, nu])
            x = apply_layer(x, chi[:, mu], sig, False, D_max, tol)
            x = apply_layer(x, chi[:, mu], sig, True, D_max, tol)
        else:
            _, i, sig = kind
            x = M.scale(psi, lam[i])
            x = apply_layer(x, u[:, i], sig, False, D_max, tol)
            x = apply_layer(x, u[:, i], sig, True, D_max, tol)
        out.append(x)
    return out


def apply_H(psi, t, chi, zeta, D_max, tol=0.0, term_begin=0, term_end=None, merge_spin=False):
    """H|psi> as a compressed MPS: all terms, then the pairwise reduction."""
    return pairwise_sum(term_states(psi, t, chi, zeta, D_max, tol, term_begin, term_end, merge_spin),
                        D_max, tol)


def apply_V_alg1(psi, chi, zeta, D_max, tol=0.0):
    """V|psi> exactly as Alg. 1 orders it (sequential accumulation)."""
    L, N = chi.shape
    zero_t = np.zeros((L, L))
    items = term_states(psi, zero_t, chi, zeta, D_max, tol, 0, 4 * N * N)
    return sequential_sum(items, D_max, tol)

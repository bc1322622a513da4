"""Seeded synthetic inputs for the THC-MPO hot path.

This module only draws random numbers and shapes them into valid inputs: a
THC-factorised Hamiltonian (t, chi, zeta) and a random matrix-product state
confined to a particle-number sector.  It holds none of the method's
arithmetic (no ladder MPO, no Hamiltonian application, no truncation rule):
both the CPU oracle and the CUDA path consume what it returns, and neither
side's code is used here.

Distributions (the paper's molecules are replaced by synthetic stand-ins of
the same shape regime, Sec. 2.3 and Sec. 4):
  * chi  : L x N, i.i.d. N(0,1) with every column scaled to unit norm;
  * zeta : Z Z^T / N with Z an N x N matrix of i.i.d. N(0,1) (symmetric, PSD);
  * t    : symmetric L x L, off-diagonal N(0, 0.5^2), diagonal t_pp = -p.
The three are drawn in that order from numpy's default_rng(seed).

Site basis (App. C): index n = 2*n_up + n_dn, i.e. |0>, |dn>, |up>, |updn>,
because the local annihilators are b_up = c (x) I2 and b_dn = Z (x) c, which
makes the spin-up mode the major Kronecker factor.
"""
from __future__ import annotations

from math import comb

import numpy as np

D_LOCAL = 4


def thc_hamiltonian(L: int, N: int, seed: int):
    """Return (t, chi, zeta) as float64 arrays of shapes (L,L), (L,N), (N,N)."""
    rng = np.random.default_rng(seed)
    chi = rng.standard_normal((L, N))
    chi /= np.linalg.norm(chi, axis=0, keepdims=True)
    Z = rng.standard_normal((N, N))
    zeta = Z @ Z.T / N
    off = rng.normal(0.0, 0.5, (L, L))
    t = np.triu(off, 1)
    t = t + t.T
    t[np.diag_indices(L)] = -np.arange(1, L + 1, dtype=np.float64)
    return t, chi, zeta


def full_bond_profile(L: int, D: int):
    """Bond dimensions min(D, 4^b, 4^(L-b)) for b = 0..L (static MPS shape)."""
    return [min(D, D_LOCAL ** b, D_LOCAL ** (L - b)) for b in range(L + 1)]


def _sector_dims(L, b, n_up, n_dn, cap):
    """Sectors (u, d) allowed on bond b and how many bond states each gets."""
    secs = []
    for u in range(max(0, n_up - (L - b)), min(b, n_up) + 1):
        for d in range(max(0, n_dn - (L - b)), min(b, n_dn) + 1):
            exact = min(comb(b, u) * comb(b, d),
                        comb(L - b, n_up - u) * comb(L - b, n_dn - d))
            if exact > 0:
                secs.append(((u, d), exact))
    total = sum(e for _, e in secs)
    if total <= cap:
        return [(q, e) for q, e in secs]
    dims = [min(e, (cap * e) // total) for _, e in secs]
    # hand out the remainder to the largest sectors that still have room
    order = sorted(range(len(secs)), key=lambda i: -secs[i][1])
    left = cap - sum(dims)
    while left > 0:
        progressed = False
        for i in order:
            if left == 0:
                break
            if dims[i] < secs[i][1]:
                dims[i] += 1
                left -= 1
                progressed = True
        if not progressed:
            break
    return [(secs[i][0], dims[i]) for i in range(len(secs)) if dims[i] > 0]


def _labels(L, b, n_up, n_dn, chi_b):
    """Sector label of every state on bond b; padding states get None."""
    lab = []
    for q, m in _sector_dims(L, b, n_up, n_dn, chi_b):
        lab += [q] * m
    lab += [None] * (chi_b - len(lab))
    return lab


def sector_mps(L: int, n_up: int, n_dn: int, D: int, seed: int,
               decay: float | None = None, dtype=np.float64):
    """Random normalised MPS in the (N_up, N_dn) sector with the full profile.

    Site i has shape [chi_{i}, 4, chi_{i+1}] with chi_b = min(D, 4^b, 4^(L-b)).
    Entries are N(0,1) inside the blocks that conserve (N_up, N_dn) and zero
    elsewhere.  The state is brought to unit norm; with ``decay`` set, every
    bond's non-zero Schmidt values are replaced by exp(-k/decay) (normalised),
    k = 0, 1, ..., which fixes the entanglement spectrum the workloads ask for.
    numpy's QR/SVD are used only to shape this input.
    """
    rng = np.random.default_rng(seed)
    prof = full_bond_profile(L, D)
    labels = [[(0, 0)]] + [_labels(L, b, n_up, n_dn, prof[b]) for b in range(1, L)] \
        + [[(n_up, n_dn)]]
    sites = []
    for i in range(L):
        left, right = labels[i], labels[i + 1]
        A = np.zeros((len(left), D_LOCAL, len(right)))
        for n in range(D_LOCAL):
            du, dd = n >> 1, n & 1
            for a, qa in enumerate(left):
                if qa is None:
                    continue
                want = (qa[0] + du, qa[1] + dd)
                cols = [c for c, qb in enumerate(right) if qb == want]
                if cols:
                    A[a, n, cols] = rng.standard_normal(len(cols))
        sites.append(A)
    # right-canonicalise (LQ sweep) so the left->right SVD sweep sees Schmidt values
    for i in range(L - 1, 0, -1):
        Dl, d, Dr = sites[i].shape
        q, r = np.linalg.qr(sites[i].reshape(Dl, d * Dr).T)
        k = q.shape[1]
        sites[i] = q.T.reshape(k, d, Dr)
        sites[i - 1] = np.tensordot(sites[i - 1], r.T, axes=(2, 0))
        if k < Dl:  # keep the static profile: pad the bond back with zeros
            pad = Dl - k
            sites[i] = np.concatenate([sites[i], np.zeros((pad, d, Dr))], 0)
            sites[i - 1] = np.concatenate(
                [sites[i - 1], np.zeros(sites[i - 1].shape[:2] + (pad,))], 2)
    if decay is not None:
        for i in range(L - 1):
            Dl, d, Dr = sites[i].shape
            u, s, vh = np.linalg.svd(sites[i].reshape(Dl * d, Dr), full_matrices=False)
            r = int(np.sum(s > 1e-12 * s[0])) if s[0] > 0 else 0
            p = np.zeros_like(s)
            p[:r] = np.exp(-np.arange(r) / decay)
            p /= np.linalg.norm(p)
            k = s.shape[0]
            sites[i] = u.reshape(Dl, d, k)
            sites[i + 1] = np.tensordot(p[:, None] * vh, sites[i + 1], axes=(1, 0))
            if k < Dr:
                pad = Dr - k
                sites[i] = np.concatenate([sites[i], np.zeros((Dl, d, pad))], 2)
                sites[i + 1] = np.concatenate(
                    [sites[i + 1], np.zeros((pad,) + sites[i + 1].shape[1:])], 0)
        nrm = np.linalg.norm(sites[-1])
    else:
        nrm = np.linalg.norm(sites[0])
    idx = L - 1 if decay is not None else 0
    sites[idx] = sites[idx] / nrm
    return [np.ascontiguousarray(A.astype(dtype)) for A in sites]


def random_mps(L: int, D: int, seed: int, dtype=np.float64):
    """Unstructured random MPS with the full bond profile (not normalised)."""
    rng = np.random.default_rng(seed)
    prof = full_bond_profile(L, D)
    return [rng.standard_normal((prof[i], D_LOCAL, prof[i + 1])).astype(dtype)
            for i in range(L)]


# Named workloads: (L, N, D_max, hamiltonian seed, mps seed, sector, decay)
WORKLOADS = {
    "L6_N12_D16": dict(L=6, N=12, D=16, hseed=0, mseed=1000, n_up=3, n_dn=3, decay=None),
    "L16_N48_D128": dict(L=16, N=48, D=128, hseed=0, mseed=1001, n_up=8, n_dn=8, decay=12.0),
    "L24_N96_D256": dict(L=24, N=96, D=256, hseed=1, mseed=1002, n_up=12, n_dn=12, decay=12.0),
}


def workload(name: str, dtype=np.float64):
    """Return (t, chi, zeta, psi_sites, D_max) for a named workload."""
    w = WORKLOADS[name]
    t, chi, zeta = thc_hamiltonian(w["L"], w["N"], w["hseed"])
    psi = sector_mps(w["L"], w["n_up"], w["n_dn"], w["D"], w["mseed"],
                     decay=w["decay"], dtype=dtype)
    return t, chi, zeta, psi, w["D"]

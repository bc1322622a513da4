"""<phi|H|psi> and its derivatives with respect to t, chi, zeta and psi.

Test infrastructure only (see oracle/__init__.py).

E(t, chi, zeta, psi) = <phi| H |psi> with H of Eq. 1 and v_pqrs of Eq. thc,
built densely in the Fock space (L <= 6).  Writing E_pq = sum_s a+_ps a_qs and
Ghat_mu = sum_pq chi^mu_p chi^mu_q E_pq (the spin sum of Eq. G's
G_{mu s} = A+_{mu s} A_{mu s}),

  E = sum_pq t_pq <phi|E_pq|psi> + 1/2 sum_{mu nu} zeta^{mu nu} <phi|Ghat_mu Ghat_nu|psi>,

so, treating every entry as an independent variable,

  dE/dt_pq         = <phi|E_pq|psi>
  dE/dzeta^{mu nu} = 1/2 <phi|Ghat_mu Ghat_nu|psi>
  dE/dchi^k_p      = 1/2 sum_nu zeta^{k nu} <phi|D_pk Ghat_nu|psi>
                   + 1/2 sum_mu zeta^{mu k} <phi|Ghat_mu D_pk|psi>,
                     D_pk = dGhat_k/dchi^k_p = sum_q chi^k_q (E_pq + E_qp)
  dE/dpsi          = H^T phi (a dense vector; for an MPS, contracted with
                     every site of psi but the one differentiated).
"""
from __future__ import annotations

import numpy as np

from . import fock as F


def one_body(L, a=None):
    """E_pq = sum_sigma a+_{p sigma} a_{q sigma} (sparse), as a list of lists."""
    a = a if a is not None else F.mode_annihilators(L)
    return [[(a[p][0].T @ a[q][0] + a[p][1].T @ a[q][1]).tocsr() for q in range(L)] for p in range(L)]


def _ghat(c, E):
    L = len(c)
    return sum(c[p] * c[q] * E[p][q] for p in range(L) for q in range(L))


def expectation(phi, psi, t, chi, zeta):
    """<phi|H|psi> with the dense Eq. 1 Hamiltonian (phi, psi dense real vectors)."""
    H = F.hamiltonian_eq1(t, F.thc_v(chi, zeta))
    return float(phi @ (H @ psi))


def gradients(phi, psi, t, chi, zeta):
    """(dE/dt [L, L], dE/dchi [L, N], dE/dzeta [N, N], dE/dpsi [4^L]) for real
    dense vectors phi and psi."""
    L, N = chi.shape
    E = one_body(L)
    dt = np.array([[phi @ (E[p][q] @ psi) for q in range(L)] for p in range(L)])
    G = [_ghat(chi[:, k], E) for k in range(N)]
    Gpsi = np.array([g @ psi for g in G])          # Ghat_nu |psi>
    Gphi = np.array([g.T @ phi for g in G])        # Ghat_mu^T |phi> (Ghat is symmetric)
    dzeta = 0.5 * Gphi @ Gpsi.T                    # <phi|Ghat_mu Ghat_nu|psi>
    Zpsi = zeta @ Gpsi                             # sum_nu zeta^{k nu} Ghat_nu |psi>
    Zphi = zeta.T @ Gphi                           # sum_mu zeta^{mu k} Ghat_mu^T |phi>
    dchi = np.zeros((L, N))
    for k in range(N):
        for p in range(L):
            D = sum(chi[q, k] * (E[p][q] + E[q][p]) for q in range(L))
            dchi[p, k] = 0.5 * (phi @ (D @ Zpsi[k])) + 0.5 * (Zphi[k] @ (D @ psi))
    H = F.hamiltonian_eq1(t, F.thc_v(chi, zeta))
    dpsi = H.T @ phi
    return dt, dchi, dzeta, dpsi


def site_gradient(dvec, sites, i):
    """d<dvec|psi>/d(site i of psi) for real vectors: the dense vector dvec
    (4^L, site 0 most significant) contracted with every site of the MPS psi
    except site i; shape of site i."""
    L = len(sites)
    left = np.ones((1, 1))                       # [4^i, D_i]
    for s in range(i):
        left = np.einsum("xa,anb->xnb", left, sites[s]).reshape(-1, sites[s].shape[2])
    right = np.ones((1, 1))                      # [D_{i+1}, 4^(L-1-i)]
    for s in range(L - 1, i, -1):
        right = np.einsum("anb,by->any", sites[s], right).reshape(sites[s].shape[0], -1)
    d = dvec.reshape(left.shape[0], 4, right.shape[1])
    return np.einsum("xa,xny,by->anb", left, d, right)

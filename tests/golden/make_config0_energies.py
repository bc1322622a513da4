"""Write tests/golden/config0_energies.txt from the CPU oracle alone.

The L = 6, N = 12 workload (Hamiltonian seed 0, start state: the random
(3, 3)-sector MPS of seed 1000): the exact ground energy of the (3, 3) sector
by dense diagonalisation of Eq. 1 in the 4096-dimensional Fock space, and the
lowest Ritz value of K-step Lanczos (Sec. 2.2) on the dense start vector, for
K = 10 (the workload's Krylov dimension) and K = 40.

    python tests/golden/make_config0_energies.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import fock as F  # noqa: E402
from oracle import mps as OM  # noqa: E402
from paper_2409_12708_gb300.workloads import workload  # noqa: E402

OUT = os.path.join(HERE, "config0_energies.txt")


def dense_lanczos_lowest(Hs, v0, K):
    """Lowest Ritz value of K-step Lanczos with full reorthogonalisation."""
    V = [v0 / np.linalg.norm(v0)]
    for _ in range(K - 1):
        w = Hs @ V[-1]
        for _ in range(2):
            for v in V:
                w = w - (v @ w) * v
        V.append(w / np.linalg.norm(w))
    Vm = np.array(V).T
    return float(np.linalg.eigvalsh(Vm.T @ Hs @ Vm)[0])


def compute():
    t, chi, zeta, psi, _ = workload("L6_N12_D16")
    H = F.hamiltonian_eq1(t, F.thc_v(chi, zeta))
    s = F.sector(6, 3, 3)
    Hs = H[s][:, s].toarray()
    v0 = OM.to_dense(psi)[s]
    return {"ed_ground_energy": float(F.ground_energy(H, 6, 3, 3)),
            "dense_lanczos_K10": dense_lanczos_lowest(Hs, v0, 10),
            "dense_lanczos_K40": dense_lanczos_lowest(Hs, v0, 40)}


def read(path=OUT):
    vals = {}
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            k, v = line.split()
            vals[k] = float(v)
    return vals


if __name__ == "__main__":
    vals = compute()
    with open(OUT, "w") as f:
        f.write("# L=6 N=12 workload, (3,3) sector; written by make_config0_energies.py (oracle only)\n")
        for k, v in vals.items():
            f.write(f"{k} {v:.15f}\n")
    print(open(OUT).read())

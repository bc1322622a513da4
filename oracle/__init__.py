"""CPU oracle for the THC-MPO hot path -- TEST INFRASTRUCTURE ONLY.

Plain, slow, float64 (complex128 where the state is complex) restatement of
what the method computes, written from the paper (arXiv 2409.12708):

  fock.py    dense Jordan-Wigner Fock space: Eq. 1 Hamiltonian, THC sub-terms
             (Eq. G), exact diagonalisation and exp(-i dt H).
  mps.py     MPS engine: bond-2 ladder MPOs (elementary-MPO equations with the
             Jordan-Wigner Z(x)Z strings), MPO x MPS by explicit loops, the
             QR-then-SVD compression of Fig. 3, direct sums, inner products.
  thc.py     Alg. 1 with the reuse of G_{nu sigma'}|psi>, the kinetic
             decomposition of App. D and the pairwise reduction of Sec. 4.5.
  krylov.py  global Krylov methods of Sec. 2.2: Lanczos ground state with the
             canonical-orthogonalisation correction (reortho / eff_H equations)
             and one Krylov time step.

It shares no code with the CUDA path and imports nothing from it.  Only
tests/, __graft_entry__.smoke() and bench.py (its cpu_baseline leg and
--impl reference arm) may import or run anything in this directory; the
product path never does.
"""

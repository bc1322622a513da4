"""GB300 (sm_103a) THC-MPO Krylov hot path: apply a tensor-hypercontraction
factorised molecular Hamiltonian to a matrix-product state and recompress it.

The compute path is the CUDA library built from csrc/ (C ABI in
include/thc.h); `binding` is its Python marshalling layer and `workloads`
the seeded synthetic inputs.  Import `binding` explicitly: it loads the
library and raises if the build is missing.
"""

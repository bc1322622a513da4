// inst_f32.cu -- the entry points' typed bodies for float site tensors.
#include "abi_impl.cuh"

using thc::c32;
using thc::c64;

THC_ABI_FOR(template, float)
THC_ABI_FOR_REAL(template, float)

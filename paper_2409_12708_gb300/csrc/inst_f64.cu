// inst_f64.cu -- the entry points' typed bodies for double site tensors.
#include "abi_impl.cuh"

using thc::c32;
using thc::c64;

THC_ABI_FOR(template, double)
THC_ABI_FOR_REAL(template, double)

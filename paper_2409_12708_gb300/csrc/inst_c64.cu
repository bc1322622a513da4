// inst_c64.cu -- the entry points' typed bodies for c32 site tensors.
#include "abi_impl.cuh"

using thc::c32;
using thc::c64;

THC_ABI_FOR(template, c32)
THC_ABI_FOR_EXPM(template, c32)

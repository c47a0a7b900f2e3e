// The 32-warp plain-launch division kernel whose full products may use the
// number-theoretic transform.
#include "mp_kernels.cuh"
#include "mpdiv_kernels.h"

void* mp_kernel_ntt_uniform32() { return (void*)mp::k_div_uniform<32, 1, true>; }

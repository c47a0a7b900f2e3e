// The 16-warp plain-launch division kernel whose full products may use the
// number-theoretic transform.
#include "mp_kernels.cuh"
#include "mpdiv_kernels.h"

void* mp_kernel_ntt_uniform16() { return (void*)mp::k_div_uniform<16, 2, true>; }

// The shifted-inverse test entry whose full products may use the
// number-theoretic transform (16-warp blocks).
#include "mp_kernels.cuh"
#include "mpdiv_kernels.h"

void* mp_kernel_ntt_shinv() { return (void*)mp::k_shinv<16, 2, true>; }

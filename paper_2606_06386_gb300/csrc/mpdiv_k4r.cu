// The plain division kernel for 4-warp blocks with the register budget of
// 4 resident block(s) per SM, 128 registers per thread, without the spills of the
// 64-register build: a candidate of the tuner (a separate translation unit,
// so that the block sizes build in parallel).
#define MP_STRIP_T3_UNROLL 1  // two row groups per loop trip at T = 3 (see mp_block.cuh)
#include "mp_kernels.cuh"
#include "mpdiv_kernels.h"

void* mp_kernel_w4_wide() { return (void*)mp::k_div_uniform<4, 4>; }

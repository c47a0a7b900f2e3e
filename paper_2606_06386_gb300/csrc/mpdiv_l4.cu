// The plain division kernel for 4-warp blocks over a ragged batch's item
// list (the class form of mpdiv_batch_ragged), with the compile-time choices of
// the strided kernel of the same block size (a separate translation unit, so
// that the kernels build in parallel).
#define MP_STRIP_T3_UNROLL 1  // two row groups per loop trip at T = 3 (see mp_block.cuh)
#include "mp_kernels.cuh"
#include "mpdiv_kernels.h"

void* mp_kernel_list4() { return (void*)mp::k_div_uniform<4, 8, false, true>; }

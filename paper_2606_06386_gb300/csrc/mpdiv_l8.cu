// The plain division kernel for 8-warp blocks over a ragged batch's item
// list (the class form of mpdiv_batch_ragged), with the compile-time choices of
// the strided kernel of the same block size (a separate translation unit, so
// that the kernels build in parallel).
#include "mp_kernels.cuh"
#include "mpdiv_kernels.h"

void* mp_kernel_list8() { return (void*)mp::k_div_uniform<8, 4, false, true>; }

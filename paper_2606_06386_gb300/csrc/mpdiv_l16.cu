// The plain division kernel for 16-warp blocks over a ragged batch's item
// list (the class form of mpdiv_batch_ragged), with the compile-time choices of
// the strided kernel of the same block size (a separate translation unit, so
// that the kernels build in parallel).
#include "mp_kernels.cuh"
#include "mpdiv_kernels.h"

void* mp_kernel_list16() { return (void*)mp::k_div_uniform<16, 2, false, true>; }

// The plain division kernel for 1-warp blocks over a ragged batch's item
// list (the class form of mpdiv_batch_ragged), with the compile-time choices of
// the strided kernel of the same block size (a separate translation unit, so
// that the kernels build in parallel).
#define MP_MUL_NOINLINE 1  // the strip multiply as one called copy (see mp_block.cuh)
#define MP_VECTOR_IO 0  // digit-by-digit operand loads and result stores (see mp_block.cuh)
#define MP_STRIP_T3_UNROLL 1  // two row groups per loop trip at T = 3 (see mp_block.cuh)
#include "mp_kernels.cuh"
#include "mpdiv_kernels.h"

void* mp_kernel_list1() { return (void*)mp::k_div_uniform<1, 32, false, true>; }

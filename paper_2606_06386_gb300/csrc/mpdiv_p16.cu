// The self-splitting persistent division kernel in 16-warp blocks (splitting
// to 8 and 4 warps), in a translation unit of its own so that it builds in
// parallel with the rest.
#define MP_NAMED_GROUPS 1  // groups are slices of a block under named barriers (see mp_block.cuh)
#define MP_EARLY_ON_ONE_WARP 0  // every Refine iteration on the whole group (see mp_div.cuh)
#include "mp_kernels.cuh"
#include "mpdiv_kernels.h"

void* mp_kernel_persistent16() { return (void*)mp::k_div_persistent<16, 1>; }

void* mp_kernel_persistent(int warps) { return warps <= 8 ? mp_kernel_persistent8() : mp_kernel_persistent16(); }

// The self-splitting persistent division kernel in 8-warp blocks (two per SM,
// splitting to 4 and 2 warps), in a translation unit of its own so that it
// builds in parallel with the rest; the 16-warp form is in mpdiv_p16.cu.
#define MP_NAMED_GROUPS 1  // groups are slices of a block under named barriers (see mp_block.cuh)
#define MP_EARLY_ON_ONE_WARP 0  // every Refine iteration on the whole group (see mp_div.cuh)
#include "mp_kernels.cuh"
#include "mpdiv_kernels.h"

void* mp_kernel_persistent8() { return (void*)mp::k_div_persistent<8, 2>; }

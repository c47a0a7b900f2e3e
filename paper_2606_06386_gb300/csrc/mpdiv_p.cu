// The self-splitting persistent division kernels: 8-warp blocks (two per SM,
// splitting to 4 and 2 warps) and 16-warp blocks (splitting to 8 and 4), in a
// translation unit of their own so that they build in parallel with the rest.
#define MP_NAMED_GROUPS 1  // groups are slices of a block under named barriers (see mp_block.cuh)
#include "mp_kernels.cuh"
#include "mpdiv_kernels.h"

void* mp_kernel_persistent(int warps) {
  return warps <= 8 ? (void*)mp::k_div_persistent<8, 2> : (void*)mp::k_div_persistent<16, 1>;
}

// Division kernels instantiated for two-warp blocks: one division per warp
// pair for the small precisions, so that many divisions share an SM and a
// group barrier spans two warps (a separate translation unit, so that the
// block sizes build in parallel).
#define MP_MUL_NOINLINE 1  // the strip multiply as one called copy (see mp_block.cuh)
#define MP_VECTOR_IO 0  // digit-by-digit operand loads and result stores (see mp_block.cuh)
#define MP_STRIP_T3_UNROLL 1  // two row groups per loop trip at T = 3 (see mp_block.cuh)
#include "mp_kernels.cuh"
#include "mpdiv_kernels.h"

void* mp_kernel_w2(int kind) {
  switch (kind) {
    case MP_K_UNIFORM: return (void*)mp::k_div_uniform<2, 16>;
    case MP_K_MUL: return (void*)mp::k_mul_low<2, 16>;
    default: return nullptr;
  }
}

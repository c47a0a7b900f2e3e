// Division kernels instantiated for 128-thread blocks (compiled as a
// separate translation unit so that the block sizes build in parallel).
#define MP_STRIP_T3_UNROLL 1  // two row groups per loop trip at T = 3 (see mp_block.cuh)
#include "mp_kernels.cuh"
#include "mpdiv_kernels.h"

void* mp_kernel_w4(int kind) {
  switch (kind) {
    case MP_K_UNIFORM: return (void*)mp::k_div_uniform<4, 8>;
    case MP_K_MUL: return (void*)mp::k_mul_low<4, 8>;
    default: return nullptr;
  }
}

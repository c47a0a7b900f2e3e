// Division kernels instantiated for 256-thread blocks (compiled as a
// separate translation unit so that the block sizes build in parallel).
#include "mp_kernels.cuh"
#include "mpdiv_kernels.h"

void* mp_kernel_w8(int kind) {
  switch (kind) {
    case MP_K_UNIFORM: return (void*)mp::k_div_uniform<8, 4>;
    case MP_K_MUL: return (void*)mp::k_mul_low<8, 4>;
    case MP_K_PERSIST: return mp_kernel_persistent(8);
    default: return nullptr;
  }
}

// Division kernels instantiated for 512-thread blocks (compiled as a
// separate translation unit so that the block sizes build in parallel).
#include "mp_kernels.cuh"
#include "mpdiv_kernels.h"

void* mp_kernel_w16(int kind) {
  switch (kind) {
    case MP_K_UNIFORM: return (void*)mp::k_div_uniform<16, 2>;
    case MP_K_RAGGED: return mp_kernel_w16_queue(kind);
    case MP_K_SHINV: return mp_kernel_w16_queue(kind);
    case MP_K_MUL: return (void*)mp::k_mul_low<16, 2>;
    case MP_K_PERSIST: return mp_kernel_persistent(16);
    default: return nullptr;
  }
}

// The one-block-per-item queue kernel and the shifted-inverse test entry, both
// in 16-warp blocks, in a translation unit of their own so that they build in
// parallel with the rest.
#define MP_VECTOR_IO 0  // digit-by-digit operand loads and result stores (see mp_block.cuh)
#include "mp_kernels.cuh"
#include "mpdiv_kernels.h"

void* mp_kernel_w16_queue(int kind) {
  switch (kind) {
    case MP_K_RAGGED: return (void*)mp::k_div_ragged<16, 2>;
    case MP_K_SHINV: return (void*)mp::k_shinv<16, 2>;
    default: return nullptr;
  }
}

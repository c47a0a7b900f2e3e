// The one-block-per-item queue kernel whose full products may use the
// number-theoretic transform (16-warp blocks), and the getter for it and for
// the shifted-inverse test entry (mpdiv_n3.cu).
#include "mp_kernels.cuh"
#include "mpdiv_kernels.h"

void* mp_kernel_ntt_queue(int kind) {
  switch (kind) {
    case MP_K_RAGGED: return (void*)mp::k_div_ragged<16, 2, true>;
    case MP_K_SHINV: return mp_kernel_ntt_shinv();
    default: return nullptr;
  }
}

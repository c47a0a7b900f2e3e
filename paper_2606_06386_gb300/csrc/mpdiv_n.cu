// Plain-launch division kernels whose full products may use the
// number-theoretic transform (MPDIV_FLAG_NTT_PRODUCTS), at 4, 8, 16 and 32
// warps per block with the registers of the strip kernels of the same block
// size (8, 16 and 32 in mpdiv_n8.cu, mpdiv_n16.cu and mpdiv_n32.cu, which
// build in parallel), and the multiplication cost unit by the transform.
#include "mp_kernels.cuh"
#include "mpdiv_kernels.h"

void* mp_kernel_ntt_uniform(int warps) {
  if (warps <= 4) return (void*)mp::k_div_uniform<4, 8, true>;
  if (warps <= 8) return mp_kernel_ntt_uniform8();
  if (warps <= 16) return mp_kernel_ntt_uniform16();
  return mp_kernel_ntt_uniform32();
}

void* mp_kernel_ntt_mul(int warps) {
  if (warps <= 4) return (void*)mp::k_mul_low<4, 8, true>;
  if (warps <= 8) return (void*)mp::k_mul_low<8, 4, true>;
  if (warps <= 16) return (void*)mp::k_mul_low<16, 2, true>;
  return (void*)mp::k_mul_low<32, 1, true>;
}

// The group-primitive test kernel for every block size, in a translation unit
// of its own.
#include "mp_kernels.cuh"
#include "mpdiv_kernels.h"

void* mp_kernel_prim(int warps) {
  switch (warps) {
    case 1: return (void*)mp::k_prim<1, 32>;
    case 2: return (void*)mp::k_prim<2, 16>;
    case 4: return (void*)mp::k_prim<4, 8>;
    case 8: return (void*)mp::k_prim<8, 4>;
    case 16: return (void*)mp::k_prim<16, 2>;
    default: return (void*)mp::k_prim<32, 1>;
  }
}

// Microbenchmarks of the integer multiply pipe, the measured ceiling of the
// roofline (mpdiv_measure_peak). Each thread runs `iters` rounds over kAcc
// independent accumulators held in registers. The operands differ per thread,
// and the accumulators are written out at the end, so nothing folds away.
namespace {
constexpr int kAcc = 8;

// The strip multiply's digit product: mad.lo.cc / madc.hi.cc / addc into a
// three-word column accumulator (mp::mac3), kAcc products per round.
__global__ void __launch_bounds__(256) k_peak_mac3(uint32_t* out, int iters) {
  const uint32_t x = threadIdx.x * 2654435761u + blockIdx.x, y = 0x9e3779b9u ^ (blockIdx.x * 40503u);
  uint32_t c0[kAcc], c1[kAcc], c2[kAcc], a[kAcc];
#pragma unroll
  for (int k = 0; k < kAcc; k++) {
    c0[k] = (uint32_t)k;
    c1[k] = c2[k] = 0u;
    a[k] = x + 977u * (uint32_t)k;
  }
  for (int it = 0; it < iters; it++) {
#pragma unroll
    for (int k = 0; k < kAcc; k++) mp::mac3(c0[k], c1[k], c2[k], a[k], y);
  }
  uint32_t s = 0u;
#pragma unroll
  for (int k = 0; k < kAcc; k++) s ^= c0[k] ^ c1[k] ^ c2[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Independent 32-bit multiply-adds (mad.lo.u32), kAcc per round.
__global__ void __launch_bounds__(256) k_peak_imad(uint32_t* out, int iters) {
  const uint32_t y = 0x9e3779b9u ^ (blockIdx.x * 40503u), z = threadIdx.x | 1u;
  uint32_t a[kAcc];
#pragma unroll
  for (int k = 0; k < kAcc; k++) a[k] = threadIdx.x * 2654435761u + 977u * (uint32_t)k;
  for (int it = 0; it < iters; it++) {
#pragma unroll
    for (int k = 0; k < kAcc; k++) asm("mad.lo.u32 %0, %0, %1, %2;" : "+r"(a[k]) : "r"(y), "r"(z));
  }
  uint32_t s = 0u;
#pragma unroll
  for (int k = 0; k < kAcc; k++) s ^= a[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
}  // namespace

void* mp_kernel_peak(int kind, int* ops_per_round) {
  *ops_per_round = kAcc;
  return kind == 0 ? (void*)k_peak_mac3 : (void*)k_peak_imad;
}

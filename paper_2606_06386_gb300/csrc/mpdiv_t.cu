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
// The strip multiply's inner loop as the division kernels run it (mp::mul_strip
// at 5 columns per lane): each lane keeps a 5-digit window of the longer
// operand in a register ring refilled from shared memory, and each row digit
// of the shorter operand is a shared-memory broadcast. Every block holds
// kStripRows row digits and kStripWin window digits; lane L reads window
// digits 5 L + 1 up to kStripRows + 5 L + 4 < kStripWin. One round is one
// pass over the rows.
constexpr int kStripT = 5, kStripRows = 4200;
constexpr int kStripWin = kStripRows + 32 * kStripT + 64;

__global__ void __launch_bounds__(256) k_peak_strip(uint32_t* out, int iters) {
  extern __shared__ uint32_t sm[];
  uint32_t* A = sm;
  uint32_t* Bv = sm + kStripWin;
  for (int i = threadIdx.x; i < kStripWin; i += blockDim.x) A[i] = (uint32_t)(i * 2654435761u) ^ blockIdx.x;
  for (int i = threadIdx.x; i < kStripRows; i += blockDim.x) Bv[i] = (uint32_t)(i * 40503u + 7u) ^ (blockIdx.x << 8);
  __syncthreads();
  const uint32_t* Aw = A + kStripRows + (threadIdx.x & 31) * kStripT;
  constexpr int T = kStripT;
  uint32_t a0[T], a1[T], a2[T];
#pragma unroll
  for (int c = 0; c < T; c++) a0[c] = a1[c] = a2[c] = 0u;
  for (int it = 0; it < iters; it++) {
    uint32_t ring[T];
#pragma unroll
    for (int c = 1; c < T; c++) ring[c] = Aw[c];
    ring[0] = 0u;
    for (int j = 0; j < kStripRows; j += T) {
#pragma unroll
      for (int r = 0; r < T; r++) {
        ring[(T - r) % T] = Aw[-(j + r)];
        const uint32_t bj = Bv[j + r];
#pragma unroll
        for (int c = 0; c < T; c++) mp::mac3(a0[c], a1[c], a2[c], ring[(c - r + T) % T], bj);
      }
    }
  }
  uint32_t s = 0u;
#pragma unroll
  for (int c = 0; c < T; c++) s ^= a0[c] ^ a1[c] ^ a2[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
static_assert(kStripRows % kStripT == 0, "whole row groups");
}  // namespace

void* mp_kernel_peak(int kind, int* ops_per_round, int* smem_bytes, int* blocks_per_sm) {
  *ops_per_round = kind == 2 ? kStripRows * kStripT : kAcc;
  *smem_bytes = kind == 2 ? (kStripWin + kStripRows) * 4 : 0;
  *blocks_per_sm = kind == 2 ? 2 : 8;
  return kind == 0 ? (void*)k_peak_mac3 : kind == 1 ? (void*)k_peak_imad : (void*)k_peak_strip;
}

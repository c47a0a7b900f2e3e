// Allocation-free form of the mixed-precision persistent launch.
//
// mpdiv_batch_ragged needs a library context, and the context allocates device
// memory (its queue head and the size-sorted order array) and captures CUDA
// graphs. Some callers cannot allocate device memory at the point they divide:
// code that runs while a memory pool owns the whole device, allocators that
// forbid cudaMalloc after start-up, or hosts embedding the library under a
// strict memory budget. mpdiv_batch_ragged_noalloc serves them: the queue head
// and the order array live in the fixed scratch array below, which is part of
// the loaded library image, and nothing is allocated on any call.
//
// The scratch is one array per GPU that loads the library, held until the
// process exits. Every call uses the same array: a call first clears the queue
// head and the bucket counters, then builds the order, then runs the division
// kernel. Two calls whose work overlaps on the GPU (for instance on two
// streams) race on the array and corrupt each other's queue; serialise them.
#define MP_VECTOR_IO 0  // digit-by-digit operand loads and result stores (see mp_block.cuh)
#include <algorithm>
#include <mutex>

#include <cuda_runtime.h>

#include "mp_kernels.cuh"
#include "mpdiv.h"

cudaError_t mpdiv_open_kernel_smem(void* k, int smem);  // mpdiv.cu: raise-only, shared with the context path

namespace {

constexpr int kBuckets = 64;
constexpr int kScratchInts = MPDIV_NOALLOC_MAX_ITEMS + 2 * kBuckets + 64;

// [0, 64): queue head and padding; [64, 64 + 2*kBuckets): bucket counts and
// cursors; then the order array of at most MPDIV_NOALLOC_MAX_ITEMS items.
static __device__ __align__(256) int32_t g_noalloc_scratch[kScratchInts];

constexpr int kHead = 0;
constexpr int kCount = 64;
constexpr int kCursor = 64 + kBuckets;
constexpr int kOrder = 64 + 2 * kBuckets;

// Cost bucket of an item: floor(log2) of the quotient/remainder/Newton product
// estimate, so that larger buckets hold the more expensive divisions.
__device__ __forceinline__ int cost_bucket(int n, int kl) {
  const long long a = (long long)max(1, n - kl + 1);
  const long long c = a * (long long)(n + kl) + 2 * a * min((long long)kl, a) + 64;
  // lengths are validated on the host only, so keep the bucket in range for any
  // device values (c >= 64 gives a bucket of at least 6)
  return max(0, min(kBuckets - 1, 63 - __clzll((unsigned long long)max(c, 64LL))));
}

// One block: clear the head and counters, then order the items by cost bucket,
// most expensive bucket first (within a bucket the order is arbitrary: each
// division is independent of the others, so the results do not depend on it).
__global__ void __launch_bounds__(1024) k_noalloc_order(int32_t* scratch, const int32_t* u_len,
                                                        const int32_t* v_len, int n) {
  int32_t* count = scratch + kCount;
  int32_t* cursor = scratch + kCursor;
  int32_t* order = scratch + kOrder;
  if (threadIdx.x < 64) scratch[kHead + threadIdx.x] = 0;
  if (threadIdx.x < kBuckets) count[threadIdx.x] = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) atomicAdd(&count[cost_bucket(u_len[i], v_len[i])], 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    int acc = 0;
    for (int b = kBuckets - 1; b >= 0; b--) {
      cursor[b] = acc;
      acc += count[b];
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const int slot = atomicAdd(&cursor[cost_bucket(u_len[i], v_len[i])], 1);
    order[slot] = i;
  }
}

constexpr int kWarps = 16;
constexpr int kMinBlocks = 2;

std::mutex g_setup_mu;
int32_t* g_scratch_ptr[64] = {};  // device address of the scratch array, per device

// Per-device set-up on the first call: the device address of the scratch array.
int scratch_for_current_device(int32_t** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return MPDIV_ECUDA;
  std::lock_guard<std::mutex> g(g_setup_mu);
  if (g_scratch_ptr[dev] == nullptr) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) return MPDIV_ECUDA;
    g_scratch_ptr[dev] = static_cast<int32_t*>(p);
  }
  *out = g_scratch_ptr[dev];
  return MPDIV_OK;
}

}  // namespace

extern "C" int mpdiv_batch_ragged_noalloc(int64_t n_items, const uint32_t* u, const int64_t* u_off,
                                          const int32_t* u_len, const uint32_t* v, const int64_t* v_off,
                                          const int32_t* v_len, uint32_t* q, const int64_t* q_off,
                                          const int32_t* q_len, uint32_t* r, const int64_t* r_off,
                                          const int32_t* r_len, int32_t* status, const int32_t* u_len_host,
                                          void* stream) {
  if (n_items < 0) return MPDIV_EINVAL;
  if (n_items == 0) return MPDIV_OK;
  if (n_items > MPDIV_NOALLOC_MAX_ITEMS) return MPDIV_EUNSUPPORTED;
  if (!u || !u_off || !u_len || !v || !v_off || !v_len || !q || !q_off || !q_len || !r || !r_off || !r_len ||
      !status || !u_len_host)
    return MPDIV_EINVAL;
  int max_u = 1;
  for (int64_t i = 0; i < n_items; i++) {
    if (u_len_host[i] < 1) return MPDIV_EINVAL;
    if (u_len_host[i] > MPDIV_MAX_LIMBS) return MPDIV_EUNSUPPORTED;
    max_u = std::max(max_u, (int)u_len_host[i]);
  }
  int32_t* scratch = nullptr;
  int rc = scratch_for_current_device(&scratch);
  if (rc != MPDIV_OK) return rc;
  int dev = 0, num_sms = 0, max_smem = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  const int smem = (mp::smem_words_for(max_u, true, mp::PAD) * 4 + 15) & ~15;
  if (smem > max_smem) return MPDIV_EUNSUPPORTED;
  void* k = (void*)mp::k_div_ragged<kWarps, kMinBlocks>;
  if (mpdiv_open_kernel_smem(k, smem) != cudaSuccess) return MPDIV_ECUDA;
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, 32 * kWarps, smem) != cudaSuccess || occ < 1)
    return MPDIV_ECUDA;
  cudaStream_t s = (cudaStream_t)stream;
  k_noalloc_order<<<1, 1024, 0, s>>>(scratch, u_len, v_len, (int)n_items);
  if (cudaGetLastError() != cudaSuccess) return MPDIV_ECUDA;
  mp::RaggedArgs a{};
  a.u = u;
  a.u_off = u_off;
  a.u_len = u_len;
  a.v = v;
  a.v_off = v_off;
  a.v_len = v_len;
  a.q = q;
  a.q_off = q_off;
  a.q_len = q_len;
  a.r = r;
  a.r_off = r_off;
  a.r_len = r_len;
  a.status = status;
  a.iters = nullptr;
  a.products = nullptr;
  a.order = scratch + kOrder;
  a.head = scratch + kHead;
  a.n = n_items;
  a.smem_words = smem / 4;
  a.flags = 0;
  const int64_t grid = std::max<int64_t>(1, std::min<int64_t>((int64_t)num_sms * occ, n_items));
  void* args[] = {&a};
  if (cudaLaunchKernel(k, dim3((unsigned)grid), dim3(32 * kWarps), args, smem, s) != cudaSuccess) return MPDIV_ECUDA;
  return MPDIV_OK;
}

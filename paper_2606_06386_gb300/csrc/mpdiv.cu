// Host side of the C ABI in include/mpdiv.h: argument checks, launch
// configuration, the size-sorted queue of the persistent launch and its CUDA
// graph cache, the shifted-inverse test entry and the block-size tuner.
// The serving loop lives in mpdiv_serve.cu.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "mp_div.cuh"
#include "mpdiv_kernels.h"
#include "mpdiv.h"
#include "mpdiv_internal.h"

using namespace mp;

// ------------------------------------------------------------------ kernels
namespace {

enum KernKind {
  KK_UNIFORM = MP_K_UNIFORM,
  KK_RAGGED = MP_K_RAGGED,
  KK_SHINV = MP_K_SHINV,
  KK_PERSIST = MP_K_PERSIST,
  KK_MUL = MP_K_MUL
};

// Instantiations by block size (mpdiv_k*.cu); the minimum-blocks bound caps
// registers at 64 per thread so that several blocks of the smaller size
// classes share an SM. The persistent kernel runs 8- or 16-warp blocks, the
// queue and test kernels 16-warp blocks.
void* kernel_for(KernKind kk, int warps) {
  if (kk == KK_PERSIST) return warps <= 8 ? mp_kernel_w8(MP_K_PERSIST) : mp_kernel_w16(MP_K_PERSIST);
  if (kk == KK_RAGGED || kk == KK_SHINV) return mp_kernel_w16(kk);  // 16-warp blocks only
  if (warps <= 1) return mp_kernel_w1(kk);
  if (warps <= 2) return mp_kernel_w2(kk);
  if (warps <= 4) return mp_kernel_w4(kk);
  if (warps <= 8) return mp_kernel_w8(kk);
  if (warps <= 16) return mp_kernel_w16(kk);
  return mp_kernel_w32(kk);
}

// Block size of the transform-enabled plain kernel that serves a request for
// w warps (4, 8, 16 or 32), and the kernel of a kind with the transform
// enabled (the plain launch at that block size; the queue and test kernels at
// 16).
int ntt_kernel_warps(int w) { return w <= 4 ? 4 : w <= 8 ? 8 : w <= 16 ? 16 : 32; }
void* ntt_kernel_for(KernKind kk, int warps) {
  if (kk == KK_UNIFORM) return mp_kernel_ntt_uniform(ntt_kernel_warps(warps));
  return mp_kernel_ntt_queue(kk);
}

}  // namespace

// ------------------------------------------------------------------ context helpers
int mpdiv_set_error(mpdiv_ctx* ctx, int code, const char* fmt, ...) {
  if (ctx) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    std::lock_guard<std::mutex> g(ctx->err_mu);
    ctx->err = buf;
  }
  return code;
}

int mpdiv_cuda_check(mpdiv_ctx* ctx, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return MPDIV_OK;
  return mpdiv_set_error(ctx, MPDIV_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

int mpdiv_smem_bytes(int max_digits, int flags, int tcols) {
  const bool clip = (flags & MPDIV_FLAG_FULL_PRODUCTS) == 0;
  return (smem_words_for(max_digits, clip, layout_pad(clip, tcols)) * 4 + 15) & ~15;
}

// Transform tables for the division kernels (null unless the context's full
// products may use the transform) and the digit count from which they do.
static const uint32_t* ntt_tables(const mpdiv_ctx* ctx) {
  return (ctx->cfg.flags & MPDIV_FLAG_NTT_PRODUCTS) ? ctx->d_ntt : nullptr;
}
static int ntt_cutoff(const mpdiv_ctx* ctx) {
  return ctx->cfg.transform_cutoff > 0 ? ctx->cfg.transform_cutoff : 4096;  // measured break-even on GB300
}

// Shared memory of a division launch whose dividends have at most max_digits
// digits: the layout, and with the transform enabled its scratch after it,
// four words per point of the longest transform that a product of two such
// operands can use within the device's limit (longer products take the strip
// multiply).
static int launch_smem_bytes(mpdiv_ctx* ctx, int max_digits, int tcols) {
  const int smem = mpdiv_smem_bytes(max_digits, ctx->cfg.flags, tcols);
  if (ntt_tables(ctx) == nullptr || smem > ctx->max_smem) return smem;
  int t = std::min(NTT_LOG_MAX, ntt_log(2 * max_digits));
  while (t > 0 && smem + (16 << t) > ctx->max_smem) t--;
  if (t == 0 || (1 << t) < ntt_cutoff(ctx)) return smem;
  return smem + (16 << t);
}

// The block size of the kernel instantiation that serves a request for w
// warps: 1, 2, 4, 8, 16 or 32 (the kernels are built for exactly that many
// warps, so a launch always uses this value).
static int kernel_warps(int w) {
  int k = 1;
  while (k < w && k < 32) k *= 2;
  return k;
}

int mpdiv_default_warps(mpdiv_ctx* ctx, int max_digits) {
  if (ctx->cfg.warps_per_block > 0) return kernel_warps(ctx->cfg.warps_per_block);
  {
    std::lock_guard<std::mutex> g(ctx->tune_mu);
    const int cls = mpdiv_size_class(max_digits);
    auto it = ctx->tuned.find(cls);
    if (it != ctx->tuned.end()) return kernel_warps(it->second.warps);
  }
  if (max_digits <= 2048) return 4;
  if (max_digits <= 4096) return 8;
  return 16;
}

int mpdiv_default_tcols(mpdiv_ctx* ctx, int max_digits) {
  if (ctx->cfg.mul_columns > 0) return ctx->cfg.mul_columns;
  {
    std::lock_guard<std::mutex> g(ctx->tune_mu);
    auto it = ctx->tuned.find(mpdiv_size_class(max_digits));
    if (it != ctx->tuned.end()) return it->second.tcols;
  }
  return 3;  // measured fastest at every size class on GB300 (mpdiv_autotune)
}

int mpdiv_default_kcut(mpdiv_ctx* ctx, int max_digits) {
  if (ctx->cfg.karatsuba_cutoff != 0) return ctx->cfg.karatsuba_cutoff < 0 ? 0 : ctx->cfg.karatsuba_cutoff;
  {
    std::lock_guard<std::mutex> g(ctx->tune_mu);
    auto it = ctx->tuned.find(mpdiv_size_class(max_digits));
    if (it != ctx->tuned.end()) return it->second.kcut;
  }
  return 0;  // untuned: schoolbook only
}

int mpdiv_ragged_form(const mpdiv_ctx* ctx) {
  return (ctx->cfg.flags & MPDIV_FLAG_PERSISTENT_QUEUE) ? RF_SPLIT : RF_CLASSES;
}

int mpdiv_default_regs(mpdiv_ctx* ctx, int max_digits) {
  if (ctx->cfg.registers == 64 || ctx->cfg.registers == 128) return ctx->cfg.registers;
  std::lock_guard<std::mutex> g(ctx->tune_mu);
  auto it = ctx->tuned.find(mpdiv_size_class(max_digits));
  return it != ctx->tuned.end() ? it->second.regs : 0;
}

int mpdiv_size_class(int digits) {
  int c = 128;
  while (c < digits) c *= 2;
  return c;
}

// The dynamic shared memory each kernel has been opened to, per device. The
// attribute belongs to the kernel, not to a context, so it is only ever raised:
// a launch that needs less than an earlier one (of any context) keeps the
// larger opening and skips the driver call.
static std::mutex g_open_mu;
static std::map<std::pair<int, void*>, int> g_smem_opened;

cudaError_t mpdiv_open_kernel_smem(void* k, int smem) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> g(g_open_mu);
  int& opened = g_smem_opened[std::make_pair(dev, k)];
  if (opened >= smem) return cudaSuccess;
  e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess) opened = smem;
  return e;
}

static int prepare_kernel(mpdiv_ctx* ctx, void* k, int smem) {
  return mpdiv_cuda_check(ctx, mpdiv_open_kernel_smem(k, smem), "cudaFuncSetAttribute(max dynamic shared memory)");
}

void* mp_kernel_list(int warps) {
  switch (warps) {
    case 1: return mp_kernel_list1();
    case 2: return mp_kernel_list2();
    case 4: return mp_kernel_list4();
    case 8: return mp_kernel_list8();
    case 16: return mp_kernel_list16();
    default: return mp_kernel_list32();
  }
}

// The 128-register build of the plain kernel for a block of w warps (4, 8
// or 16), or null.
static void* wide_uniform_kernel(int w) {
  return w == 4 ? mp_kernel_w4_wide() : w == 8 ? mp_kernel_w8_wide() : w == 16 ? mp_kernel_w16_wide() : nullptr;
}

// Resident blocks per SM of kernel k at that block size and shared memory (cached).
static int kernel_occupancy(mpdiv_ctx* ctx, void* k, int threads, int smem) {
  std::lock_guard<std::mutex> g(ctx->attr_mu);
  const auto key = std::make_tuple(k, threads, smem);
  auto it = ctx->occupancy.find(key);
  if (it != ctx->occupancy.end()) return it->second;
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, threads, smem) != cudaSuccess) occ = 0;
  ctx->occupancy[key] = occ;
  return occ;
}

// ------------------------------------------------------------------ init / destroy
// Streams and events of the class form's forked launches. The class runs are
// ordered largest first, and side stream i has the i-th highest priority, so
// that the block scheduler starts the largest divisions first and the smaller
// classes' blocks fill the SMs that free up (largest-first across the classes).
static int mpdiv_create_side_streams(mpdiv_ctx* ctx) {
  int rc = mpdiv_cuda_check(ctx, cudaEventCreateWithFlags(&ctx->fork_ev, cudaEventDisableTiming), "cudaEventCreate");
  int least = 0, greatest = 0;
  if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) least = greatest = 0;
  for (int i = 0; i < kMaxRuns && rc == MPDIV_OK; i++) {
    const int prio = std::min(least, greatest + i);  // numerically lower is higher priority
    rc = mpdiv_cuda_check(ctx, cudaStreamCreateWithPriority(&ctx->side[i], cudaStreamNonBlocking, prio),
                          "cudaStreamCreate");
    if (rc == MPDIV_OK)
      rc = mpdiv_cuda_check(ctx, cudaEventCreateWithFlags(&ctx->join_ev[i], cudaEventDisableTiming), "cudaEventCreate");
  }
  return rc;
}

static void mpdiv_destroy_side_streams(mpdiv_ctx* ctx) {
  for (int i = 0; i < kMaxRuns; i++) {
    if (ctx->side[i]) cudaStreamDestroy(ctx->side[i]);
    if (ctx->join_ev[i]) cudaEventDestroy(ctx->join_ev[i]);
    ctx->side[i] = nullptr;
    ctx->join_ev[i] = nullptr;
  }
  if (ctx->fork_ev) cudaEventDestroy(ctx->fork_ev);
  ctx->fork_ev = nullptr;
}
extern "C" int mpdiv_init(mpdiv_ctx** out, int device, const mpdiv_config* cfg) {
  if (!out) return MPDIV_EINVAL;
  *out = nullptr;
  mpdiv_ctx* ctx = new mpdiv_ctx();
  ctx->device = device;
  if (cfg) ctx->cfg = *cfg;
  if (ctx->cfg.registers != 0 && ctx->cfg.registers != 64 && ctx->cfg.registers != 128) {
    delete ctx;
    return MPDIV_EINVAL;
  }
  int rc;
  if ((rc = mpdiv_cuda_check(ctx, cudaSetDevice(device), "cudaSetDevice")) != MPDIV_OK) {
    delete ctx;
    return rc;
  }
  cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
  cudaDeviceGetAttribute(&ctx->max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
  cudaDeviceGetAttribute(&ctx->smem_per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, device);
  if (ctx->cfg.flags & MPDIV_FLAG_NTT_PRODUCTS) ctx->cfg.flags |= MPDIV_FLAG_FULL_PRODUCTS;
  if ((rc = mpdiv_cuda_check(ctx, cudaMalloc(&ctx->d_head, 64), "cudaMalloc(queue head)")) != MPDIV_OK) {
    delete ctx;
    return rc;
  }
  {
    std::vector<uint32_t> tab(mp_ntt::kWords);
    mp_ntt::build_tables(tab.data());
    rc = mpdiv_cuda_check(ctx, cudaMalloc(&ctx->d_ntt, sizeof(uint32_t) * tab.size()), "cudaMalloc(transform tables)");
    if (rc == MPDIV_OK)
      rc = mpdiv_cuda_check(
          ctx, cudaMemcpy(ctx->d_ntt, tab.data(), sizeof(uint32_t) * tab.size(), cudaMemcpyHostToDevice),
          "upload of the transform tables");
    if (rc != MPDIV_OK) {
      if (ctx->d_ntt) cudaFree(ctx->d_ntt);
      cudaFree(ctx->d_head);
      delete ctx;
      return rc;
    }
  }
  if ((rc = mpdiv_cuda_check(ctx, cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking),
                             "cudaStreamCreate")) != MPDIV_OK ||
      (rc = mpdiv_cuda_check(ctx, cudaEventCreateWithFlags(&ctx->ragged_ev, cudaEventDisableTiming),
                             "cudaEventCreate")) != MPDIV_OK ||
      (rc = mpdiv_create_side_streams(ctx)) != MPDIV_OK) {
    mpdiv_destroy_side_streams(ctx);
    if (ctx->ragged_ev) cudaEventDestroy(ctx->ragged_ev);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    cudaFree(ctx->d_ntt);
    cudaFree(ctx->d_head);
    delete ctx;
    return rc;
  }
  const char* tf = getenv("MPDIV_TUNE_FILE");
  if (tf) mpdiv_tune_load(ctx, tf);
  *out = ctx;
  return MPDIV_OK;
}

extern "C" void mpdiv_destroy(mpdiv_ctx* ctx) {
  if (!ctx) return;
  mpdiv_serve_shutdown(ctx);
  cudaSetDevice(ctx->device);
  if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
  if (ctx->d_order) cudaFree(ctx->d_order);
  if (ctx->d_head) cudaFree(ctx->d_head);
  if (ctx->d_ntt) cudaFree(ctx->d_ntt);
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  if (ctx->ragged_ev) cudaEventDestroy(ctx->ragged_ev);
  if (ctx->cgexec) cudaGraphExecDestroy(ctx->cgexec);
  mpdiv_destroy_side_streams(ctx);
  delete ctx;
}

extern "C" const char* mpdiv_last_error(const mpdiv_ctx* ctx) {
  if (!ctx) return "null context";
  return ctx->err.c_str();
}

// ------------------------------------------------------------------ plain batch
// Kernel, arguments and launch shape of a plain launch (the kernel's shared
// memory attribute is raised here, outside any stream capture).
int mpdiv_prepare_uniform(mpdiv_ctx* ctx, const UniformLaunch& L, PreparedLaunch* P) {
  const int max_digits = L.un;
  const int tcols = L.tcols > 0 ? L.tcols : mpdiv_default_tcols(ctx, max_digits);
  const int smem = launch_smem_bytes(ctx, max_digits, tcols);
  if (smem > ctx->max_smem)
    return mpdiv_set_error(ctx, MPDIV_EUNSUPPORTED, "needs %d bytes of shared memory, device allows %d", smem,
                           ctx->max_smem);
  int warps = L.warps > 0 ? kernel_warps(L.warps) : mpdiv_default_warps(ctx, max_digits);
  if (ntt_tables(ctx)) warps = ntt_kernel_warps(warps);
  if (L.list != nullptr && ntt_tables(ctx) != nullptr)
    return mpdiv_set_error(ctx, MPDIV_EINVAL, "item lists are not built with the transform");
  void* k = L.list != nullptr ? mp_kernel_list(warps)
            : ntt_tables(ctx)  ? ntt_kernel_for(KK_UNIFORM, warps)
                               : kernel_for(KK_UNIFORM, warps);
  int rc = prepare_kernel(ctx, k, smem);
  if (rc) return rc;
  // 128 registers per thread where the block size has such a build and the
  // tuner or the configuration asks for it (strided launches only). Not by
  // default: on GB300 the 128-register builds ran 0.5-6 % slower than the
  // 64-register ones at every sweep size, although shared memory held the SM
  // to as few blocks as 128 registers allow and the 64-register builds spill a
  // few hundred bytes
  if (void* kw = (ntt_tables(ctx) || L.list) ? nullptr : wide_uniform_kernel(warps)) {
    const int regs = L.regs > 0 ? L.regs : mpdiv_default_regs(ctx, max_digits);
    if (regs == 128) {
      if ((rc = prepare_kernel(ctx, kw, smem))) return rc;
      k = kw;
    }
  }
  UniformArgs& a = P->args;
  std::memset(&a, 0, sizeof a);  // launch descriptors are compared bytewise by the graph cache
  a.u = L.u;
  a.v = L.v;
  a.q = L.q;
  a.r = L.r;
  a.status = L.status;
  a.iters = L.iters;
  a.products = L.products;
  a.n = L.n;
  a.us = L.us;
  a.vs = L.vs;
  a.qs = L.qs;
  a.rs = L.rs;
  a.un = L.un;
  a.vn = L.vn;
  a.qn = L.qn;
  a.rn = L.rn;
  a.smem_words = smem / 4;
  a.flags = ctx->cfg.flags;
  a.tcols = tcols;
  a.kcut = L.kcut >= 0 ? L.kcut : mpdiv_default_kcut(ctx, max_digits);
  a.ntt = ntt_tables(ctx);
  a.ntt_cut = ntt_cutoff(ctx);
  a.list = L.list;
  a.u_off = L.u_off;
  a.v_off = L.v_off;
  a.q_off = L.q_off;
  a.r_off = L.r_off;
  a.u_len = L.u_len;
  a.v_len = L.v_len;
  a.q_len = L.q_len;
  a.r_len = L.r_len;
  P->kernel = k;
  P->grid = std::min<int64_t>(L.n, 0x7fffffff);
  P->threads = 32 * warps;
  P->smem = smem;
  P->retry_grid = 0;
  P->retry_smem = 0;
  // clipped products without the transform: a fit pass with shared memory for
  // the batch's own operand lengths (the largest plan of the listed items, or
  // of a uniform batch's digit counts) when it lets more blocks share an SM,
  // then a retry pass for the items whose effective lengths need more
  const bool clip = (ctx->cfg.flags & MPDIV_FLAG_FULL_PRODUCTS) == 0;
  if (clip && ntt_tables(ctx) == nullptr) {
    const int pad = layout_pad(true, tcols);
    int fit_words = 0;
    if (L.list == nullptr) {
      fit_words = layout_words(L.un, std::min(L.vn, L.un), true, pad);
    } else if (L.list_host != nullptr) {
      for (int64_t i = 0; i < L.n; i++) {
        const int it = L.list_host[i];
        const int h = L.u_len_host[it], kl = std::min(L.v_len_host[it], h);
        fit_words = std::max(fit_words, layout_words(h, kl, true, pad));
      }
    }
    const int fit = (fit_words * 4 + 15) & ~15;
    if (fit > 0 && fit < smem) {
      const int occ_fit = kernel_occupancy(ctx, k, 32 * warps, fit);
      const int occ_full = kernel_occupancy(ctx, k, 32 * warps, smem);
      // only a batch of more than one wave of full-size blocks gains from
      // more blocks per SM; a smaller one keeps one launch
      if (occ_full >= 1 && occ_fit > occ_full && L.n > (int64_t)ctx->num_sms * occ_full) {
        a.pass = 1;
        a.smem_words = fit / 4;
        P->smem = fit;
        P->retry_smem = smem;
        // one block per item, as the fit pass: the items it leaves can be many
        // and of uneven cost (divisors shorter than the batch's digit count),
        // and the block scheduler balances them; the others exit at once
        P->retry_grid = std::min<int64_t>(L.n, 0x7fffffff);
      }
    }
  }
  return MPDIV_OK;
}

int mpdiv_launch_prepared(mpdiv_ctx* ctx, const PreparedLaunch& P, cudaStream_t stream) {
  UniformArgs a = P.args;
  void* args[] = {&a};
  cudaError_t e = cudaLaunchKernel(P.kernel, dim3((unsigned)P.grid), dim3(P.threads), args, P.smem, stream);
  int rc = mpdiv_cuda_check(ctx, e, "launch of the division kernel");
  if (rc != MPDIV_OK || P.retry_grid == 0) return rc;
  // the retry pass: the items the fit pass left, in shared memory for any item
  a.pass = 2;
  a.smem_words = P.retry_smem / 4;
  e = cudaLaunchKernel(P.kernel, dim3((unsigned)P.retry_grid), dim3(P.threads), args, P.retry_smem, stream);
  return mpdiv_cuda_check(ctx, e, "launch of the division kernel's retry pass");
}

int mpdiv_launch_uniform(mpdiv_ctx* ctx, const UniformLaunch& L, cudaStream_t stream) {
  PreparedLaunch P;
  int rc = mpdiv_prepare_uniform(ctx, L, &P);
  if (rc) return rc;
  return mpdiv_launch_prepared(ctx, P, stream);
}

extern "C" int mpdiv_batch(mpdiv_ctx* ctx, int64_t n_items, const uint32_t* u, int32_t u_limbs, int64_t u_stride,
                           const uint32_t* v, int32_t v_limbs, int64_t v_stride, uint32_t* q, int32_t q_limbs,
                           int64_t q_stride, uint32_t* r, int32_t r_limbs, int64_t r_stride, int32_t* status,
                           int32_t* iters, int64_t* products, void* stream) {
  MpdivRange nvtx_range("mpdiv.batch");
  if (!ctx) return MPDIV_EINVAL;
  if (n_items < 0) return mpdiv_set_error(ctx, MPDIV_EINVAL, "n_items < 0");
  if (n_items == 0) return MPDIV_OK;
  if (!u || !v || !q || !r || !status) return mpdiv_set_error(ctx, MPDIV_EINVAL, "null pointer argument");
  if (u_limbs < 1 || v_limbs < 1 || q_limbs < 1 || r_limbs < 1)
    return mpdiv_set_error(ctx, MPDIV_EINVAL, "digit counts must be positive");
  if (u_limbs > MPDIV_MAX_LIMBS || v_limbs > MPDIV_MAX_LIMBS)
    return mpdiv_set_error(ctx, MPDIV_EUNSUPPORTED, "at most %d digits per operand", MPDIV_MAX_LIMBS);
  if (r_limbs < v_limbs) return mpdiv_set_error(ctx, MPDIV_EINVAL, "r_limbs < v_limbs");
  if (u_stride < u_limbs || v_stride < v_limbs || q_stride < q_limbs || r_stride < r_limbs)
    return mpdiv_set_error(ctx, MPDIV_EINVAL, "a stride is shorter than its digit count");
  cudaSetDevice(ctx->device);
  UniformLaunch L{};
  L.u = u;
  L.v = v;
  L.q = q;
  L.r = r;
  L.status = status;
  L.iters = iters;
  L.products = products;
  L.n = n_items;
  L.us = u_stride;
  L.vs = v_stride;
  L.qs = q_stride;
  L.rs = r_stride;
  L.un = u_limbs;
  L.vn = v_limbs;
  L.qn = q_limbs;
  L.rn = r_limbs;
  L.warps = 0;
  L.tcols = 0;
  L.kcut = -1;
  L.regs = 0;
  return mpdiv_launch_uniform(ctx, L, (cudaStream_t)stream);
}

extern "C" int mpdiv_batch_launches(mpdiv_ctx* ctx, int64_t n_items, int32_t u_limbs, int32_t v_limbs) {
  if (!ctx) return MPDIV_EINVAL;
  if (n_items < 1 || u_limbs < 1 || v_limbs < 1) return mpdiv_set_error(ctx, MPDIV_EINVAL, "bad shape");
  if (u_limbs > MPDIV_MAX_LIMBS || v_limbs > MPDIV_MAX_LIMBS)
    return mpdiv_set_error(ctx, MPDIV_EUNSUPPORTED, "at most %d digits per operand", MPDIV_MAX_LIMBS);
  cudaSetDevice(ctx->device);
  UniformLaunch L{};
  L.n = n_items;
  L.un = u_limbs;
  L.vn = v_limbs;
  L.kcut = -1;
  PreparedLaunch P;
  const int rc = mpdiv_prepare_uniform(ctx, L, &P);
  if (rc) return rc;
  return P.retry_grid > 0 ? 2 : 1;
}

// ------------------------------------------------------------------ ragged (persistent) batch
// Cost estimate used to order the queue (largest first): limb products of the
// quotient and remainder products plus the Newton refinement, from the
// multiplication-count model of Section 2.3.
static double item_cost(int n, int kl) {
  if (kl > n) return 1.0;
  const double a = n - kl + 1;
  const double newton = 2.0 * a * std::min<double>(kl, a);
  return a * n + a * kl + newton + 64.0;
}

// The self-splitting persistent launch's shape: per size class the strip
// width, Karatsuba cutoff and warps wanted (the plain launch's tuned shape),
// the block size (8 warps, or 16 when a class wants more than 8) and the
// shared memory per block: enough for the largest item, and where the budget
// of two (one) resident blocks per SM allows, for a class that wants half
// (a quarter) of the block's warps to run in half (a quarter) of it.
static void persistent_shape(mpdiv_ctx* ctx, int max_u, RaggedArgs& a, int* warps, int* smem_words) {
  static const int kClassMax[5] = {1024, 2048, 4096, 8192, 16384};
  const bool clip = (ctx->cfg.flags & MPDIV_FLAG_FULL_PRODUCTS) == 0;
  const int cmax = class_of(max_u);
  int wmax = 1;
  for (int c = 0; c < 5; c++) {
    a.tcols_class[c] = mpdiv_default_tcols(ctx, kClassMax[c]);
    a.kcut_class[c] = mpdiv_default_kcut(ctx, kClassMax[c]);
    a.want_class[c] = std::max(1, std::min(32, mpdiv_default_warps(ctx, kClassMax[c])));
    if (c <= cmax) wmax = std::max(wmax, a.want_class[c]);
  }
  const int nw = wmax > 8 ? 16 : 8;
  const int minb = nw == 8 ? 2 : 1;
  for (int c = 0; c < 5; c++) a.want_class[c] = std::max(nw / 4, std::min(nw, a.want_class[c]));
  auto need = [&](int c) {
    const int d = std::min(max_u, kClassMax[c]);
    return smem_words_for(d, clip, layout_pad(clip, a.tcols_class[c]));
  };
  int words = 0;
  for (int c = 0; c <= cmax; c++) words = std::max(words, need(c));
  const int budget = std::min(ctx->max_smem, (ctx->smem_per_sm - minb * 1024) / minb) / 4;
  for (int c = 0; c <= cmax; c++) {
    int cand = 0;
    if (a.want_class[c] <= nw / 2) cand = 2 * need(c) + 8;
    if (a.want_class[c] <= nw / 4) cand = std::max(cand, 4 * need(c) + 16);
    if (cand <= budget) words = std::max(words, cand);
  }
  *warps = nw;
  *smem_words = (words + 3) & ~3;
}

// The order of a ragged batch's items on the device (and its host copy):
// the caller's (L.order, L.order_host), else built here and cached with a
// copy of the shape list and the form it was made for, reused only when both
// length arrays are equal to the cached ones entry for entry. Called with
// ctx->ragged_mu held. The class form orders by size class, largest first,
// then by cost; the queue forms by dividend length (the shared memory a
// self-splitting group must hold), then by cost.
static int ragged_order(mpdiv_ctx* ctx, const RaggedLaunch& L, int form, const int32_t** d_order,
                        const int32_t** h_order, bool* same_shapes) {
  if (L.order != nullptr) {
    *d_order = L.order;
    *h_order = L.order_host;
    *same_shapes = true;
    return MPDIV_OK;
  }
  *same_shapes = L.n == ctx->order_n && ctx->order_form == form && (size_t)L.n == ctx->order_u_len.size() &&
                 std::memcmp(ctx->order_u_len.data(), L.u_len_host, sizeof(int32_t) * L.n) == 0 &&
                 std::memcmp(ctx->order_v_len.data(), L.v_len_host, sizeof(int32_t) * L.n) == 0;
  if (!*same_shapes) {
    int rc;
    // the previous launch may still read the order array on another stream
    if ((rc = mpdiv_cuda_check(ctx, cudaEventSynchronize(ctx->ragged_ev), "wait for the previous queue launch")))
      return rc;
    std::vector<int32_t>& order = ctx->order_host;
    order.resize(L.n);
    std::iota(order.begin(), order.end(), 0);
    std::vector<double> cost(L.n);
    for (int64_t i = 0; i < L.n; i++) cost[i] = item_cost(L.u_len_host[i], L.v_len_host[i]);
    if (form == RF_CLASSES) {
      std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        const int ca = class_of(L.u_len_host[a]), cb = class_of(L.u_len_host[b]);
        if (ca != cb) return ca > cb;
        return cost[a] > cost[b];
      });
    } else {
      std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        if (L.u_len_host[a] != L.u_len_host[b]) return L.u_len_host[a] > L.u_len_host[b];
        return cost[a] > cost[b];
      });
    }
    if ((size_t)L.n > ctx->order_cap) {
      if (ctx->d_order) cudaFree(ctx->d_order);
      ctx->d_order = nullptr;
      ctx->order_cap = 0;
      if ((rc = mpdiv_cuda_check(ctx, cudaMalloc(&ctx->d_order, sizeof(int32_t) * L.n), "cudaMalloc(order)")))
        return rc;
      ctx->order_cap = L.n;
    }
    if ((rc = mpdiv_cuda_check(
             ctx, cudaMemcpy(ctx->d_order, order.data(), sizeof(int32_t) * L.n, cudaMemcpyHostToDevice),
             "upload of the queue order")))
      return rc;
    ctx->order_u_len.assign(L.u_len_host, L.u_len_host + L.n);
    ctx->order_v_len.assign(L.v_len_host, L.v_len_host + L.n);
    ctx->order_n = L.n;
    ctx->order_form = form;
  }
  *d_order = ctx->d_order;
  *h_order = ctx->order_host.data();
  return MPDIV_OK;
}

// The class form: the ordered items fall into runs of one size class; each
// run is one plain launch (the class's tuned warps, strip width and register
// budget, shared memory for its largest dividend) over its item list. With
// several runs the launches are independent branches forked from `stream`
// and joined back to it, so that the blocks of one class fill the last wave
// of another; with use_graph they are captured and replayed as one CUDA graph.
static int launch_ragged_classes(mpdiv_ctx* ctx, const RaggedLaunch& L, const int32_t* d_order,
                                 const int32_t* h_order, bool same_shapes, cudaStream_t stream) {
  std::vector<PreparedLaunch> runs;
  int64_t start = 0;
  while (start < L.n) {
    const int cls = class_of(L.u_len_host[h_order[start]]);
    int64_t end = start;
    int max_u = 1;
    while (end < L.n && class_of(L.u_len_host[h_order[end]]) == cls) max_u = std::max(max_u, L.u_len_host[h_order[end++]]);
    UniformLaunch U{};
    U.u = L.u;
    U.v = L.v;
    U.q = L.q;
    U.r = L.r;
    U.status = L.status;
    U.iters = L.iters;
    U.products = L.products;
    U.n = end - start;
    U.un = max_u;
    U.vn = U.qn = U.rn = 1;
    U.kcut = -1;
    U.list = d_order + start;
    U.u_off = L.u_off;
    U.v_off = L.v_off;
    U.q_off = L.q_off;
    U.r_off = L.r_off;
    U.u_len = L.u_len;
    U.v_len = L.v_len;
    U.q_len = L.q_len;
    U.r_len = L.r_len;
    U.list_host = h_order + start;
    U.u_len_host = L.u_len_host;
    U.v_len_host = L.v_len_host;
    runs.emplace_back();
    int rc = mpdiv_prepare_uniform(ctx, U, &runs.back());
    if (rc) return rc;
    start = end;
  }
  if ((int)runs.size() > kMaxRuns) return mpdiv_set_error(ctx, MPDIV_EINVAL, "more size classes than expected");
  auto fork_join = [&](cudaStream_t s) -> int {
    if (runs.size() == 1) return mpdiv_launch_prepared(ctx, runs[0], s);
    int rc = mpdiv_cuda_check(ctx, cudaEventRecord(ctx->fork_ev, s), "fork");
    for (size_t i = 0; i < runs.size() && rc == MPDIV_OK; i++) {
      rc = mpdiv_cuda_check(ctx, cudaStreamWaitEvent(ctx->side[i], ctx->fork_ev, 0), "fork");
      if (rc == MPDIV_OK) rc = mpdiv_launch_prepared(ctx, runs[i], ctx->side[i]);
      if (rc == MPDIV_OK) rc = mpdiv_cuda_check(ctx, cudaEventRecord(ctx->join_ev[i], ctx->side[i]), "join");
      if (rc == MPDIV_OK) rc = mpdiv_cuda_check(ctx, cudaStreamWaitEvent(s, ctx->join_ev[i], 0), "join");
    }
    return rc;
  };
  if (!L.use_graph) return fork_join(stream);
  // the graph is replayed while the launches are unchanged
  std::vector<char> desc(sizeof(PreparedLaunch) * runs.size());
  for (size_t i = 0; i < runs.size(); i++) {
    PreparedLaunch P{};
    std::memset(&P, 0, sizeof P);
    P.kernel = runs[i].kernel;
    P.args = runs[i].args;
    P.grid = runs[i].grid;
    P.threads = runs[i].threads;
    P.smem = runs[i].smem;
    P.retry_grid = runs[i].retry_grid;
    P.retry_smem = runs[i].retry_smem;
    std::memcpy(desc.data() + i * sizeof P, &P, sizeof P);
  }
  int rc;
  if (!(ctx->cgexec && same_shapes && desc == ctx->c_desc)) {
    if (ctx->cgexec) {
      cudaGraphExecDestroy(ctx->cgexec);
      ctx->cgexec = nullptr;
    }
    cudaGraph_t graph = nullptr;
    if ((rc = mpdiv_cuda_check(ctx, cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal),
                               "begin graph capture")))
      return rc;
    const int le = fork_join(ctx->cap_stream);
    cudaError_t ee = cudaStreamEndCapture(ctx->cap_stream, &graph);
    if (le != MPDIV_OK) {
      if (graph) cudaGraphDestroy(graph);
      return le;
    }
    if ((rc = mpdiv_cuda_check(ctx, ee, "end graph capture"))) return rc;
    cudaError_t ie = cudaGraphInstantiate(&ctx->cgexec, graph, 0);
    cudaGraphDestroy(graph);
    if ((rc = mpdiv_cuda_check(ctx, ie, "graph instantiate"))) {
      ctx->cgexec = nullptr;
      return rc;
    }
    ctx->c_desc = desc;
    ctx->graph_captures++;
  } else {
    ctx->graph_replays++;
  }
  return mpdiv_cuda_check(ctx, cudaGraphLaunch(ctx->cgexec, stream), "graph launch");
}

int mpdiv_launch_ragged(mpdiv_ctx* ctx, const RaggedLaunch& L, cudaStream_t stream) {
  int max_u = 1;
  for (int64_t i = 0; i < L.n; i++) max_u = std::max(max_u, (int)L.u_len_host[i]);
  // the self-splitting kernel and the item-list kernels are built without the transform
  const int form = (L.form != RF_QUEUE && ntt_tables(ctx) != nullptr) ? RF_QUEUE : L.form;
  std::lock_guard<std::mutex> g(ctx->ragged_mu);
  // launches with the context's queue head and order array are ordered on the
  // GPU one after another, whatever their streams (ragged_ev marks the last one)
  const bool ctx_queue = L.order == nullptr;
  const int32_t* d_order = nullptr;
  const int32_t* h_order = nullptr;
  bool same_shapes = false;
  int rc = ragged_order(ctx, L, form, &d_order, &h_order, &same_shapes);
  if (rc) return rc;
  if (ctx_queue &&
      (rc = mpdiv_cuda_check(ctx, cudaStreamWaitEvent(stream, ctx->ragged_ev, 0), "order after the previous launch")))
    return rc;
  if (form == RF_CLASSES) {
    rc = launch_ragged_classes(ctx, L, d_order, h_order, same_shapes, stream);
    if (rc == MPDIV_OK && ctx_queue) rc = mpdiv_cuda_check(ctx, cudaEventRecord(ctx->ragged_ev, stream), "event");
    return rc;
  }
  RaggedArgs a;
  std::memset(&a, 0, sizeof a);  // the graph cache compares argument blocks bytewise
  int warps = 0, smem = 0;
  const bool split = form == RF_SPLIT;
  if (split) {
    int words = 0;
    persistent_shape(ctx, max_u, a, &warps, &words);
    smem = words * 4;
  } else {
    smem = launch_smem_bytes(ctx, max_u, T_MAX);  // any strip width per item
    warps = 16;  // the one-block-per-item queue kernel is built for 16-warp blocks
  }
  if (smem > ctx->max_smem)
    return mpdiv_set_error(ctx, MPDIV_EUNSUPPORTED, "needs %d bytes of shared memory", smem);
  void* k = split ? kernel_for(KK_PERSIST, warps)
                  : (ntt_tables(ctx) ? ntt_kernel_for(KK_RAGGED, warps) : kernel_for(KK_RAGGED, warps));
  if ((rc = prepare_kernel(ctx, k, smem))) return rc;
  int occ = kernel_occupancy(ctx, k, 32 * warps, smem);
  if (occ < 1) return mpdiv_set_error(ctx, MPDIV_EUNSUPPORTED, "kernel does not fit on an SM");
  if (ctx->cfg.blocks_per_sm > 0) occ = std::min(occ, ctx->cfg.blocks_per_sm);
  int64_t grid = (int64_t)ctx->num_sms * occ;
  if (L.grid_items) grid = L.n;  // one block per item: later launches backfill freed SMs
  grid = std::max<int64_t>(1, std::min<int64_t>(grid, std::min<int64_t>(L.n, 0x7fffffff)));
  a.u = L.u;
  a.u_off = L.u_off;
  a.u_len = L.u_len;
  a.v = L.v;
  a.v_off = L.v_off;
  a.v_len = L.v_len;
  a.q = L.q;
  a.q_off = L.q_off;
  a.q_len = L.q_len;
  a.r = L.r;
  a.r_off = L.r_off;
  a.r_len = L.r_len;
  a.status = L.status;
  a.iters = L.iters;
  a.products = L.products;
  a.order = d_order;
  a.head = L.head ? L.head : ctx->d_head;
  a.n = L.n;
  a.smem_words = smem / 4;
  a.flags = ctx->cfg.flags;
  a.tcols = split ? 0 : mpdiv_default_tcols(ctx, max_u);  // persistent: per class (configured or tuned)
  a.kcut = split ? -1 : mpdiv_default_kcut(ctx, max_u);
  a.ntt = ntt_tables(ctx);
  a.ntt_cut = ntt_cutoff(ctx);
  if (!L.use_graph) {
    if ((rc = mpdiv_cuda_check(ctx, cudaMemsetAsync(a.head, 0, sizeof(int32_t), stream), "queue reset"))) return rc;
    void* args[] = {&a};
    rc = mpdiv_cuda_check(ctx, cudaLaunchKernel(k, dim3((unsigned)grid), dim3(32 * warps), args, smem, stream),
                          "launch of the persistent division kernel");
    if (rc == MPDIV_OK && ctx_queue) rc = mpdiv_cuda_check(ctx, cudaEventRecord(ctx->ragged_ev, stream), "event");
    return rc;
  }
  // CUDA graph: [reset queue head, persistent kernel], replayed while the
  // arguments are unchanged.
  const bool same_args = ctx->gexec && same_shapes && std::memcmp(&a, &ctx->g_args, sizeof a) == 0 &&
                         ctx->g_grid == grid && ctx->g_warps == warps && ctx->g_smem == smem;
  if (!same_args) {
    if (ctx->gexec) {
      cudaGraphExecDestroy(ctx->gexec);
      ctx->gexec = nullptr;
    }
    cudaGraph_t graph = nullptr;
    if ((rc = mpdiv_cuda_check(ctx, cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal),
                               "begin graph capture")))
      return rc;
    cudaMemsetAsync(a.head, 0, sizeof(int32_t), ctx->cap_stream);
    void* args[] = {&a};
    cudaError_t le = cudaLaunchKernel(k, dim3((unsigned)grid), dim3(32 * warps), args, smem, ctx->cap_stream);
    cudaError_t ee = cudaStreamEndCapture(ctx->cap_stream, &graph);
    if ((rc = mpdiv_cuda_check(ctx, le, "captured launch"))) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    if ((rc = mpdiv_cuda_check(ctx, ee, "end graph capture"))) return rc;
    cudaError_t ie = cudaGraphInstantiate(&ctx->gexec, graph, 0);
    cudaGraphDestroy(graph);
    if ((rc = mpdiv_cuda_check(ctx, ie, "graph instantiate"))) {
      ctx->gexec = nullptr;
      return rc;
    }
    ctx->g_args = a;
    ctx->g_grid = grid;
    ctx->g_warps = warps;
    ctx->g_smem = smem;
    ctx->graph_captures++;
  } else {
    ctx->graph_replays++;
  }
  rc = mpdiv_cuda_check(ctx, cudaGraphLaunch(ctx->gexec, stream), "graph launch");
  if (rc == MPDIV_OK && ctx_queue) rc = mpdiv_cuda_check(ctx, cudaEventRecord(ctx->ragged_ev, stream), "event");
  return rc;
}

extern "C" int mpdiv_batch_ragged(mpdiv_ctx* ctx, int64_t n_items, const uint32_t* u, const int64_t* u_off,
                                  const int32_t* u_len, const uint32_t* v, const int64_t* v_off,
                                  const int32_t* v_len, uint32_t* q, const int64_t* q_off, const int32_t* q_len,
                                  uint32_t* r, const int64_t* r_off, const int32_t* r_len, int32_t* status,
                                  int32_t* iters, int64_t* products, const int32_t* u_len_host,
                                  const int32_t* v_len_host, void* stream) {
  MpdivRange nvtx_range("mpdiv.batch_ragged");
  if (!ctx) return MPDIV_EINVAL;
  if (n_items < 0) return mpdiv_set_error(ctx, MPDIV_EINVAL, "n_items < 0");
  if (n_items == 0) return MPDIV_OK;
  if (!u || !u_off || !u_len || !v || !v_off || !v_len || !q || !q_off || !q_len || !r || !r_off || !r_len ||
      !status || !u_len_host || !v_len_host)
    return mpdiv_set_error(ctx, MPDIV_EINVAL, "null pointer argument");
  for (int64_t i = 0; i < n_items; i++) {
    if (u_len_host[i] < 1 || v_len_host[i] < 1)
      return mpdiv_set_error(ctx, MPDIV_EINVAL, "item %lld: digit counts must be positive", (long long)i);
    if (u_len_host[i] > MPDIV_MAX_LIMBS || v_len_host[i] > MPDIV_MAX_LIMBS)
      return mpdiv_set_error(ctx, MPDIV_EUNSUPPORTED, "item %lld: at most %d digits", (long long)i,
                             MPDIV_MAX_LIMBS);
  }
  cudaSetDevice(ctx->device);
  RaggedLaunch L{};
  L.u = u;
  L.u_off = u_off;
  L.u_len = u_len;
  L.v = v;
  L.v_off = v_off;
  L.v_len = v_len;
  L.q = q;
  L.q_off = q_off;
  L.q_len = q_len;
  L.r = r;
  L.r_off = r_off;
  L.r_len = r_len;
  L.status = status;
  L.iters = iters;
  L.products = products;
  L.u_len_host = u_len_host;
  L.v_len_host = v_len_host;
  L.n = n_items;
  L.use_graph = true;
  L.form = mpdiv_ragged_form(ctx);
  return mpdiv_launch_ragged(ctx, L, (cudaStream_t)stream);
}

// ------------------------------------------------------------------ shinv test entry
extern "C" int mpdiv_debug_shinv(mpdiv_ctx* ctx, int64_t n_items, const uint32_t* v, int32_t v_limbs,
                                 int64_t v_stride, const int32_t* h_digits, uint32_t* out, int32_t out_limbs,
                                 int64_t out_stride, int32_t* iters, int32_t* status, void* stream) {
  if (!ctx) return MPDIV_EINVAL;
  if (n_items <= 0) return n_items == 0 ? MPDIV_OK : mpdiv_set_error(ctx, MPDIV_EINVAL, "n_items < 0");
  if (!v || !h_digits || !out || !status) return mpdiv_set_error(ctx, MPDIV_EINVAL, "null pointer argument");
  if (v_limbs < 1 || out_limbs < 1 || v_stride < v_limbs || out_stride < out_limbs)
    return mpdiv_set_error(ctx, MPDIV_EINVAL, "bad sizes");
  if (v_limbs > MPDIV_MAX_LIMBS || out_limbs > MPDIV_MAX_LIMBS + 1)
    return mpdiv_set_error(ctx, MPDIV_EUNSUPPORTED, "too many digits");
  cudaSetDevice(ctx->device);
  // h_digits live on the device: size for the largest h that fits (the kernel
  // reports MPDIV_ST_INTERNAL for an item whose working set does not)
  const int tcols = ctx->cfg.mul_columns > 0 ? ctx->cfg.mul_columns : 5;
  int max_h = MPDIV_MAX_LIMBS;
  while (max_h > 256 && mpdiv_smem_bytes(max_h, ctx->cfg.flags, tcols) > ctx->max_smem) max_h -= 256;
  const int smem = mpdiv_smem_bytes(max_h, ctx->cfg.flags, tcols);
  const int warps = 16;  // the test entry is built for 16-warp blocks
  void* k = ntt_tables(ctx) ? ntt_kernel_for(KK_SHINV, warps) : kernel_for(KK_SHINV, warps);
  int rc = prepare_kernel(ctx, k, smem);
  if (rc) return rc;
  ShinvArgs a{};
  a.ntt = ntt_tables(ctx);  // per item, the shared memory its layout leaves
  a.ntt_cut = ntt_cutoff(ctx);
  a.v = v;
  a.h = h_digits;
  a.out = out;
  a.iters = iters;
  a.status = status;
  a.n = n_items;
  a.vs = v_stride;
  a.os = out_stride;
  a.vn = v_limbs;
  a.on = out_limbs;
  a.smem_words = smem / 4;
  a.tcols = tcols;
  a.kcut = ctx->cfg.karatsuba_cutoff > 0 ? ctx->cfg.karatsuba_cutoff : 0;
  a.flags = ctx->cfg.flags & MPDIV_FLAG_FULL_PRODUCTS;
  void* args[] = {&a};
  const int64_t grid = std::min<int64_t>(n_items, 0x7fffffff);
  return mpdiv_cuda_check(ctx, cudaLaunchKernel(k, dim3((unsigned)grid), dim3(32 * warps), args, smem,
                                                (cudaStream_t)stream),
                          "launch of the shifted-inverse kernel");
}

extern "C" int mpdiv_debug_primitive(mpdiv_ctx* ctx, int32_t op, int64_t n_items, const uint32_t* x, int32_t nx,
                                     const uint32_t* y, int32_t ny, int32_t arg, uint32_t* out, int32_t cap,
                                     int32_t* result, int32_t warps, void* stream) {
  if (!ctx) return MPDIV_EINVAL;
  if (n_items <= 0) return n_items == 0 ? MPDIV_OK : mpdiv_set_error(ctx, MPDIV_EINVAL, "n_items < 0");
  if (!x || !y || !out || !result) return mpdiv_set_error(ctx, MPDIV_EINVAL, "null pointer argument");
  if (op < 0 || op > 9) return mpdiv_set_error(ctx, MPDIV_EINVAL, "unknown primitive %d", op);
  if (op == 9 && nx + ny > NTT_MAX) return mpdiv_set_error(ctx, MPDIV_EUNSUPPORTED, "transform longer than %d", NTT_MAX);
  if (nx < 1 || ny < 1 || cap < 1 || arg < 0 || (op == 7 && cap < 3))
    return mpdiv_set_error(ctx, MPDIV_EINVAL, "bad sizes");
  if ((op == 0 || op == 1 || op == 8) && cap < std::max(nx, ny))
    return mpdiv_set_error(ctx, MPDIV_EINVAL, "cap shorter than the operands");
  if ((op == 4 || op == 5) && (cap < nx || arg >= cap)) return mpdiv_set_error(ctx, MPDIV_EINVAL, "bad power");
  cudaSetDevice(ctx->device);
  const int w = kernel_warps(warps < 1 ? 1 : warps);
  int words = 3 * PAD + nx + ny + cap + 4 + ov_words(cap);
  if (op == 9) words = ((words + 3) & ~3) + (4 << ntt_log(nx + ny));  // the transform's scratch
  const int smem = (words * 4 + 15) & ~15;
  if (smem > ctx->max_smem) return mpdiv_set_error(ctx, MPDIV_EUNSUPPORTED, "needs %d bytes of shared memory", smem);
  void* k = mp_kernel_prim(w);
  int rc = prepare_kernel(ctx, k, smem);
  if (rc) return rc;
  PrimArgs a;
  std::memset(&a, 0, sizeof a);
  a.x = x;
  a.y = y;
  a.out = out;
  a.result = result;
  a.n = n_items;
  a.nx = nx;
  a.ny = ny;
  a.cap = cap;
  a.op = op;
  a.arg = arg;
  a.tcols = ctx->cfg.mul_columns > 0 ? ctx->cfg.mul_columns : 3;
  a.smem_words = smem / 4;
  a.ntt = ctx->d_ntt;
  void* args[] = {&a};
  const int64_t grid = std::min<int64_t>(n_items, 0x7fffffff);
  return mpdiv_cuda_check(ctx, cudaLaunchKernel(k, dim3((unsigned)grid), dim3(32 * w), args, smem, (cudaStream_t)stream),
                          "launch of the primitive test kernel");
}

extern "C" int mpdiv_tuning(mpdiv_ctx* ctx, int32_t u_limbs, int32_t* warps, int32_t* mul_columns,
                            int32_t* karatsuba_cutoff, int32_t* regs) {
  if (!ctx || u_limbs < 1) return MPDIV_EINVAL;
  if (regs) *regs = mpdiv_default_regs(ctx, u_limbs);
  if (warps) *warps = mpdiv_default_warps(ctx, u_limbs);
  if (mul_columns) *mul_columns = mpdiv_default_tcols(ctx, u_limbs);
  if (karatsuba_cutoff) *karatsuba_cutoff = mpdiv_default_kcut(ctx, u_limbs);
  return MPDIV_OK;
}

// ------------------------------------------------------------------ multiply-pipe microbenchmark
extern "C" int mpdiv_measure_peak(mpdiv_ctx* ctx, int32_t kind, int32_t iters, double* rate, double* ms) {
  if (!ctx) return MPDIV_EINVAL;
  if (kind < 0 || kind > 2 || iters < 0 || !rate || !ms)
    return mpdiv_set_error(ctx, MPDIV_EINVAL, "bad microbenchmark arguments");
  if (iters == 0) iters = kind == 2 ? 8 : 4096;
  cudaSetDevice(ctx->device);
  int per_round = 0, smem = 0, per_sm = 0;
  void* k = mp_kernel_peak(kind, &per_round, &smem, &per_sm);
  if (smem > 0 && mpdiv_open_kernel_smem(k, smem) != cudaSuccess)
    return mpdiv_set_error(ctx, MPDIV_ECUDA, "microbenchmark shared memory");
  const int threads = 256, blocks = per_sm * ctx->num_sms;
  uint32_t* out = nullptr;
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = mpdiv_cuda_check(ctx, cudaMalloc(&out, sizeof(uint32_t) * blocks * threads), "cudaMalloc(microbenchmark)");
  if (rc == MPDIV_OK) rc = mpdiv_cuda_check(ctx, cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking), "cudaStreamCreate");
  if (rc == MPDIV_OK) rc = mpdiv_cuda_check(ctx, cudaEventCreate(&e0), "cudaEventCreate");
  if (rc == MPDIV_OK) rc = mpdiv_cuda_check(ctx, cudaEventCreate(&e1), "cudaEventCreate");
  void* args[] = {&out, &iters};
  if (rc == MPDIV_OK)
    rc = mpdiv_cuda_check(ctx, cudaLaunchKernel(k, dim3(blocks), dim3(threads), args, smem, s), "microbenchmark warm-up");
  if (rc == MPDIV_OK) rc = mpdiv_cuda_check(ctx, cudaEventRecord(e0, s), "cudaEventRecord");
  if (rc == MPDIV_OK)
    rc = mpdiv_cuda_check(ctx, cudaLaunchKernel(k, dim3(blocks), dim3(threads), args, smem, s), "microbenchmark launch");
  if (rc == MPDIV_OK) rc = mpdiv_cuda_check(ctx, cudaEventRecord(e1, s), "cudaEventRecord");
  if (rc == MPDIV_OK) rc = mpdiv_cuda_check(ctx, cudaEventSynchronize(e1), "microbenchmark");
  float t = 0.f;
  if (rc == MPDIV_OK) rc = mpdiv_cuda_check(ctx, cudaEventElapsedTime(&t, e0, e1), "cudaEventElapsedTime");
  if (rc == MPDIV_OK) {
    *ms = t;
    *rate = (double)blocks * threads * iters * per_round / (t * 1e-3);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s) cudaStreamDestroy(s);
  if (out) cudaFree(out);
  return rc;
}

// ------------------------------------------------------------------ multiplication (cost unit)
extern "C" int mpdiv_mul_batch(mpdiv_ctx* ctx, int64_t n_items, const uint32_t* u, const uint32_t* v, int32_t n_limbs,
                               int64_t stride, uint32_t* out, int64_t out_stride, void* stream) {
  MpdivRange nvtx_range("mpdiv.mul_batch");
  if (!ctx) return MPDIV_EINVAL;
  if (n_items < 0) return mpdiv_set_error(ctx, MPDIV_EINVAL, "n_items < 0");
  if (n_items == 0) return MPDIV_OK;
  if (!u || !v || !out) return mpdiv_set_error(ctx, MPDIV_EINVAL, "null pointer argument");
  if (n_limbs < 1 || stride < n_limbs || out_stride < n_limbs) return mpdiv_set_error(ctx, MPDIV_EINVAL, "bad sizes");
  if (n_limbs > 2 * MPDIV_MAX_LIMBS) return mpdiv_set_error(ctx, MPDIV_EUNSUPPORTED, "too many digits");
  cudaSetDevice(ctx->device);
  const int n = n_limbs;
  const int tc = mpdiv_default_tcols(ctx, n);
  int words = 4 * PAD + 3 * n + 8 + ov_words(n);
  // with the transform enabled, n-digit products up to its length use it
  const bool use_ntt = ntt_tables(ctx) != nullptr && 2 * n <= NTT_MAX && 2 * n >= ntt_cutoff(ctx);
  if (use_ntt) words = std::max(words, ((3 * PAD + 3 * n + 4 + ov_words(n) + 3) & ~3) + (4 << ntt_log(2 * n)));
  const int smem = (words * 4 + 15) & ~15;
  if (smem > ctx->max_smem) return mpdiv_set_error(ctx, MPDIV_EUNSUPPORTED, "needs %d bytes of shared memory", smem);
  const int warps = use_ntt ? ntt_kernel_warps(mpdiv_default_warps(ctx, n)) : mpdiv_default_warps(ctx, n);
  void* k = use_ntt ? mp_kernel_ntt_mul(warps) : kernel_for(KK_MUL, warps);
  int rc = prepare_kernel(ctx, k, smem);
  if (rc) return rc;
  UniformArgs a;
  std::memset(&a, 0, sizeof a);
  a.u = u;
  a.v = v;
  a.q = out;
  a.n = n_items;
  a.us = stride;
  a.vs = stride;
  a.qs = out_stride;
  a.un = n;
  a.tcols = tc;
  a.ntt = use_ntt ? ctx->d_ntt : nullptr;
  void* args[] = {&a};
  const int64_t grid = std::min<int64_t>(n_items, 0x7fffffff);
  return mpdiv_cuda_check(ctx, cudaLaunchKernel(k, dim3((unsigned)grid), dim3(32 * warps), args, smem,
                                                (cudaStream_t)stream),
                          "launch of the multiplication kernel");
}

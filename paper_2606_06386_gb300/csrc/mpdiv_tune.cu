// Tuner for the division kernels (Section 5 of arXiv 2606.06386 names
// autotuning of block size, sequentialisation and multiplication
// specialisation as future work): for a size class it times the plain kernel
// at each candidate warps per block (1 and 2 for dividends of at most 1024
// digits, then 4, 8, 16, 32), columns per lane of the strip multiply (3, 5,
// 7) and registers per thread (64, and 128 for 4, 8 and 16 warps), then, in
// the full-product mode, at Karatsuba cutoffs for the Newton
// step's full products (never, 2048, 1024, 512 digits), on synthetic
// divisions, and records the fastest in the context's table, which can be
// saved to and loaded from a text file (MPDIV_TUNE_FILE).
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "mpdiv_internal.h"

namespace {

// splitmix64 finaliser on a counter: synthetic digits for timing only
__global__ void k_fill(uint32_t* x, int64_t n_items, int digits, int64_t stride, uint64_t seed) {
  const int64_t total = n_items * (int64_t)digits;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    uint64_t z = seed + (uint64_t)(t + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    const int64_t item = t / digits;
    const int d = (int)(t - item * digits);
    uint32_t val = (uint32_t)z;
    if (d == digits - 1 && val == 0u) val = 1u;
    x[item * stride + d] = val;
  }
}

}  // namespace

void mpdiv_tune_load(mpdiv_ctx* ctx, const char* path) {
  FILE* f = fopen(path, "r");
  if (!f) return;
  char line[128];
  std::lock_guard<std::mutex> g(ctx->tune_mu);
  while (fgets(line, sizeof line, f)) {
    int cls, w, t, kc, regs = 0;  // the register budget column is optional (0: by occupancy)
    if (sscanf(line, "%d %d %d %d %d", &cls, &w, &t, &kc, &regs) < 4) continue;
    if (cls > 0 && w > 0 && w <= 32 && (t == 3 || t == 5 || t == 7) && kc >= 0 &&
        (regs == 0 || regs == 64 || regs == 128))
      ctx->tuned[cls] = {w, t, kc, regs};
  }
  fclose(f);
}

static void tune_save(mpdiv_ctx* ctx, const char* path) {
  FILE* f = fopen(path, "w");
  if (!f) return;
  std::lock_guard<std::mutex> g(ctx->tune_mu);
  for (auto& kv : ctx->tuned)
    fprintf(f, "%d %d %d %d %d\n", kv.first, kv.second.warps, kv.second.tcols, kv.second.kcut, kv.second.regs);
  fclose(f);
}

extern "C" int mpdiv_autotune(mpdiv_ctx* ctx, int32_t u_limbs, int32_t v_limbs, int32_t n_items) {
  MpdivRange nvtx_range("mpdiv.autotune");
  if (!ctx) return MPDIV_EINVAL;
  if (u_limbs < 1 || v_limbs < 1 || v_limbs > u_limbs || n_items < 1)
    return mpdiv_set_error(ctx, MPDIV_EINVAL, "autotune: bad shape");
  if (u_limbs > MPDIV_MAX_LIMBS) return mpdiv_set_error(ctx, MPDIV_EUNSUPPORTED, "autotune: too many digits");
  cudaSetDevice(ctx->device);
  uint32_t *u = nullptr, *v = nullptr, *q = nullptr, *r = nullptr;
  int32_t* st = nullptr;
  const size_t n = (size_t)n_items;
  int rc = MPDIV_OK;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int best_w = 0, best_t = 5, best_k = 0, best_r = 64;
  float best_ms = 1e30f;
  // launch shapes: warps per block (one and two warps only for dividends of at
  // most 1024 digits) x columns per lane x registers per thread (128 where the
  // block size has that build), schoolbook products
  struct Cand {
    int w, t, regs;
  };
  std::vector<Cand> shapes;
  for (int w = u_limbs <= 1024 ? 1 : 4; w <= 32; w *= 2)
    for (int t = 3; t <= 7; t += 2)
      for (int regs : {64, 128})
        if (regs == 64 || w == 4 || w == 8 || w == 16) shapes.push_back({w, t, regs});
  const int n_shape = (int)shapes.size();
  if ((rc = mpdiv_cuda_check(ctx, cudaMalloc(&u, n * u_limbs * 4), "autotune alloc"))) goto done;
  if ((rc = mpdiv_cuda_check(ctx, cudaMalloc(&v, n * v_limbs * 4), "autotune alloc"))) goto done;
  if ((rc = mpdiv_cuda_check(ctx, cudaMalloc(&q, n * u_limbs * 4), "autotune alloc"))) goto done;
  if ((rc = mpdiv_cuda_check(ctx, cudaMalloc(&r, n * v_limbs * 4), "autotune alloc"))) goto done;
  if ((rc = mpdiv_cuda_check(ctx, cudaMalloc(&st, n * 4), "autotune alloc"))) goto done;
  k_fill<<<256, 256>>>(u, n_items, u_limbs, u_limbs, 0x1234567ull);
  k_fill<<<256, 256>>>(v, n_items, v_limbs, v_limbs, 0x7654321ull);
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  // the shapes, then the Karatsuba cutoff (0 = never, 2048, 1024, 512 digits)
  // at the best shape
  for (int cand = 0; cand < n_shape + 3; cand++) {
    const bool shape = cand < n_shape;
    const int w = shape ? shapes[cand].w : best_w;
    const int tc = shape ? shapes[cand].t : best_t;
    const int regs = shape ? shapes[cand].regs : best_r;
    const int kc = shape ? 0 : (2048 >> (cand - n_shape));
    // Karatsuba splits only the full Newton-step products of the paper's
    // full-product mode; clipped steps leave nothing for it to split
    if (!shape && (best_w == 0 || !(ctx->cfg.flags & MPDIV_FLAG_FULL_PRODUCTS))) break;
    UniformLaunch L{};
    L.u = u;
    L.v = v;
    L.q = q;
    L.r = r;
    L.status = st;
    L.iters = nullptr;
    L.n = n_items;
    L.us = L.qs = u_limbs;
    L.vs = L.rs = v_limbs;
    L.un = u_limbs;
    L.vn = v_limbs;
    L.qn = u_limbs;
    L.rn = v_limbs;
    L.warps = w;
    L.tcols = tc;
    L.kcut = kc;
    L.regs = regs;
    if (mpdiv_launch_uniform(ctx, L, 0) != MPDIV_OK) continue;  // e.g. does not fit
    // the best of three timed pairs of launches: shapes a few percent apart
    // are told apart only above the run-to-run noise of a single pair
    float ms = 1e30f;
    for (int rep = 0; rep < 3; rep++) {
      cudaEventRecord(e0, 0);
      mpdiv_launch_uniform(ctx, L, 0);
      mpdiv_launch_uniform(ctx, L, 0);
      cudaEventRecord(e1, 0);
      if ((rc = mpdiv_cuda_check(ctx, cudaEventSynchronize(e1), "autotune timing"))) goto done;
      float t = 0.f;
      cudaEventElapsedTime(&t, e0, e1);
      ms = std::min(ms, t);
    }
    if (ms < best_ms) {
      best_ms = ms;
      best_w = w;
      best_t = tc;
      best_k = kc;
      best_r = regs;
    }
  }
  if (best_w == 0) {
    rc = mpdiv_set_error(ctx, MPDIV_EUNSUPPORTED, "autotune: no candidate block size ran");
    goto done;
  }
  {
    std::lock_guard<std::mutex> g(ctx->tune_mu);
    ctx->tuned[mpdiv_size_class(u_limbs)] = {best_w, best_t, best_k, best_r};
  }
  if (const char* tf = getenv("MPDIV_TUNE_FILE")) tune_save(ctx, tf);
  rc = best_w;
done:
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(u);
  cudaFree(v);
  cudaFree(q);
  cudaFree(r);
  cudaFree(st);
  return rc;
}

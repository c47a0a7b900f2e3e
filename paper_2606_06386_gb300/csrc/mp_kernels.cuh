// Kernels of the division library: the plain launch (one thread block per
// division, grid over the batch), the persistent launch over a size-sorted
// work queue for mixed precisions, and the shifted-inverse test entry.
#pragma once
#include "mp_args.h"
#include "mp_div.cuh"

namespace mp {

// Plain launch: block b handles items b, b + gridDim.x, ... of a uniform
// batch, or (LIST) of a ragged batch's item list (a.list: one size class of a
// ragged batch, most expensive first); a compile-time choice, since the list's
// indirection measured 1-2 % slower in the strided launch. NTT: full products
// may use the transform, with its scratch after the item's layout. a.pass
// selects the fit pass or the retry pass (UniformArgs).
template <int NW, int MINB, bool NTT = false, bool LIST = false>
__global__ void __launch_bounds__(NW * 32, MINB) k_div_uniform(UniformArgs a) {
  extern __shared__ __align__(16) uint32_t sm[];
  __shared__ int red[RED_WORDS];
  Blk b = make_block<NW>(red);
  b.tcols = a.tcols;
  b.kcut = a.kcut;
  const int flags = a.pass == 1 ? (a.flags | FLAG_FIT_OR_RETRY) : a.flags;
  for (int64_t slot = blockIdx.x; slot < a.n; slot += gridDim.x) {
    const int64_t item = LIST ? (int64_t)a.list[slot] : slot;
    // retry pass: only the items the fit pass left (every thread reads the
    // status before the item's first barrier, so the branch is uniform)
    if (a.pass == 2 && a.status[item] != ST_RETRY) continue;
    ItemIO io;
    if (!LIST) {
      io.u = a.u + item * a.us;
      io.un = a.un;
      io.v = a.v + item * a.vs;
      io.vn = a.vn;
      io.q = a.q + item * a.qs;
      io.qn = a.qn;
      io.r = a.r + item * a.rs;
      io.rn = a.rn;
    } else {
      io.u = a.u + a.u_off[item];
      io.un = a.u_len[item];
      io.v = a.v + a.v_off[item];
      io.vn = a.v_len[item];
      io.q = a.q + a.q_off[item];
      io.qn = a.q_len[item];
      io.r = a.r + a.r_off[item];
      io.rn = a.r_len[item];
    }
    int it = 0;
    unsigned long long work = 0ull;
    Blk bw = b;
    bw.work = a.products ? &work : nullptr;
    const int st = div_item<NTT>(bw, sm, a.smem_words, io, flags, &it, nullptr, 0, 0, a.ntt, a.ntt_cut);
    if (b.tid == 0) {
      a.status[item] = st;
      if (a.iters) a.iters[item] = it;
      if (a.products) a.products[item] = (int64_t)work;
    }
    b.sync();
  }
}

// Persistent launch over a size-sorted queue: each block repeatedly takes the
// next item (largest first) until the queue is empty.
template <int NW, int MINB, bool NTT = false>
__global__ void __launch_bounds__(NW * 32, MINB) k_div_ragged(RaggedArgs a) {
  extern __shared__ __align__(16) uint32_t sm[];
  __shared__ int red[RED_WORDS];
  Blk b = make_block<NW>(red);
  b.tcols = a.tcols > 0 ? a.tcols : 5;
  b.kcut = a.kcut > 0 ? a.kcut : 0;
  while (true) {
    if (b.tid == 0) red[RED_AUX] = atomicAdd(a.head, 1);
    b.sync();
    const int idx = red[RED_AUX];
    b.sync();
    if ((int64_t)idx >= a.n) break;
    const int item = a.order[idx];
    ItemIO io;
    io.u = a.u + a.u_off[item];
    io.un = a.u_len[item];
    io.v = a.v + a.v_off[item];
    io.vn = a.v_len[item];
    io.q = a.q + a.q_off[item];
    io.qn = a.q_len[item];
    io.r = a.r + a.r_off[item];
    io.rn = a.r_len[item];
    int it = 0;
    unsigned long long work = 0ull;
    Blk bw = b;
    bw.work = a.products ? &work : nullptr;
    const int st = div_item<NTT>(bw, sm, a.smem_words, io, a.flags, &it, nullptr, 0, 0, a.ntt, a.ntt_cut);
    if (b.tid == 0) {
      a.status[item] = st;
      if (a.iters) a.iters[item] = it;
      if (a.products) a.products[item] = (int64_t)work;
    }
    b.sync();
  }
}

// Persistent launch that splits itself for smaller items. The block starts as
// one group of all its NW warps over all of its dynamic shared memory and
// takes items largest-first from the queue. When a group draws an item whose
// size class wants at most half of its warps (a.want_class, the tuned block
// size of the plain launch) and whose working set fits in half of its shared
// memory, the group splits into two independent halves, each with its own
// named barrier and scratch: the first half divides the drawn item, the second
// draws the next one. Groups split down to NW/4 warps. Results are those of the
// plain launch: the division code is the same, only the number of cooperating
// warps differs.
constexpr int kMaxGroups = 7;  // binary tree of groups: NW -> NW/2 -> NW/4 warps

template <int NW, int MINB>
__global__ void __launch_bounds__(NW * 32, MINB) k_div_persistent(RaggedArgs a) {
  constexpr int kMinGroupWarps = NW / 4;
  extern __shared__ __align__(16) uint32_t sm[];
  __shared__ int red[kMaxGroups][RED_WORDS];
  int node = 0, w0 = 0, nw = NW;
  uint32_t* base = sm;
  int words = a.smem_words;
  int pending = -1;
  const bool clip = (a.flags & FLAG_FULL_PRODUCTS) == 0;
  while (true) {
    Blk b = make_group(red[node], w0, nw, node);
    int idx;
    if (pending >= 0) {
      idx = pending;
      pending = -1;
    } else {
      if (b.tid == 0) b.red[RED_AUX] = atomicAdd(a.head, 1);
      b.sync();
      idx = b.red[RED_AUX];
      b.sync();
    }
    if ((int64_t)idx >= a.n) break;
    const int item = a.order[idx];
    const int ul = a.u_len[item];
    const int cls = class_of(ul);
    const int tcols = a.tcols > 0 ? a.tcols : a.tcols_class[cls];
    const int half_words = (words / 2) & ~3;
    if (nw >= 2 * kMinGroupWarps && 2 * node + 2 < kMaxGroups && a.want_class[cls] <= nw / 2 &&
        smem_words_for(ul, clip, layout_pad(clip, tcols)) <= half_words) {
      const bool left = b.warp < nw / 2;
      node = 2 * node + (left ? 1 : 2);
      nw /= 2;
      if (!left) {
        w0 += nw;
        base += half_words;
      }
      words = half_words;
      if (left) pending = idx;
      continue;
    }
    ItemIO io;
    io.u = a.u + a.u_off[item];
    io.un = ul;
    io.v = a.v + a.v_off[item];
    io.vn = a.v_len[item];
    io.q = a.q + a.q_off[item];
    io.qn = a.q_len[item];
    io.r = a.r + a.r_off[item];
    io.rn = a.r_len[item];
    int it = 0;
    unsigned long long work = 0ull;
    Blk bw = b;
    bw.work = a.products ? &work : nullptr;
    bw.tcols = tcols;
    bw.kcut = a.kcut >= 0 ? a.kcut : a.kcut_class[cls];
    const int st = div_item(bw, base, words, io, a.flags, &it, nullptr, 0, 0);
    if (b.tid == 0) {
      a.status[item] = st;
      if (a.iters) a.iters[item] = it;
      if (a.products) a.products[item] = (int64_t)work;
    }
    b.sync();
  }
}

// The cost unit of the paper's multiplication count (Section 2.3, Fig. 3): the
// product of two n-digit numbers kept to n digits, one per block (NTT: by the
// transform, with its scratch after OV, 16-byte aligned).
template <int NW, int MINB, bool NTT = false>
__global__ void __launch_bounds__(NW * 32, MINB) k_mul_low(UniformArgs a) {
  extern __shared__ __align__(16) uint32_t sm[];
  __shared__ int red[RED_WORDS];
  Blk b = make_block<NW>(red);
  b.tcols = a.tcols;
  const int n = a.un;
  uint32_t* X = sm + PAD;
  uint32_t* Y = X + n + PAD;
  uint32_t* P = Y + n + PAD;
  uint32_t* OV = P + n + 4;
  uint32_t* S = sm + ((PAD + n + PAD + n + PAD + n + 4 + ov_words(n) + 3) & ~3);
  for (int64_t item = blockIdx.x; item < a.n; item += gridDim.x) {
    for (int i = b.tid; i < PAD; i += b.nt) sm[i] = 0u;
    load_global(b, X, n, [&](int i) { return a.u[item * a.us + i]; });
    load_global(b, Y, n, [&](int i) { return a.v[item * a.vs + i]; });
    if (NTT)
      ntt_mul<true>(b, P, n, X, n, Y, n, S, a.ntt, 0, false);
    else
      mul(b, P, n, X, n, Y, n, OV);
    store_digits(b, a.q + item * a.qs, n, P, n);
    b.sync();
  }
}

// Test entry: one group primitive per item on operands in shared memory
// (x of nx digits, y of ny digits, result digits C of cap digits), the ops of
// mpdiv_debug_primitive.
template <int NW, int MINB>
__global__ void __launch_bounds__(NW * 32, MINB) k_prim(PrimArgs a) {
  extern __shared__ __align__(16) uint32_t sm[];
  __shared__ int red[RED_WORDS];
  Blk b = make_block<NW>(red);
  b.tcols = a.tcols;
  uint32_t* X = sm + PAD;
  uint32_t* Y = X + a.nx + PAD;
  uint32_t* C = Y + a.ny + PAD;
  uint32_t* OV = C + a.cap + 4;
  uint32_t* S = sm + ((PAD + a.nx + PAD + a.ny + PAD + a.cap + 4 + ov_words(a.cap) + 3) & ~3);
  for (int64_t item = blockIdx.x; item < a.n; item += gridDim.x) {
    for (int i = b.tid; i < a.smem_words; i += b.nt) sm[i] = 0u;
    b.sync();
    load_global(b, X, a.nx, [&](int i) { return a.x[item * a.nx + i]; });
    load_global(b, Y, a.ny, [&](int i) { return a.y[item * a.ny + i]; });
    auto xd = [&](int i) -> uint32_t { return i < a.nx ? X[i] : 0u; };
    auto yd = [&](int i) -> uint32_t { return i < a.ny ? Y[i] : 0u; };
    int res = 0;
    switch (a.op) {
      case 0: res = (int)addsub<false>(b, C, a.cap, xd, yd, 0u); break;
      case 1: res = (int)addsub<true>(b, C, a.cap, xd, yd, 0u); break;
      case 2: res = cmp(b, X, a.nx, Y, a.ny); break;
      case 3: res = prec(b, X, a.nx); break;
      case 4:
        copy(b, C, a.cap, xd);
        res = sub_pow(b, C, a.arg, a.cap) ? 1 : 0;
        break;
      case 5:
        copy(b, C, a.cap, xd);
        res = add_pow(b, C, a.arg, a.cap) ? 1 : 0;
        break;
      case 6: res = mul(b, C, a.cap, X, a.nx, Y, a.ny, OV, a.arg); break;
      case 7: {
        int z, t1, t2;
        scan3(b, X, a.nx, &z, &t1, &t2);
        if (b.tid == 0) {
          C[0] = (uint32_t)z;
          C[1] = (uint32_t)t1;
          C[2] = (uint32_t)t2;
        }
        b.sync();
        break;
      }
      case 8: negate(b, C, a.cap, X, a.nx); break;
      case 9: res = ntt_mul<true>(b, C, a.cap, X, a.nx, Y, a.ny, S, a.ntt, a.arg, false); break;
      default: res = -1;
    }
    for (int i = b.tid; i < a.cap; i += b.nt) a.out[item * a.cap + i] = C[i];
    if (b.tid == 0) a.result[item] = res;
    b.sync();
  }
}

// Test entry: shinv_h(v) as the division path computes it.
template <int NW, int MINB, bool NTT = false>
__global__ void __launch_bounds__(NW * 32, MINB) k_shinv(ShinvArgs a) {
  extern __shared__ __align__(16) uint32_t sm[];
  __shared__ int red[RED_WORDS];
  Blk b = make_block<NW>(red);
  b.tcols = a.tcols > 0 ? a.tcols : 5;
  b.kcut = a.kcut > 0 ? a.kcut : 0;
  for (int64_t item = blockIdx.x; item < a.n; item += gridDim.x) {
    ItemIO io;
    io.u = nullptr;
    io.un = 0;
    io.v = a.v + item * a.vs;
    io.vn = a.vn;
    io.q = a.out + item * a.os;  // unused by the debug path except on v == 0
    io.qn = a.on;
    io.r = a.out + item * a.os;
    io.rn = 0;
    int it = 0;
    const int h = max(a.h[item], 1);
    const int st =
        div_item<NTT>(b, sm, a.smem_words, io, a.flags & FLAG_FULL_PRODUCTS, &it, a.out + item * a.os, a.on, h,
                      a.ntt, a.ntt_cut);
    if (b.tid == 0) {
      a.status[item] = st;
      if (a.iters) a.iters[item] = it;
    }
    b.sync();
  }
}

}  // namespace mp

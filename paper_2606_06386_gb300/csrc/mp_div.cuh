// One exact division per thread block: Algorithms 1-3 of arXiv 2606.06386.
//
//   h = prec(u);  w = Shinv(v, h)                 (Algorithm 1)
//   q = shift_{-h}(u * w);  m = v * q             (Algorithm 3)
//   if u < m: q -= 1, m -= v;  r = u - m;  if r >= v: q += 1, r -= v
//
// Shinv handles the special cases of Algorithm 1 (v < B: B^h quo v by a
// parallel short division; 2v > B^h: 1; v = B^k: B^(h-k)), forms the two-digit
// initial approximation w = B^3 quo (v_{k-1} + v_k B), and refines it with
// Refine / Step / PowDiff (Algorithm 2, with the sign kept explicitly).
//
// By default the products are clipped (the refinement Section 5 proposes):
// Step's w x and the quotient's u w skip the digit products below their kept
// columns (less two guard digits), PowDiff's close product skips the digit
// products whose sum moves Step's result by less than one unit, and the
// remainder is taken modulo B^(kl+1). MPDIV_FLAG_FULL_PRODUCTS runs the algorithms with the paper's full
// products instead. The corrections of Algorithm 3 run at most twice each way
// with full products (Theorem 2 allows one) and four times with clipped ones;
// more would set MPDIV_ST_CORRECTION_OVERFLOW.
//
// Shared-memory plan for an item with h dividend digits and kl divisor digits
// (all digit counts; `pad` zero digits between buffers, shared by neighbours:
// pad_for(T) with clipped products, PAD with full ones, whose Karatsuba views
// borrow PAD digits around their splits):
//   V  [kl]            divisor, whole run
//   W  [h-kl+9]        shifted inverse; later the quotient q
//   X  [kl+32]         divisor prefix v' and PowDiff result x      } u overlays
//   R  [h-kl+16]       Step result before its shift                } X..R later
//   P  products: clipped, max(h-kl+17, kl+32) (the clipped products keep
//      only their top columns, stored from the lowest kept column up);
//      full, max(h+41, 2h-kl+9)
//   OV [two words per 96-column strip of P] multiply overflow digits
// The total is largest at kl = 1 or kl = h: about 3 h digits clipped, 4 h
// full; at kl = h/2 it is about 2.5 h clipped.
// With full products and the number-theoretic transform enabled, the shared
// memory left after OV is the transform's scratch: products of up to 2^s_log
// digits with 4 * 2^s_log <= the words left use the transform.
#pragma once
#include "mp_block.cuh"
#include "mp_ntt.cuh"

namespace mp {

enum : int { ST_OK = 0, ST_DIV_BY_ZERO = 1, ST_CORR = 2, ST_QOVF = 3, ST_INTERNAL = 4 };
// Internal status of a launch's fit pass: the item's plan exceeds the
// launch's shared memory, and the retry pass divides it (never returned).
constexpr int ST_RETRY = 5;
enum : int { FLAG_INJECT_LAMBDA = 1, FLAG_FULL_PRODUCTS = 2 };
// Internal flag (above the library's flags): an item whose plan exceeds the
// shared memory gets ST_RETRY instead of ST_INTERNAL.
constexpr int FLAG_FIT_OR_RETRY = 1 << 20;

// Whether the early Refine iterations of a group of several warps run on its
// first warp alone (see shinv), and up to which ell. The one- and two-warp
// kernels, whose strip multiply is a called function, keep every iteration on
// the whole group: there the one-warp copy of the iteration raised register
// spills, and 2^15-bit divisions got slower (0.951 to 1.148 ms per 8192). So
// does the self-splitting persistent kernel (its translation units set this
// to 0), which ran the sweep's divisions 1.4 % slower with it.
#ifndef MP_EARLY_ON_ONE_WARP
#define MP_EARLY_ON_ONE_WARP (!MP_MUL_NOINLINE)
#endif
#ifndef MP_TINY_ELL
#define MP_TINY_ELL 64
#endif

// Guard digits of the clipped products: skipping the digit products below
// position c - QGUARD of a product whose digits below c are shifted away drops
// less than min(digit counts) B^(c-1) < B^c, so the shifted result is at most
// one short.
constexpr int QGUARD = 2;

// Corrections each way with clipped products: q0 = shift_{-h}(u w) can be one
// short from the clipped quotient product, and w can differ from shinv_h(v) by
// -1..+2 (Theorem 2's lambda plus one unit from the clipped Newton steps), so
// q0 lies in [q - 3, q + 2]; four each way is a bound with room.
constexpr int CLIP_CORR = 4;

struct Layout {
  uint32_t *V, *W, *X, *R, *U, *P, *OV;
  int capV, capW, capX, capR, capP, capOV, total;
  uint32_t* S;  // transform scratch (4 * 2^s_log words) or null
  int s_log;
  const uint32_t* ntt;  // transform tables (ntt_tables.h), with S
  int ntt_cut;          // the transform for products of at least this many digits
};

// Product buffer. Clipped: the Newton step keeps at most |R| - 1 digits above
// its dropped ones plus QGUARD guard digits, i.e. at most h-kl+17 digits (its
// result's length is checked against |R| first); the quotient at most
// |W| + QGUARD = h-kl+11; PowDiff's products and the remainder fit in
// |X| = kl+32 digits (checked against |X|). Full: the Newton step's and the
// quotient's full products.
__host__ __device__ __forceinline__ int cap_p(int h, int kl, bool clip) {
  if (clip) {
    const int a = h - kl + 17, c = kl + 32;
    return a > c ? a : c;
  }
  const int a = h + 41, c = 2 * h - kl + 9;
  return a > c ? a : c;
}

__host__ __device__ __forceinline__ int cap_ov(int capP) { return ov_words(capP); }

// Zero digits between the buffers: the strip multiply's reach for the launch's
// strip width with clipped products, PAD with full ones.
__host__ __device__ __forceinline__ int layout_pad(bool clip, int tcols) { return clip ? pad_for(tcols) : PAD; }

// Buffer starts are rounded up to 16 bytes (four digits), so that digits move
// between global and shared memory as 128-bit vectors.
__host__ __device__ __forceinline__ int align4(int words) { return (words + 3) & ~3; }

__host__ __device__ __forceinline__ int layout_words(int h, int kl, bool clip, int pad) {
  const int capP = cap_p(h, kl, clip);
  const int capOV = cap_ov(capP);
  return 5 * pad + kl + (h - kl + 9) + (kl + 32) + (h - kl + 16) + capP + capOV + 5 * 3;
}

// Words of dynamic shared memory that cover every item with at most h
// dividend digits (the plan is largest for a one-digit divisor or one as long
// as the dividend; only divisors of at most h digits get a plan).
__host__ __device__ __forceinline__ int smem_words_for(int h, bool clip, int pad) {
  const int a = layout_words(h, 1, clip, pad), b = layout_words(h, h, clip, pad);
  return a > b ? a : b;
}

__device__ __forceinline__ Layout make_layout(uint32_t* sm, int h, int kl, bool clip, int pad) {
  Layout L;
  L.capV = kl;
  L.capW = h - kl + 9;
  L.capX = kl + 32;
  L.capR = h - kl + 16;
  L.capP = cap_p(h, kl, clip);
  L.capOV = cap_ov(L.capP);
  int off = align4(pad);
  L.V = sm + off;
  off = align4(off + L.capV + pad);
  L.W = sm + off;
  off = align4(off + L.capW + pad);
  L.X = sm + off;
  off = align4(off + L.capX + pad);
  L.R = sm + off;
  off = align4(off + L.capR + pad);
  L.P = sm + off;
  off += L.capP;
  L.OV = sm + off;
  off += L.capOV;
  L.total = off;
  L.U = L.X;  // u (h digits) overlays X, the pad and R once the shifted inverse is known
  L.S = nullptr;
  L.s_log = 0;
  L.ntt = nullptr;
  L.ntt_cut = 0;
  return L;
}

// The transform's scratch in the shared memory after the layout (words in
// all): the longest transform whose four arrays fit; tab and cut as in Layout.
__device__ __forceinline__ void layout_ntt_scratch(Layout& L, uint32_t* sm, int words, const uint32_t* tab, int cut) {
  const int off = (L.total + 3) & ~3;
  int t = NTT_LOG_MAX;
  while (t > 0 && off + (4 << t) > words) t--;
  if (t > 0) {
    L.S = sm + off;
    L.s_log = t;
    L.ntt = tab;
    L.ntt_cut = cut;
  }
}

// An exact product C[0..npos) = (X Y) mod B^npos of full-product mode: in
// kernels built with the transform (NTT) by the transform when nx + ny
// reaches the cutoff and the transform fits the scratch, else by the strip
// multiply (X and Y are then multiply operands). Both give the same digits.
template <bool NTT>
__device__ __forceinline__ bool ntt_fits(const Blk& b, const Layout& L, int nx, int ny) {
  return NTT && L.s_log > 0 && nx > 0 && ny > 0 && nx + ny >= L.ntt_cut && nx + ny <= (1 << L.s_log);
}
template <bool NTT>
__device__ __forceinline__ void mul_exact(const Blk& b, const Layout& L, uint32_t* C, int npos, uint32_t* X, int nx,
                                          uint32_t* Y, int ny) {
  if (ntt_fits<NTT>(b, L, nx, ny)) {
    if (b.work != nullptr && b.tid == 0) *b.work += pair_count(nx, ny, npos);
    ntt_mul<!MP_NAMED_GROUPS>(b, C, npos, X, nx, Y, ny, L.S, L.ntt, 0, false);
  } else {
    mul(b, C, npos, X, nx, Y, ny, L.OV);
  }
}

__device__ __forceinline__ int ceil_log2(int x) {  // x >= 1
  return 32 - __clz(x - 1);
}

struct ItemIO {
  const uint32_t* u;
  int un;
  const uint32_t* v;
  int vn;
  uint32_t* q;
  int qn;
  uint32_t* r;
  int rn;
};

// Refine loop count of Algorithm 1: ceil(max(log2(h-k-1), 0)) + 2, taken as 2
// when h-k-1 <= 1.
__device__ __forceinline__ int refine_iters(int h, int k) {
  const int t = h - k - 1;
  return t <= 1 ? 2 : ceil_log2(t) + 2;
}

// Algorithm 1 for v (in L.V, kl digits, top digit nonzero) and h >= kl.
// Leaves shinv_h(v) in L.W and returns its digit count bound in *lw.
// Returns a status.
template <bool NTT>
__device__ __forceinline__ int shinv(const Blk& b, const Layout& L, int h, int kl, int* lw_out, int* iters_out,
                            bool clip_step) {
  const int k = kl - 1;
  uint32_t* V = L.V;
  uint32_t* W = L.W;
  *iters_out = 0;
  if (kl == 1) {
    // v < B: B^h quo v by short division from the top. The running remainder
    // above digit i is B^(h-1-i) mod v, so each thread starts its chunk with a
    // modular power and then steps down one digit at a time.
    const uint32_t v0 = V[0];
    if (h + 1 > L.capW) return ST_INTERNAL;
    const int chunk = (h + b.nt - 1) / b.nt;
    const int c0 = b.tid * chunk, c1 = min(h, c0 + chunk);
    if (c0 < c1) {
      const uint64_t beta = (1ull << 32) % v0;
      uint64_t rho = 1 % v0, base = beta;
      for (int e = h - c1; e > 0; e >>= 1) {  // rho = beta^(h - c1) mod v0
        if (e & 1) rho = (rho * base) % v0;
        base = (base * base) % v0;
      }
      for (int i = c1 - 1; i >= c0; i--) {
        const uint64_t cur = rho << 32;
        W[i] = (uint32_t)(cur / v0);
        rho = cur % v0;
      }
    }
    if (b.tid == 0) W[h] = (v0 == 1u) ? 1u : 0u;
    b.sync();
    *lw_out = h + 1;
    return ST_OK;
  }
  const bool low_zero = find_first(b, 0, k, [&](int i) { return V[i] != 0u; }) < 0;
  const uint32_t vtop = V[k];
  if (h == kl && (vtop > 0x80000000u || (vtop == 0x80000000u && !low_zero))) {
    // 2v > B^h
    if (b.tid == 0) W[0] = 1u;
    b.sync();
    *lw_out = 1;
    return ST_OK;
  }
  if (vtop == 1u && low_zero) {
    // v = B^k
    if (h - k + 1 > L.capW) return ST_INTERNAL;
    if (b.tid == 0) W[h - k] = 1u;
    b.sync();
    *lw_out = h - k + 1;
    return ST_OK;
  }
  // initial approximation: w = B^3 quo (v_{k-1} + v_k B), then shift_g with g = 2
  {
    const uint64_t V2 = ((uint64_t)vtop << 32) | V[k - 1];
    const unsigned __int128 num = (unsigned __int128)1 << 96;
    const unsigned __int128 w0 = num / V2;  // in (B, B^2]
    if (b.tid == 0) {
      W[2] = (uint32_t)w0;
      W[3] = (uint32_t)(w0 >> 32);
      W[4] = (uint32_t)(w0 >> 64);
    }
    b.sync();
  }
  int lw = 5;
  int ell = 2;
  const int g = 2;
  const int nit = refine_iters(h, k);
  uint32_t* X = L.X;
  uint32_t* P = L.P;
  uint32_t* R = L.R;
  int pw = prec(b, W, lw);
  // The early iterations work on a few dozen digits. In a group of several
  // warps they run on its first warp alone (a one-warp group: warp barriers,
  // no cross-warp reductions) while the other warps skip ahead; the group
  // joins at the first iteration with ell > kTinyEll (or after the last),
  // where the first warp hands over pw, lw and its status. The loop control
  // (ell, m, s, ...) depends on h and k only, so every warp follows it.
  constexpr int kTinyEll = MP_TINY_ELL;
#if MP_EARLY_ON_ONE_WARP
  const Blk b1 = first_warp(b);
#endif
  bool split = MP_EARLY_ON_ONE_WARP && b.nw > 1;
  int st_split = ST_OK;
  auto join = [&]() {
    if (b.warp == 0 && b.lane == 0) {
      b.red[RED_AUX] = pw;
      b.red[RED_AUX + 1] = lw;
      b.red[RED_AUX + 2] = st_split;
    }
    b.sync();
    pw = b.red[RED_AUX];
    lw = b.red[RED_AUX + 1];
    st_split = b.red[RED_AUX + 2];
    split = false;
  };
  for (int it = 0; it < nit; it++) {
    const int m = min(h - k + 1 - ell, ell);
    const int s = max(0, k - 2 * ell + 1 - g);
    const int hh = k + ell + m - s + g;  // Step's h
    const int e = hh - 2 * m;            // digits Step drops from w*x
    if (m < 0 || e < 1) return ST_INTERNAL;
    // v' = shift_{-s}(v), copied so that it can be the product's window
    // operand (zero digits below it); its top digit is v's: prec(v') = kl - s
    const int pv = kl - s;
    if (pv > L.capX) return ST_INTERNAL;
    if (split && ell > kTinyEll) {
      join();
      if (st_split != ST_OK) return st_split;
    }
    // one iteration (PowDiff, Step, the shift) by group gb: the whole group,
    // or in the early iterations its first warp while the others skip it; a
    // failure leaves the block with its status in rs
#if MP_EARLY_ON_ONE_WARP
    const Blk& gb = split ? b1 : b;
#else
    const Blk& gb = b;
#endif
    int rs = ST_OK;
    if (!split || (b.warp == 0 && st_split == ST_OK)) do {
      copy(gb, X, pv, [&](int i) { return V[s + i]; });
      // ---- PowDiff(v', w, hp, ellp): (sign, |B^hp - v' w|)
      const int hp = hh - m;
      const int ellp = ell - g;
      const int Lc = pv + pw - ellp + 1;
      int sign, px;
      if (pw == 0 || Lc >= hp) {
        const int np = pv + pw;
        if (np > L.capP || np > L.capX || hp + 1 > L.capX) { rs = ST_INTERNAL; break; }
        mul_exact<NTT>(gb, L, P, np, X, pv, W, pw);
        const bool ge = find_first(gb, hp, np, [&](int i) { return P[i] != 0u; }) >= 0;
        if (!ge) {
          sign = 1;
          if (pw == 0) {  // v' w = 0: x = B^hp
            for (int i = gb.tid; i <= hp; i += gb.nt) X[i] = (i == hp) ? 1u : 0u;
            gb.sync();
            px = hp + 1;
          } else {
            negate(gb, X, hp, P, np);
            px = hp;
          }
        } else {
          sign = 0;
          copy(gb, X, np, [&](int i) { return P[i]; });
          sub_pow(gb, X, hp, np);
          px = np;
        }
        px = (px > 0) ? prec(gb, X, px) : 0;
      } else {
        if (Lc > L.capP || Lc > L.capX) { rs = ST_INTERNAL; break; }
        if (clip_step) {
          // MultMod clipped with the Newton step: only the digit products at
          // columns plo = e - pw - 1 - QGUARD and up (the columns below are
          // zero). The dropped sum D < B^(plo+2) makes the signed x larger by D,
          // so w x grows by less than B^(e-1) and Step's result by at most one
          // unit, which the later steps absorb
          const int plo = max(0, e - pw - 1 - QGUARD);
          for (int i = gb.tid; i < min(plo, Lc); i += gb.nt) P[i] = 0u;
          mul(gb, P, Lc, X, pv, W, pw, L.OV, plo);
        } else {
          mul_exact<NTT>(gb, L, P, Lc, X, pv, W, pw);  // MultMod: v' w mod B^L
        }
        // one pass gives the sign test, the negation's pivot and |x|'s length
        int z, t1, t2;
        scan3(gb, P, Lc, &z, &t1, &t2);
        if (t1 < 0) {
          sign = 1;
          px = 0;
        } else if (t1 < Lc - 1) {  // top digit P_{L-1} = 0: v' w > B^hp, x = P
          sign = 0;
          copy(gb, X, t1 + 1, [&](int i) { return P[i]; });
          px = t1 + 1;
        } else {  // x = B^L - P: digits above z are the complements of P's
          sign = 1;
          negate_at(gb, X, Lc, P, Lc, z);
          px = max(t2, z) + 1;
        }
      }
      // ---- Step: res = w B^m +/- shift_{2m-hh}(w x), floor semantics
      int lr;
      if (px == 0) {
        lr = pw + m;
        if (lr > L.capR) { rs = ST_INTERNAL; break; }
        copy(gb, R, lr, [&](int i) { return i >= m ? W[i - m] : 0u; });
      } else {
        const int nt = pw + px;
        if (!clip_step && nt > L.capP) { rs = ST_INTERNAL; break; }
        int p0 = 0;  // lowest column of w x; column c of the product is at P[c - p0]
        if (clip_step) {
          // clipped: only the digit products at columns e - QGUARD and up, so
          // shift_{-e} of the product may come out one short (and the floor's
          // sticky digit is read from the computed columns only); the iterate may
          // then differ from Algorithm 1's by one unit, which Refine's later steps
          // and the quotient's corrections absorb
          const int plo = max(0, e - QGUARD);
          p0 = mul_first_column(nt, plo);
          if (nt - p0 > L.capP || ov_words(nt - p0) > L.capOV) { rs = ST_INTERNAL; break; }
          mul(gb, P, nt, W, pw, X, px, L.OV, plo, false, true);
        } else if (ntt_fits<NTT>(gb, L, pw, px)) {
          mul_exact<NTT>(gb, L, P, nt, W, pw, X, px);
        } else {
          // Karatsuba scratch: the product buffer's free tail, and R (free until
          // Step's sum below) for chunk products
          const int sa = (nt + 3) & ~3;
          mul_full(gb, P, W, pw, X, px, L.OV, P + sa, L.capP - sa, R, L.capR);
        }
        lr = max(pw + m, nt - e) + 1;
        if (lr > L.capR) { rs = ST_INTERNAL; break; }
        auto wm = [&](int i) -> uint32_t { return (i >= m && i - m < pw) ? W[i - m] : 0u; };
        const uint32_t* Pc = P - p0;
        auto pe = [&](int i) -> uint32_t { return (i + e < nt) ? Pc[i + e] : 0u; };
        if (sign) {
          addsub<false>(gb, R, lr, wm, pe, 0u);
        } else {
          const uint32_t c = find_first(gb, p0, min(e, nt), [&](int i) { return Pc[i] != 0u; }) >= 0 ? 1u : 0u;
          const uint32_t bout = addsub<true>(gb, R, lr, wm, pe, c);
          if (bout) { rs = ST_INTERNAL; break; }  // a negative iterate never happens (Theorem 2)
        }
      }
      // ---- w <- shift_{-m}(res) for the first two iterations, else shift_{-1}(res)
      const int d = (it < 2) ? m : 1;
      lw = max(lr - d, 0);
      if (lw > L.capW) { rs = ST_INTERNAL; break; }
      pw = copy_prec(gb, W, lw, [&](int i) { return R[i + d]; });
    } while (false);
    if (rs != ST_OK) {
      if (!split) return rs;
      st_split = rs;  // a failed early iteration stops the first warp's work until the join
    }
    if (it >= 2) ell = ell + m - 1;
  }
  if (split) {
    join();
    if (st_split != ST_OK) return st_split;
  }
  // final shift of Refine: h-k-4 digits when h-k < 2, else -2
  const int dd = (h - k < 2) ? 4 - (h - k) : 2;
  const int nl = max(lw - dd, 0);
  copy(b, R, nl, [&](int i) { return W[i + dd]; });
  copy(b, W, lw, [&](int i) { return i < nl ? R[i] : 0u; });  // clear the vacated top digits
  *lw_out = nl;
  *iters_out = nit;
  return ST_OK;
}

// Store digits [0, n) of S to global g[0..cap), zero-padded; S digits at or
// above n are treated as zero and not read. Where g's first 16-byte boundary
// falls on one of S's, the body moves as coalesced 128-bit vectors.
__device__ __forceinline__ void store_digits(const Blk& b, uint32_t* g, int cap, const uint32_t* S, int n) {
  const int head = min(cap, (int)(((16u - ((uint32_t)(uintptr_t)g & 15u)) & 15u) >> 2));
  if (!MP_VECTOR_IO || S == nullptr || (((uint32_t)(uintptr_t)(S + head)) & 15u) != 0u) {
    for (int i = b.tid; i < cap; i += b.nt) g[i] = (i < n) ? S[i] : 0u;
    return;
  }
  const int nv = (cap - head) >> 2;
  uint4* gv = reinterpret_cast<uint4*>(g + head);
  for (int c = b.tid; c < nv; c += b.nt) {
    const int i = head + 4 * c;
    uint4 v;
    if (i + 3 < n) {
      v = *reinterpret_cast<const uint4*>(S + i);
    } else {
      v.x = i < n ? S[i] : 0u;
      v.y = i + 1 < n ? S[i + 1] : 0u;
      v.z = i + 2 < n ? S[i + 2] : 0u;
      v.w = i + 3 < n ? S[i + 3] : 0u;
    }
    gv[c] = v;
  }
  for (int i = b.tid; i < head; i += b.nt) g[i] = (i < n) ? S[i] : 0u;
  for (int i = head + 4 * nv + b.tid; i < cap; i += b.nt) g[i] = (i < n) ? S[i] : 0u;
}

// The whole of Algorithm 3 for one item. Returns a status; q and r are always
// written (zeros on division by zero).
template <bool NTT = false>
__device__ __forceinline__ int div_item(const Blk& b, uint32_t* sm, int smem_words, const ItemIO& io, int flags, int* iters_out,
                        uint32_t* dbg_w, int dbg_cap, int h_override, const uint32_t* ntt_tab = nullptr,
                        int ntt_cut = 0) {
  const uint32_t* gu = io.u;
  const uint32_t* gv = io.v;
  *iters_out = 0;
  const int kl = find_last(b, 0, io.vn, [&](int i) { return gv[i] != 0u; }) + 1;
  int h;
  if (h_override > 0) {
    h = h_override;  // debug entry: shinv_h(v) only
  } else {
    h = find_last(b, 0, io.un, [&](int i) { return gu[i] != 0u; }) + 1;
  }
  if (kl == 0) {
    store_digits(b, io.q, io.qn, nullptr, 0);
    store_digits(b, io.r, io.rn, nullptr, 0);
    return ST_DIV_BY_ZERO;
  }
  if (h_override <= 0) {
    bool ult = h < kl;
    if (h == kl) ult = cmp(b, gu, h, gv, kl) < 0;
    if (ult) {  // u < v: q = 0, r = u
      store_digits(b, io.q, io.qn, nullptr, 0);
      for (int i = b.tid; i < io.rn; i += b.nt) io.r[i] = (i < h) ? gu[i] : 0u;
      return (h > io.rn) ? ST_INTERNAL : ST_OK;
    }
  } else if (h < kl) {
    return ST_INTERNAL;
  }
  const bool clip = (flags & FLAG_FULL_PRODUCTS) == 0;
  Layout L = make_layout(sm, h, kl, clip, layout_pad(clip, b.tcols));
  if (L.total > smem_words) return (flags & FLAG_FIT_OR_RETRY) ? ST_RETRY : ST_INTERNAL;
  if (NTT && ntt_tab != nullptr && !clip) layout_ntt_scratch(L, sm, smem_words, ntt_tab, ntt_cut);
  for (int i = b.tid; i < L.total; i += b.nt) sm[i] = 0u;
  b.sync();
  load_digits(b, L.V, kl, gv);
  int lw = 0, iters = 0;
  int st = shinv<NTT>(b, L, h, kl, &lw, &iters, clip);
  *iters_out = iters;
  if (st != ST_OK) return st;
  uint32_t* W = L.W;
  if (flags & FLAG_INJECT_LAMBDA) {
    if (!add_pow(b, W, 0, L.capW)) return ST_INTERNAL;
    lw = min(lw + 1, L.capW);
  }
  lw = prec(b, W, lw);
  if (dbg_w != nullptr) {
    store_digits(b, dbg_w, dbg_cap, W, lw);
    return lw > dbg_cap ? ST_QOVF : ST_OK;
  }
  // ---- q0 = shift_{-h}(u * w)
  uint32_t* U = L.U;
  uint32_t* P = L.P;
  const bool full = !clip;
  load_digits(b, U, h, gu);
  const int np = h + lw;
  // full: the exact product; clipped (Section 5's clipped products): only the
  // digit products at columns h - QGUARD and up (stored from that column up),
  // so q0 may come out one short
  const int qlo = full ? 0 : max(0, h - QGUARD);
  const int q0c = mul_first_column(np, qlo);
  if (np - q0c > L.capP || ov_words(np - q0c) > L.capOV) return ST_INTERNAL;
  if (NTT && full)
    mul_exact<NTT>(b, L, P, np, U, h, W, lw);
  else
    mul(b, P, np, U, h, W, lw, L.OV, qlo, false, true);
  const uint32_t* Pq = P - q0c;
  int lq = np - h;
  if (lq + 1 > L.capW) return ST_INTERNAL;
  // q lives in W from here (one zero digit above it for a later +1)
  lq = copy_prec(b, W, lq + 1, [&](int i) { return i < np - h ? Pq[h + i] : 0u; });
  uint32_t* V = L.V;
  int lr;
  if (full) {
    // ---- m = v * q
    int nm = kl + lq;
    if (nm > L.capP) return ST_INTERNAL;
    mul_exact<NTT>(b, L, P, nm, V, kl, W, lq);
    nm = prec(b, P, nm);
    // ---- if u < m: q -= 1, m -= v   (Theorem 2: delta = -1)
    for (int t = 0;; t++) {
      if (cmp(b, U, h, P, nm) >= 0) break;
      if (t == 2) return ST_CORR;
      if (!sub_pow(b, W, 0, lq)) return ST_INTERNAL;
      addsub<true>(b, P, nm, [&](int i) { return P[i]; }, [&](int i) { return i < kl ? V[i] : 0u; }, 0u);
      lq = prec(b, W, lq);
      nm = prec(b, P, nm);
    }
    // ---- r = u - m (into P, in place)
    addsub<true>(b, P, h, [&](int i) { return U[i]; }, [&](int i) { return i < nm ? P[i] : 0u; }, 0u);
    lr = prec(b, P, h);
  } else {
    // ---- t = u - v q0 is in [-2v, 4v) (q0 in [q - 3, q + 2]), so it is
    // determined by its value modulo B^(kl+1): only the low product is needed.
    const int K1 = kl + 1;
    if (K1 > L.capP) return ST_INTERNAL;
    mul(b, P, K1, V, kl, W, lq, L.OV);  // v q0 mod B^(kl+1)
    addsub<true>(b, P, K1, [&](int i) { return i < h ? U[i] : 0u; }, [&](int i) { return P[i]; }, 0u);
    // ---- while t < 0 (top digit of the two's complement): q -= 1, t += v
    for (int t = 0;; t++) {
      if (P[K1 - 1] < 0x80000000u) break;
      if (t == CLIP_CORR) return ST_CORR;
      if (!sub_pow(b, W, 0, lq)) return ST_INTERNAL;
      addsub<false>(b, P, K1, [&](int i) { return P[i]; }, [&](int i) { return i < kl ? V[i] : 0u; }, 0u);
    }
    // ---- if r >= v: q += 1, r -= v   (Theorem 2: delta = +1); r < B^(kl+1)
    for (int t = 0;; t++) {
      if (cmp(b, P, K1, V, kl) < 0) break;
      if (t == CLIP_CORR) return ST_CORR;
      if (!add_pow(b, W, 0, lq + 1)) return ST_INTERNAL;
      lq = lq + 1;  // a bound: q may have grown by a digit
      addsub<true>(b, P, K1, [&](int i) { return P[i]; }, [&](int i) { return i < kl ? V[i] : 0u; }, 0u);
    }
    // r < v has at most kl <= rn digits; q's digits above its bound lq are zero
    if (lq > io.qn) lq = prec(b, W, lq);
    store_digits(b, io.q, io.qn, W, lq);
    store_digits(b, io.r, io.rn, P, min(K1, io.rn));
    return lq > io.qn ? ST_QOVF : ST_OK;
  }
  // ---- if r >= v: q += 1, r -= v   (Theorem 2: delta = +1)
  lr = prec(b, P, lr);
  for (int t = 0;; t++) {
    if (cmp(b, P, lr, V, kl) < 0) break;
    if (t == 2) return ST_CORR;
    if (!add_pow(b, W, 0, L.capW)) return ST_INTERNAL;
    lq = min(lq + 1, L.capW);
    addsub<true>(b, P, lr, [&](int i) { return P[i]; }, [&](int i) { return i < kl ? V[i] : 0u; }, 0u);
    lq = prec(b, W, lq);
    lr = prec(b, P, lr);
  }
  store_digits(b, io.q, io.qn, W, lq);
  store_digits(b, io.r, io.rn, P, lr);
  if (lr > io.rn) return ST_INTERNAL;
  return lq > io.qn ? ST_QOVF : ST_OK;
}

}  // namespace mp

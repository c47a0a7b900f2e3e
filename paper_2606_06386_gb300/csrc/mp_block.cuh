// Block-level multi-precision primitives for one division per thread block.
//
// Numbers are little-endian arrays of 32-bit digits in shared memory. Every
// primitive is called by all threads of a group (the whole block, or a slice
// of whole warps with its own named barrier) with group-uniform arguments and
// ends with a barrier of that group, so its result is visible to every thread
// of the group on return.
//
// Linear operations (Section 3.2-3.3 of arXiv 2606.06386: compare, subtract,
// add, shift, subtract a power of B) give each warp a contiguous range of
// digits and walk it 32 digits at a time, one digit per lane, so that shared
// memory is read without bank conflicts. Carries and borrows are resolved with
// the (generate, propagate) formulation of the paper's map-scan-map
// subtraction (Listings 5-6), but the scan over a 32-digit row is one integer
// addition of two ballot masks instead of a shuffle ladder, and the scan over
// warps is the same trick on the per-warp summaries: one barrier per
// operation.
//
// Multiplication (Section 3.4, Fig. 3) is the classical product scheduled as
// column strips: lane L of a warp owns T consecutive output columns and walks
// the rows of the shorter operand, keeping a sliding window of T digits of the
// longer operand in registers and three-word column accumulators updated with
// mad.lo.cc / madc.hi.cc / addc. Warps take 32-lane strips from a shared
// counter, heaviest first; within a strip the lanes' overflow digits are folded
// into their neighbours with a ballot-mask carry resolution, and each strip's
// two overflow digits are then added to the next strip's first two columns.
#pragma once
#include <cstdint>

namespace mp {

constexpr unsigned FULL = 0xffffffffu;
// Output columns per lane of the strip multiply: 3, 5 or 7, chosen per launch
// (odd, so that the lanes' window loads fall in distinct banks). Fewer columns
// waste fewer digit products in the triangular ends of a product; more columns
// reuse each loaded digit more often.
constexpr int T_MIN = 3, T_MAX = 7;
constexpr int PAD = 32 * T_MAX + T_MAX;  // zero digits kept on each side of a multiply operand
constexpr int RED_WORDS = 100;           // block scratch: 3 x 32 per-warp slots + counters

// block scratch layout
constexpr int RED_CNT = 96;     // multiply work counter
constexpr int RED_AUX = 97;     // misc broadcast

// A group of whole warps that cooperates on one division: the whole thread
// block, or a slice of it synchronised by its own named barrier.
struct Blk {
  int tid, lane, warp, nw, nt;
  int bar;   // named barrier id (0: the whole block)
  int* red;  // RED_WORDS ints of shared scratch owned by this group
  unsigned long long* work;  // thread 0's running count of algorithmic digit products (may be null)
  int tcols;                 // columns per lane of the strip multiply (3, 5 or 7)
  int kcut;                  // Karatsuba for full products whose shorter operand has >= kcut digits (0: never)

  __device__ __forceinline__ void sync() const {
    if (nt == 32)
      __syncwarp();  // a one-warp group
    else
      asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(nt) : "memory");
  }
};

// Group of warps [w0, w0 + nw) of the block with barrier id `bar`.
__device__ __forceinline__ Blk make_group(int* red, int w0, int nw, int bar) {
  Blk b;
  b.tid = threadIdx.x - 32 * w0;
  b.lane = threadIdx.x & 31;
  b.warp = (threadIdx.x >> 5) - w0;
  b.nw = nw;
  b.nt = 32 * nw;
  b.bar = bar;
  b.red = red;
  b.work = nullptr;
  b.tcols = 5;
  b.kcut = 0;
  return b;
}

// The first warp of group b as a one-warp group of its own (the same
// scratch, strip width, Karatsuba cutoff and work counter); its barriers are
// warp barriers.
__device__ __forceinline__ Blk first_warp(const Blk& b) {
  Blk g = make_group(b.red, (int)(threadIdx.x >> 5) - b.warp, 1, b.bar);
  g.work = b.work;
  g.tcols = b.tcols;
  g.kcut = b.kcut;
  return g;
}

// The whole block of a kernel built for NW warps: with the group size a
// compile-time constant, one-warp groups skip their cross-warp summaries.
template <int NW>
__device__ __forceinline__ Blk make_block(int* red) { return make_group(red, 0, NW, 0); }

// Whether the kernels of a translation unit divide with groups that are
// slices of a block under named barriers (the self-splitting persistent
// kernel defines it to 1); otherwise every group is a whole block.
#ifndef MP_NAMED_GROUPS
#define MP_NAMED_GROUPS 0
#endif

// Group barrier: the block's own barrier when the group is the whole block
// (WHOLE), so that a kernel whose groups are all whole blocks reserves one
// barrier only; a named barrier otherwise.
template <bool WHOLE>
__device__ __forceinline__ void group_sync(const Blk& b) {
  if (!WHOLE)
    b.sync();
  else if (b.nt > 32)
    __syncthreads();
  else
    __syncwarp();  // a one-warp block
}

// Group-wide maximum (minimum) of a warp-uniform value, one per warp; ends
// with a group barrier.
__device__ __forceinline__ int group_max(const Blk& b, int v) {
  if (b.nw == 1) {
    __syncwarp();
    return v;
  }
  if (b.lane == 0) b.red[b.warp] = v;
  b.sync();
  int r = (b.lane < b.nw) ? b.red[b.lane] : -0x7fffffff - 1;
  for (int o = 1; o < b.nw; o <<= 1) r = max(r, __shfl_xor_sync(FULL, r, o));
  r = __shfl_sync(FULL, r, 0);
  b.sync();
  return r;
}
__device__ __forceinline__ int group_min(const Blk& b, int v) { return -group_max(b, -v); }

// Range of a warp's digits for a linear operation over [0, len): a multiple of 32.
__device__ __forceinline__ void warp_range(const Blk& b, int len, int& lo, int& hi) {
  int cw = (len + b.nw - 1) / b.nw;
  cw = (cw + 31) & ~31;
  lo = b.warp * cw;
  hi = min(lo + cw, len);
}

// ---------------------------------------------------------------- carries
// C[i] = X(i) + Y(i) (+ cin at digit 0) or X(i) - Y(i) (- cin) for i < len.
// Returns the carry (borrow) out of digit len-1. C may alias X or Y only where
// that functor reads index i itself.
template <bool SUB, bool WHOLE = false, class FX, class FY>
__device__ uint32_t addsub(const Blk& b, uint32_t* C, int len, FX X, FY Y, uint32_t cin) {
  int lo, hi;
  warp_range(b, len, lo, hi);
  uint32_t c = (b.warp == 0) ? cin : 0u;
  bool allp = true;
  for (int base = lo; base < hi; base += 32) {
    const int i = base + b.lane;
    const bool valid = i < hi;
    uint32_t d = 0;
    bool g = false, p = true;
    if (valid) {
      const uint32_t x = X(i), y = Y(i);
      if (!SUB) {
        const uint64_t s = (uint64_t)x + y;
        d = (uint32_t)s;
        g = (s >> 32) != 0;
        p = (d == FULL);
      } else {
        d = x - y;
        g = x < y;
        p = (d == 0u);
      }
    }
    const uint32_t gm = __ballot_sync(FULL, g), pm = __ballot_sync(FULL, p);
    const uint64_t xm = (uint64_t)(gm | pm);
    const uint64_t sum = xm + gm + c;
    const uint32_t cinm = (uint32_t)(sum ^ xm ^ gm);  // bit L: carry into lane L
    const uint32_t ci = (cinm >> b.lane) & 1u;
    if (valid) C[i] = SUB ? d - ci : d + ci;
    c = (uint32_t)(sum >> 32);
    allp = allp && (pm == FULL);
  }
  if (b.nw == 1) {  // one warp: its carry out is the result
    __syncwarp();
    return c;
  }
  if (b.lane == 0) b.red[b.warp] = (int)(c | ((allp && b.warp != 0) ? 2u : 0u));
  group_sync<WHOLE>(b);
  const uint32_t sw = (b.lane < b.nw) ? (uint32_t)b.red[b.lane] : 2u;
  const uint32_t Gm = __ballot_sync(FULL, (sw & 1u) != 0);
  const uint32_t Pm = __ballot_sync(FULL, (sw & 3u) == 2u);
  const uint64_t xw = (uint64_t)(Gm | Pm);
  const uint64_t ws = xw + Gm;
  const uint32_t wcm = (uint32_t)(ws ^ xw ^ Gm);
  const uint32_t wcin = (wcm >> b.warp) & 1u;
  const uint32_t cout = (b.nw < 32) ? ((wcm >> b.nw) & 1u) : (uint32_t)(ws >> 32);
  if (wcin) {
    // add (subtract) one at the bottom of this warp's range
    for (int base = lo; base < hi; base += 32) {
      const int i = base + b.lane;
      const bool valid = i < hi;
      const uint32_t d = valid ? C[i] : 0u;
      const bool stop = valid && (SUB ? d != 0u : d != FULL);
      const uint32_t sm = __ballot_sync(FULL, stop);
      if (sm == 0u) {
        if (valid) C[i] = SUB ? FULL : 0u;
      } else {
        const int f = __ffs(sm) - 1;
        if (valid && b.lane < f) C[i] = SUB ? FULL : 0u;
        if (b.lane == f) C[i] = SUB ? d - 1u : d + 1u;
        break;
      }
    }
  }
  group_sync<WHOLE>(b);
  return cout;
}

// ---------------------------------------------------------------- reductions
// Largest i in [lo, hi) with pred(i), or -1.
template <class F>
__device__ inline int find_last(const Blk& b, int lo, int hi, F pred) {
  int best = -1;
  const int len = hi - lo;
  if (len > 0) {
    int wl, wh;
    warp_range(b, len, wl, wh);
    for (int top = wh; top > wl; top -= 32) {
      const int base = top - 32 >= wl ? top - 32 : wl;
      const int i = base + b.lane;
      const bool hit = (i < top) && pred(lo + i);
      const uint32_t m = __ballot_sync(FULL, hit);
      if (m) {
        best = lo + base + 31 - __clz(m);
        break;
      }
      if (base == wl) break;
    }
  }
  return group_max(b, best);
}

// Smallest i in [lo, hi) with pred(i), or -1.
template <class F>
__device__ inline int find_first(const Blk& b, int lo, int hi, F pred) {
  int best = 0x7fffffff;
  const int len = hi - lo;
  if (len > 0) {
    int wl, wh;
    warp_range(b, len, wl, wh);
    for (int base = wl; base < wh; base += 32) {
      const int i = base + b.lane;
      const bool hit = (i < wh) && pred(lo + i);
      const uint32_t m = __ballot_sync(FULL, hit);
      if (m) {
        best = lo + base + __ffs(m) - 1;
        break;
      }
    }
  }
  const int r = group_min(b, best);
  return r == 0x7fffffff ? -1 : r;
}

// number of significant digits of X[0..len)
__device__ __forceinline__ int prec(const Blk& b, const uint32_t* X, int len) {
  return find_last(b, 0, len, [&](int i) { return X[i] != 0u; }) + 1;
}

// -1, 0, 1 for X < Y, X == Y, X > Y (X has nx digits, Y has ny; zero-extended)
template <class PX, class PY>
__device__ inline int cmp(const Blk& b, PX X, int nx, PY Y, int ny) {
  const int n = max(nx, ny);
  auto xd = [&](int i) -> uint32_t { return i < nx ? X[i] : 0u; };
  auto yd = [&](int i) -> uint32_t { return i < ny ? Y[i] : 0u; };
  const int i = find_last(b, 0, n, [&](int j) { return xd(j) != yd(j); });
  if (i < 0) return 0;
  return xd(i) < yd(i) ? -1 : 1;
}

// C[i] = X(i) for i < len (C must not alias what X reads at other indices)
template <class FX>
__device__ inline void copy(const Blk& b, uint32_t* C, int len, FX X) {
  for (int i = b.tid; i < len; i += b.nt) C[i] = X(i);
  b.sync();
}

// C[i] = X(i) for i < len, returning the number of significant digits
// written (one reduction instead of a copy followed by prec). C must not
// alias what X reads at other indices.
template <class FX>
__device__ inline int copy_prec(const Blk& b, uint32_t* C, int len, FX X) {
  int lo, hi;
  warp_range(b, len, lo, hi);
  int best = -1;
  for (int base = lo; base < hi; base += 32) {
    const int i = base + b.lane;
    uint32_t d = 0u;
    if (i < hi) {
      d = X(i);
      C[i] = d;
    }
    const uint32_t m = __ballot_sync(FULL, d != 0u);
    if (m) best = base + 31 - __clz(m);
  }
  return group_max(b, best) + 1;
}

// One pass over P[0..len): the lowest nonzero digit (*z), the highest
// nonzero digit (*t1) and the highest digit that is not all ones (*t2);
// -1 where there is none.
__device__ inline void scan3(const Blk& b, const uint32_t* P, int len, int* z, int* t1, int* t2) {
  int lo, hi;
  warp_range(b, len, lo, hi);
  int bz = 0x7fffffff, b1 = -1, b2 = -1;
  for (int base = lo; base < hi; base += 32) {
    const int i = base + b.lane;
    const uint32_t d = (i < hi) ? P[i] : 0u;
    const uint32_t mn = __ballot_sync(FULL, d != 0u);
    const uint32_t mf = __ballot_sync(FULL, (i < hi) && d != FULL);
    if (mn) {
      if (bz == 0x7fffffff) bz = base + __ffs(mn) - 1;
      b1 = base + 31 - __clz(mn);
    }
    if (mf) b2 = base + 31 - __clz(mf);
  }
  int rz = bz, r1 = b1, r2 = b2;
  if (b.nw == 1) {
    __syncwarp();
  } else {
    if (b.lane == 0) {
      b.red[b.warp] = bz;
      b.red[32 + b.warp] = b1;
      b.red[64 + b.warp] = b2;
    }
    b.sync();
    rz = (b.lane < b.nw) ? b.red[b.lane] : 0x7fffffff;
    r1 = (b.lane < b.nw) ? b.red[32 + b.lane] : -1;
    r2 = (b.lane < b.nw) ? b.red[64 + b.lane] : -1;
    for (int o = 1; o < b.nw; o <<= 1) {
      rz = min(rz, __shfl_xor_sync(FULL, rz, o));
      r1 = max(r1, __shfl_xor_sync(FULL, r1, o));
      r2 = max(r2, __shfl_xor_sync(FULL, r2, o));
    }
    rz = __shfl_sync(FULL, rz, 0);
    r1 = __shfl_sync(FULL, r1, 0);
    r2 = __shfl_sync(FULL, r2, 0);
    b.sync();
  }
  *z = rz == 0x7fffffff ? -1 : rz;
  *t1 = r1;
  *t2 = r2;
}

// X <- X - B^e, digits [e, len); requires X >= B^e. Returns false if no digit
// at or above e was nonzero (X < B^e).
__device__ inline bool sub_pow(const Blk& b, uint32_t* X, int e, int len) {
  const int z = find_first(b, e, len, [&](int i) { return X[i] != 0u; });
  if (z < 0) return false;
  for (int i = e + b.tid; i <= z; i += b.nt) X[i] = (i == z) ? X[i] - 1u : FULL;
  b.sync();
  return true;
}

// X <- X + B^e over digits [e, cap); returns false on carry out of cap.
__device__ inline bool add_pow(const Blk& b, uint32_t* X, int e, int cap) {
  const int z = find_first(b, e, cap, [&](int i) { return X[i] != FULL; });
  if (z < 0) return false;
  for (int i = e + b.tid; i <= z; i += b.nt) X[i] = (i == z) ? X[i] + 1u : 0u;
  b.sync();
  return true;
}

// C <- B^L - P over L digits, P (np digits, zero-extended) nonzero below L,
// z its lowest nonzero digit. C may alias P.
__device__ inline void negate_at(const Blk& b, uint32_t* C, int L, const uint32_t* P, int np, int z) {
  for (int i = b.tid; i < L; i += b.nt) {
    const uint32_t p = i < np ? P[i] : 0u;
    C[i] = (i < z) ? 0u : ((i == z) ? (0u - p) : ~p);
  }
  b.sync();
}

// C <- B^L - P over L digits, P (np digits, zero-extended) nonzero below L.
// C may alias P.
__device__ inline void negate(const Blk& b, uint32_t* C, int L, const uint32_t* P, int np) {
  const int z = find_first(b, 0, min(L, np), [&](int i) { return P[i] != 0u; });
  for (int i = b.tid; i < L; i += b.nt) {
    const uint32_t p = i < np ? P[i] : 0u;
    C[i] = (i < z) ? 0u : ((i == z) ? (0u - p) : ~p);
  }
  b.sync();
}

// ---------------------------------------------------------------- global memory
template <class F>
__device__ inline void load_global(const Blk& b, uint32_t* dst, int len, F src) {
  for (int i = b.tid; i < len; i += b.nt) dst[i] = src(i);
  b.sync();
}

// Whether operands and results move between global and shared memory in
// 16-byte units where their alignment allows (load_digits, store_digits). The
// translation units of the one- and two-warp kernels and of the ragged queue
// kernel define it to 0: there the vector paths' registers raised spills
// (2^15 bits: -2.5 %), and ragged offsets are rarely aligned.
#ifndef MP_VECTOR_IO
#define MP_VECTOR_IO 1
#endif

// Digits g[0..len) of global memory to dst[0..len) in shared memory, then a
// group barrier. Where g's first 16-byte boundary falls on one of dst's, the
// body between the boundaries is staged by asynchronous 16-byte copies
// (cp.async, global to shared without registers; thread t the t-th 4-digit
// chunk, coalesced), waited for before the barrier; the head before it and
// the tail after it go digit by digit. Nothing at or beyond g[len] is read.
__device__ inline void load_digits(const Blk& b, uint32_t* dst, int len, const uint32_t* g) {
  const int head = min(len, (int)(((16u - ((uint32_t)(uintptr_t)g & 15u)) & 15u) >> 2));
  if (!MP_VECTOR_IO || (((uint32_t)(uintptr_t)(dst + head)) & 15u) != 0u) {
    load_global(b, dst, len, [&](int i) { return g[i]; });
    return;
  }
  const int nv = (len - head) >> 2;
  const uint32_t s0 = (uint32_t)__cvta_generic_to_shared(dst + head);
  const size_t g0 = __cvta_generic_to_global(g + head);
  for (int c = b.tid; c < nv; c += b.nt)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s0 + 16u * (uint32_t)c),
                 "l"(g0 + 16u * (size_t)c)
                 : "memory");
  for (int i = b.tid; i < head; i += b.nt) dst[i] = g[i];
  for (int i = head + 4 * nv + b.tid; i < len; i += b.nt) dst[i] = g[i];
  asm volatile("cp.async.wait_all;" ::: "memory");
  b.sync();
}

// ---------------------------------------------------------------- multiply
__device__ __forceinline__ void mac3(uint32_t& c0, uint32_t& c1, uint32_t& c2, uint32_t a, uint32_t bb) {
  asm("mad.lo.cc.u32 %0, %3, %4, %0;\n\t"
      "madc.hi.cc.u32 %1, %3, %4, %1;\n\t"
      "addc.u32 %2, %2, 0;"
      : "+r"(c0), "+r"(c1), "+r"(c2)
      : "r"(a), "r"(bb));
}

// Whether the strip multiply's loop takes two row groups per trip at T = 3. The
// translation units of the one-, two- and four-warp kernels, which run the
// sizes tuned to T = 3, define it to 1; in the larger kernels, which also
// inline the wider strips, the longer code made the 2^18-bit launch 1 % slower.
#ifndef MP_STRIP_T3_UNROLL
#define MP_STRIP_T3_UNROLL 0
#endif

// One warp strip, columns [P0, P0 + 32T): lane owns columns [p0, p0+T) of A*B
// restricted to rows j in [jlo, jhi) of B. Each lane's column sums come to T digits plus two
// overflow digits, which belong to the next lane's first two columns; they are
// added there, the carries between lanes are resolved with the ballot-mask
// addition of addsub, and the strip's own two overflow digits (those of lane
// 31 plus the carry out of the strip) go to OV[2 ws], OV[2 ws + 1]. Writes the
// strip's digits to C (columns < npos).
template <int T>
__device__ __forceinline__ void mul_strip(const Blk& b, uint32_t* C, int npos, const uint32_t* A, int na,
                                          const uint32_t* Bv, int nb, uint32_t* OV, int P0, int ws) {
  constexpr int WSPAN = 32 * T;
  const int jlo = max(0, P0 - na + 1);
  const int jhi = min(nb, P0 + WSPAN);
  const int p0 = P0 + b.lane * T;
  uint32_t a0[T], a1[T], a2[T];
#pragma unroll
  for (int c = 0; c < T; c++) a0[c] = a1[c] = a2[c] = 0u;
  if (jhi > jlo) {
    const uint32_t* Aw = A + p0;  // row j, column c reads Aw[c - j]
    uint32_t ring[T];
#pragma unroll
    for (int c = 1; c < T; c++) ring[c] = Aw[c - jlo];
    ring[0] = 0u;
    const int ngroups = (jhi - jlo + T - 1) / T;
    int j = jlo;
    // one group of T rows: each lane's window moves down one digit per row
#define MP_STRIP_GROUP                                                               \
  {                                                                                  \
    _Pragma("unroll") for (int r = 0; r < T; r++) {                                  \
      ring[(T - r) % T] = Aw[-(j + r)];                                              \
      const uint32_t bj = Bv[j + r];                                                 \
      _Pragma("unroll") for (int c = 0; c < T; c++)                                  \
          mac3(a0[c], a1[c], a2[c], ring[(c - r + T) % T], bj);                      \
    }                                                                                \
    j += T;                                                                          \
  }
    if constexpr (T == 3 && MP_STRIP_T3_UNROLL) {
      // two groups per loop trip at T = 3, whose short groups spend a larger
      // share on the loop itself (2^16 bits: 2.5 % faster); the wider strips
      // keep the compiler's own unrolling (two per trip: 4 % slower at T = 5)
#pragma unroll 2
      for (int gi = 0; gi < ngroups; gi++) MP_STRIP_GROUP
    } else {
      for (int gi = 0; gi < ngroups; gi++) MP_STRIP_GROUP
    }
#undef MP_STRIP_GROUP
  }
  // fold the three-word columns into T+2 digits
  uint32_t o[T + 2];
  uint64_t carry = 0;
#pragma unroll
  for (int c = 0; c < T + 2; c++) {
    uint64_t s = carry;
    if (c < T) s += a0[c];
    if (c >= 1 && c - 1 < T) s += a1[c - 1];
    if (c >= 2 && c - 2 < T) s += a2[c - 2];
    o[c] = (uint32_t)s;
    carry = s >> 32;
  }
  // lane L's overflow digits into lane L+1's first two columns
  uint32_t i0 = __shfl_up_sync(FULL, o[T], 1);
  uint32_t i1 = __shfl_up_sync(FULL, o[T + 1], 1);
  if (b.lane == 0) i0 = i1 = 0u;
  uint64_t t = (uint64_t)o[0] + i0;
  o[0] = (uint32_t)t;
  t = (uint64_t)o[1] + i1 + (t >> 32);
  o[1] = (uint32_t)t;
  uint32_t cy = (uint32_t)(t >> 32);
  bool allf = (o[0] == FULL) && (o[1] == FULL);
#pragma unroll
  for (int c = 2; c < T; c++) {
    t = (uint64_t)o[c] + cy;
    o[c] = (uint32_t)t;
    cy = (uint32_t)(t >> 32);
    allf = allf && (o[c] == FULL);
  }
  // carries between lanes: lane L generates when its sum overflowed and
  // propagates when its T digits are all ones
  const uint32_t gm = __ballot_sync(FULL, cy != 0u), pm = __ballot_sync(FULL, allf);
  const uint64_t xm = (uint64_t)(gm | pm);
  const uint64_t sum = xm + gm;
  uint32_t ci = ((uint32_t)(sum ^ xm ^ gm) >> b.lane) & 1u;
#pragma unroll
  for (int c = 0; c < T; c++) {
    t = (uint64_t)o[c] + ci;
    o[c] = (uint32_t)t;
    ci = (uint32_t)(t >> 32);
  }
#pragma unroll
  for (int c = 0; c < T; c++)
    if (p0 + c < npos) C[p0 + c] = o[c];
  if (b.lane == 31) {
    t = (uint64_t)o[T] + (uint32_t)(sum >> 32);  // the strip's value is below B^(32T+2)
    OV[2 * ws] = (uint32_t)t;
    OV[2 * ws + 1] = o[T + 1] + (uint32_t)(t >> 32);
  }
}

// One warp adds 1 at digit pos of C[0..npos) and propagates the carry (a carry
// out of digit npos-1 is dropped).
__device__ __forceinline__ void ripple_add_one(const Blk& b, uint32_t* C, int pos, int npos) {
  for (int base = pos; base < npos; base += 32) {
    const int i = base + b.lane;
    const bool valid = i < npos;
    const uint32_t d = valid ? C[i] : 0u;
    const uint32_t stop = __ballot_sync(FULL, valid && d != FULL);
    if (stop == 0u) {
      if (valid) C[i] = 0u;
      continue;
    }
    const int f = __ffs(stop) - 1;
    if (b.lane < f) C[i] = 0u;
    if (b.lane == f) C[i] = d + 1u;
    break;
  }
  __syncwarp();
}

// Digit pairs (i, j) with i < na, j < nb and i + j < npos: the digit products
// of a product kept modulo B^npos (all na nb of them for a full product).
__host__ __device__ __forceinline__ unsigned long long pair_count(int na, int nb, int npos) {
  if (na <= 0 || nb <= 0 || npos <= 0) return 0ull;
  const long long c1 = npos - nb + 1 < 0 ? 0 : (npos - nb + 1 < na ? npos - nb + 1 : na);
  unsigned long long s = (unsigned long long)c1 * nb;
  const long long a = c1, e = na < npos ? na : npos;
  if (e > a) s += (unsigned long long)((e - a) * npos - (a + e - 1) * (e - a) / 2);
  return s;
}

// Order of the nws warp strips of a product whose strip ws starts at column
// base + ws * WSPAN, heaviest first: strips on the plateau of the trapezoid of
// row counts (every row of the shorter operand) come first, then strips
// alternately left and right of it by distance.
__device__ __forceinline__ int strip_order(int idx, int nws, int base, int na, int nb, int WSPAN) {
  const int ws0 = 0;
  const int c_lo = min(na, nb) - 1 - base, c_hi = max(na, nb) - 1 - base;
  int lo = c_lo < 0 ? 0 : c_lo / WSPAN;  // first strip whose rows reach the shorter length
  int hi = c_hi < 0 ? 0 : c_hi / WSPAN;  // last strip before the ramp down
  lo = min(lo, nws - 1);
  hi = min(hi, nws - 1);
  if (hi < lo) hi = lo;
  const int np = hi - lo + 1;
  if (idx < np) return lo + idx;
  const int k = idx - np;
  const int nl = lo - ws0, nr = nws - 1 - hi;
  const int m = min(nl, nr);
  if (k < 2 * m) return (k & 1) ? hi + (k >> 1) + 1 : lo - (k >> 1) - 1;
  const int d = m + 1 + (k - 2 * m);
  return (nl > nr) ? lo - d : hi + d;
}

// Whether the strip multiply is a called function rather than inlined at each
// call site. A translation unit of small-block kernels defines it to 1: one
// copy per strip width and group kind then serves every call site, which keeps
// the instruction footprint of kernels that run many small divisions per SM
// small (measured faster for one- and two-warp blocks); inlined is faster for
// larger blocks.
#ifndef MP_MUL_NOINLINE
#define MP_MUL_NOINLINE 0
#endif
#if MP_MUL_NOINLINE
#define MP_MUL_ATTR __noinline__
#else
#define MP_MUL_ATTR __forceinline__
#endif

// The strip multiply for T columns per lane (see mul).
template <int T, bool WHOLE>
__device__ MP_MUL_ATTR void mul_t(const Blk& b, uint32_t* C, int npos, uint32_t* A, int na, uint32_t* Bv, int nb,
                                   uint32_t* OV, int plo, bool compact) {
  constexpr int WSPAN = 32 * T;
  // strips start at column plo exactly: strip ws covers [plo + ws WSPAN, ...)
  const int nws = (npos - plo + WSPAN - 1) / WSPAN;
  // compact: column c lives at C[c - plo]
  uint32_t* Cw = compact ? C - plo : C;
  while (true) {
    int idx = 0;
    if (b.lane == 0) idx = atomicAdd(&b.red[RED_CNT], 1);
    idx = __shfl_sync(FULL, idx, 0);
    if (idx >= nws) break;
    const int ws = strip_order(idx, nws, plo, na, nb, WSPAN);
    mul_strip<T>(b, Cw, npos, A, na, Bv, nb, OV, plo + ws * WSPAN, ws);
  }
  group_sync<WHOLE>(b);
  if (nws == 1) return;  // one strip: its overflow digits lie beyond the product
  // warp 0 folds each strip's two overflow digits into the next strip's first
  // two columns, a lane per strip boundary; a carry out of those two columns
  // (rare: it needs the high overflow digit plus the column to reach B) is
  // recorded in the consumed overflow word and added afterwards, boundary by
  // boundary, with a full carry ripple by the same warp
  if (b.warp == 0) {
    uint32_t any = 0u;
    for (int s0 = 1; s0 < nws; s0 += 32) {
      const int s = s0 + b.lane;
      uint32_t kc = 0u;
      if (s < nws) {
        const int c = plo + s * WSPAN;  // < npos
        uint64_t t = (uint64_t)Cw[c] + OV[2 * (s - 1)];
        Cw[c] = (uint32_t)t;
        if (c + 1 < npos) {
          t = (uint64_t)Cw[c + 1] + OV[2 * (s - 1) + 1] + (t >> 32);
          Cw[c + 1] = (uint32_t)t;
          kc = (c + 2 < npos) ? (uint32_t)(t >> 32) : 0u;
        }
        OV[2 * (s - 1)] = kc;
      }
      any |= __ballot_sync(FULL, kc != 0u);
    }
    if (any != 0u) {
      __syncwarp();
      for (int s = 1; s < nws; s++)
        if (OV[2 * (s - 1)] != 0u) ripple_add_one(b, Cw, plo + s * WSPAN + 2, npos);
    }
  }
  group_sync<WHOLE>(b);
}

// Zero digits a multiply operand needs on each side for T columns per lane.
__host__ __device__ __forceinline__ int pad_for(int tcols) { return 33 * (tcols == 3 ? 3 : (tcols == 7 ? 7 : 5)); }

// Lowest column that mul(b, C, npos, X, nx, Y, ny, OV, plo) writes: plo itself
// (clamped to [0, npos]); the columns from there up are complete digit-product
// sums (zeros when the product is empty or lies wholly below plo).
__device__ __forceinline__ int mul_first_column(int npos, int plo) {
  return plo <= 0 ? 0 : min(plo, npos);
}

// Overflow words a multiply of at most npos columns needs (two per strip).
__host__ __device__ __forceinline__ int ov_words(int npos) { return 2 * ((npos + 32 * T_MIN - 1) / (32 * T_MIN) + 4); }

// C[plo..npos) of X * Y: the digits of (X * Y) mod B^npos at positions plo
// and above, from the digit products at positions plo and above only; the
// carries from the products below plo are dropped (plo = 0: the exact product
// modulo B^npos). With `compact`, column c is stored at C[c - p0], p0 =
// mul_first_column(npos, plo), which is returned; otherwise at C[c].
// X (nx digits) and Y (ny digits) are multiply operands: pad_for(b.tcols) zero
// digits must be addressable below index 0 and above the digit count (the
// high pads are zeroed here); an operand passed with x_rows needs only T_MAX
// zero digits above its count. OV needs ov_words(npos - p0) words. C must not
// alias X or Y.
__device__ inline int mul(const Blk& b, uint32_t* C, int npos, uint32_t* X, int nx, uint32_t* Y, int ny, uint32_t* OV,
                          int plo = 0, bool x_rows = false, bool compact = false) {
  // the longer operand is the window operand unless X must be the row operand
  // (x_rows: X has no zero digits below index 0, only T_MAX above nx)
  uint32_t* A = X;
  uint32_t* Bv = Y;
  int na = nx, nb = ny;
  if (x_rows || nb > na) {
    A = Y;
    Bv = X;
    na = ny;
    nb = nx;
  }
  if (plo < 0) plo = 0;
  if (b.work != nullptr && b.tid == 0)
    *b.work += pair_count(na, nb, npos) - pair_count(na, nb, min(plo, npos));
  const int first = mul_first_column(npos, plo);
  if (nb <= 0 || npos <= plo) {
    for (int i = plo + b.tid; i < npos; i += b.nt) C[compact ? i - first : i] = 0u;
    b.sync();
    return first;
  }
  const int pad = pad_for(b.tcols);
  for (int i = b.tid; i < pad; i += b.nt) {
    A[na + i] = 0u;
    if (i < T_MAX) Bv[nb + i] = 0u;
  }
  if (b.tid == 0) b.red[RED_CNT] = 0;
  b.sync();
  constexpr bool kWhole = !MP_NAMED_GROUPS;
  // in groups of several warps, a product with fewer strips than the group
  // has warps at the launch's strip width runs with the narrowest strips
  // (more strips to share out; its pads, sized for the launch's width, cover
  // the narrower reach). The one- and two-warp kernels keep the launch's width.
  int tc = b.tcols;
#if !MP_MUL_NOINLINE
  if (tc != 3 && npos - plo < 32 * (tc == 7 ? 7 : 5) * b.nw) tc = 3;
#endif
  if (tc == 3)
    mul_t<3, kWhole>(b, C, npos, A, na, Bv, nb, OV, plo, compact);
  else if (tc == 7)
    mul_t<7, kWhole>(b, C, npos, A, na, Bv, nb, OV, plo, compact);
  else
    mul_t<5, kWhole>(b, C, npos, A, na, Bv, nb, OV, plo, compact);
  return first;
}

// ---------------------------------------------------------------- Karatsuba
// Save n digits at p into sv and zero them (and the reverse).
__device__ inline void save_zero(const Blk& b, uint32_t* sv, uint32_t* p, int n) {
  for (int i = b.tid; i < n; i += b.nt) {
    sv[i] = p[i];
    p[i] = 0u;
  }
  b.sync();
}
__device__ inline void restore(const Blk& b, uint32_t* p, const uint32_t* sv, int n) {
  for (int i = b.tid; i < n; i += b.nt) p[i] = sv[i];
  b.sync();
}

// Scratch words kara() needs when its longer operand has n digits.
__host__ __device__ __forceinline__ int kara_words(int n) { return 3 * PAD + 4 * ((n + 1) / 2) + 2 * T_MAX + 16; }

// C[0..na+nb) = A * B by one level of Karatsuba: with m = ceil(na/2) and
// A = A1 B^m + A0, B = B1 B^m + B0, C = Z2 B^2m + (Z1 - Z0 - Z2) B^m + Z0 with
// Z0 = A0 B0, Z2 = A1 B1, Z1 = (A0 + A1)(B0 + B1); the three products are
// strip products with A's parts as row operands and B's as window operands.
// Requires m < nb <= na and m >= PAD. A needs T_MAX zero digits above it, B
// PAD zero digits on both sides; the views B0, B1 and A0 borrow theirs by
// saving, zeroing and restoring the digits around the split.
// S: kara_words(na) scratch words.
__device__ inline void kara(const Blk& b, uint32_t* C, uint32_t* A, int na, uint32_t* B, int nb, uint32_t* OV,
                            uint32_t* S) {
  const int m = (na + 1) / 2, ha = na - m, hb = nb - m;
  uint32_t* SB = S + PAD;                  // B0 + B1: m + 1 digits, PAD zeros each side
  uint32_t* SA = SB + m + 1 + PAD;         // A0 + A1: m + 1 digits, T_MAX zeros above
  uint32_t* TZ = SA + m + 1 + T_MAX;       // Z1: 2m + 2 digits
  uint32_t* SV = TZ + 2 * m + 2 + 4;       // saved digits: PAD + T_MAX
  for (int i = b.tid; i < PAD; i += b.nt) S[i] = 0u;
  const uint32_t ca = addsub<false>(b, SA, m, [&](int i) { return A[i]; },
                                    [&](int i) { return i < ha ? A[m + i] : 0u; }, 0u);
  const uint32_t cb = addsub<false>(b, SB, m, [&](int i) { return B[i]; },
                                    [&](int i) { return i < hb ? B[m + i] : 0u; }, 0u);
  if (b.tid == 0) {
    SA[m] = ca;
    SB[m] = cb;
  }
  b.sync();
  mul(b, TZ, 2 * m + 2, SA, m + 1, SB, m + 1, OV, 0, true);
  // Z0 = A0 B0 into C[0, 2m): A0 and B0 end at the split
  save_zero(b, SV, B + m, PAD);
  save_zero(b, SV + PAD, A + m, T_MAX);
  mul(b, C, 2 * m, A, m, B, m, OV, 0, true);
  restore(b, B + m, SV, PAD);
  restore(b, A + m, SV + PAD, T_MAX);
  // Z2 = A1 B1 into C[2m, na + nb): B1 starts at the split
  save_zero(b, SV, B + m - PAD, PAD);
  mul(b, C + 2 * m, ha + hb, A + m, ha, B + m, hb, OV, 0, true);
  restore(b, B + m - PAD, SV, PAD);
  // Z1 - Z0 - Z2, added at digit m
  addsub<true>(b, TZ, 2 * m + 2, [&](int i) { return TZ[i]; }, [&](int i) { return i < 2 * m ? C[i] : 0u; }, 0u);
  addsub<true>(b, TZ, 2 * m + 2, [&](int i) { return TZ[i]; },
               [&](int i) { return i < ha + hb ? C[2 * m + i] : 0u; }, 0u);
  addsub<false>(b, C + m, na + nb - m, [&](int i) { return C[m + i]; },
                [&](int i) { return i < 2 * m + 2 ? TZ[i] : 0u; }, 0u);
}

// C[0..nx+ny) = X * Y exactly. When the shorter operand has at least b.kcut
// digits (and 2 PAD), one Karatsuba level replaces the strip product: directly
// for operands within 4:3 of each other, else on square chunks of the longer
// operand (each chunk times the shorter, added at its offset). Scratch: S
// (s_words) for Karatsuba, TC (tc_words) for a chunk product; when either is
// too small the strip product is used. X and Y are multiply operands (PAD zero
// digits on both sides). Karatsuba's digit products are counted in b.work.
__device__ inline void mul_full(const Blk& b, uint32_t* C, uint32_t* X, int nx, uint32_t* Y, int ny, uint32_t* OV,
                                uint32_t* S, int s_words, uint32_t* TC, int tc_words) {
  uint32_t* A = X;
  uint32_t* Bv = Y;
  int na = nx, nb = ny;
  if (nb > na) {
    A = Y;
    Bv = X;
    na = ny;
    nb = nx;
  }
  const bool square = 4 * nb >= 3 * na;
  if (b.kcut <= 0 || nb < b.kcut || nb < 2 * PAD || (square && kara_words(na) > s_words) ||
      (!square && (kara_words(nb) + T_MAX > s_words || 2 * nb + 2 > tc_words))) {
    mul(b, C, nx + ny, X, nx, Y, ny, OV);
    return;
  }
  if (square) {
    kara(b, C, A, na, Bv, nb, OV, S);
    return;
  }
  // chunks A_k = A[k0, k0 + lk), lk = min(nb, na - k0), times B, added at digit k0
  uint32_t* SV = S + kara_words(nb);  // A's digits above a chunk: T_MAX
  for (int i = b.tid; i < na + nb; i += b.nt) C[i] = 0u;
  b.sync();
  for (int k0 = 0; k0 < na; k0 += nb) {
    const int lk = min(nb, na - k0);
    uint32_t* Ak = A + k0;
    const bool last = k0 + lk >= na;
    if (!last) save_zero(b, SV, Ak + lk, T_MAX);
    if (lk == nb)
      kara(b, TC, Ak, nb, Bv, nb, OV, S);
    else
      mul(b, TC, lk + nb, Ak, lk, Bv, nb, OV, 0, true);
    if (!last) restore(b, Ak + lk, SV, T_MAX);
    addsub<false>(b, C + k0, na + nb - k0, [&](int i) { return C[k0 + i]; },
                  [&](int i) { return i < lk + nb ? TC[i] : 0u; }, 0u);
  }
}

}  // namespace mp

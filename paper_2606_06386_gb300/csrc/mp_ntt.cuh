// Exact products by number-theoretic transforms: the NTT/FFT multiplication
// that the paper names for larger sizes (Section 3.4) and leaves to future
// work, integrated with the changing precisions of the division (Section 6):
// the transform length is chosen per product, so that it follows the
// precision as the Newton iteration doubles it.
//
// The digits of X and Y are the coefficients of two polynomials in B. Their
// product's coefficients c_k = sum_{i+j=k} x_i y_j are below
// min(nx, ny) (B - 1)^2 < 2^76 for nx + ny <= 8192, so they are recovered
// exactly from their residues modulo three primes p_1 p_2 p_3 > 2^92. Modulo
// each prime, the cyclic convolution of length N = 2^t >= nx + ny (no
// wrap-around) is
//   forward transforms of both operands, decimation in frequency (natural
//     order in, bit-reversed order out), twiddles omega_{2m}^i at the stage of
//     half-length m;
//   the pointwise product (Montgomery multiplication, which leaves a factor
//     2^-32);
//   the inverse transform, decimation in time (bit-reversed in, natural out),
//     with twiddles omega_{2m}^-i, which leaves a factor N; both factors go
//     with one constant multiplication per coefficient.
// Garner's mixed-radix form of the Chinese remainder theorem gives
// c_k = x1 + p1 (x2 + p2 x3) as three words, and one carry pass sums
// c_k B^k into digits. Constant multiplications use Shoup's method (a
// precomputed floor(w 2^32 / p) per constant); residues stay in [0, p).
#pragma once
#include "mp_block.cuh"
#include "ntt_tables.h"

namespace mp {

constexpr int NTT_LOG_MAX = mp_ntt::kLogMax;
constexpr int NTT_MAX = mp_ntt::kMax;

// Smallest t >= 1 with 2^t >= n.
__host__ __device__ __forceinline__ int ntt_log(int n) {
  int t = 1;
  while ((1 << t) < n) t++;
  return t;
}

__device__ __forceinline__ uint32_t mod_red(uint32_t x, uint32_t p) {  // x < 2^32 < 3p
  if (x >= p) x -= p;
  if (x >= p) x -= p;
  return x;
}
__device__ __forceinline__ uint32_t mod_add(uint32_t a, uint32_t c, uint32_t p) {
  const uint32_t s = a + c;
  return s >= p ? s - p : s;
}
__device__ __forceinline__ uint32_t mod_sub(uint32_t a, uint32_t c, uint32_t p) {
  const uint32_t d = a + p - c;
  return d >= p ? d - p : d;
}
// x w mod p for a constant w < p with companion ws = floor(w 2^32 / p): the
// quotient estimate is at most one short, so x w - q p lies in [0, 2p).
__device__ __forceinline__ uint32_t mod_shoup(uint32_t x, uint32_t w, uint32_t ws, uint32_t p) {
  const uint32_t q = __umulhi(x, ws);
  const uint32_t r = x * w - q * p;
  return r >= p ? r - p : r;
}
// x y 2^-32 mod p (Montgomery reduction, pinv = -p^-1 mod 2^32), x, y < p.
__device__ __forceinline__ uint32_t mod_mont(uint32_t x, uint32_t y, uint32_t p, uint32_t pinv) {
  const uint32_t lo = x * y, hi = __umulhi(x, y);
  const uint32_t m = lo * pinv;
  const uint32_t u = hi + __umulhi(m, p) + (lo != 0u ? 1u : 0u);
  return u >= p ? u - p : u;
}

// Two stages of the forward transform on four residues a0..a3 (a radix-4
// butterfly): the stage of half-length m = 2h on (a0, a2) with w1 =
// omega_{2m}^i and on (a1, a3) with w2 = omega_{2m}^(i+h), then the stage of
// half-length h on (a0, a1) and (a2, a3) with w3 = omega_m^i. Each uint2 is a
// constant and its Shoup companion.
__device__ __forceinline__ void dif4v(uint32_t& a0, uint32_t& a1, uint32_t& a2, uint32_t& a3, uint32_t p, uint2 w1,
                                      uint2 w2, uint2 w3) {
  const uint32_t b0 = mod_add(a0, a2, p), b2 = mod_shoup(a0 + p - a2, w1.x, w1.y, p);
  const uint32_t b1 = mod_add(a1, a3, p), b3 = mod_shoup(a1 + p - a3, w2.x, w2.y, p);
  a0 = mod_add(b0, b1, p);
  a1 = mod_shoup(b0 + p - b1, w3.x, w3.y, p);
  a2 = mod_add(b2, b3, p);
  a3 = mod_shoup(b2 + p - b3, w3.x, w3.y, p);
}

// Two stages of the inverse transform on a0..a3: the stage of half-length h
// on (a0, a1) and (a2, a3) with u1 = omega_{2h}^-i, then the stage of
// half-length 2h on (a0, a2) with u2 = omega_{4h}^-i and on (a1, a3) with
// u3 = omega_{4h}^-(i+h).
__device__ __forceinline__ void dit4v(uint32_t& a0, uint32_t& a1, uint32_t& a2, uint32_t& a3, uint32_t p, uint2 u1,
                                      uint2 u2, uint2 u3) {
  uint32_t t = mod_shoup(a1, u1.x, u1.y, p);
  const uint32_t b0 = mod_add(a0, t, p), b1 = mod_sub(a0, t, p);
  t = mod_shoup(a3, u1.x, u1.y, p);
  const uint32_t b2 = mod_add(a2, t, p), b3 = mod_sub(a2, t, p);
  t = mod_shoup(b2, u2.x, u2.y, p);
  a0 = mod_add(b0, t, p);
  a2 = mod_sub(b0, t, p);
  t = mod_shoup(b3, u3.x, u3.y, p);
  a1 = mod_add(b1, t, p);
  a3 = mod_sub(b1, t, p);
}

// dif4v / dit4v on z[0], z[h], z[2h], z[3h] in shared memory.
__device__ __forceinline__ void dif4(uint32_t* z, int h, uint32_t p, uint2 w1, uint2 w2, uint2 w3) {
  uint32_t a0 = z[0], a1 = z[h], a2 = z[2 * h], a3 = z[3 * h];
  dif4v(a0, a1, a2, a3, p, w1, w2, w3);
  z[0] = a0;
  z[h] = a1;
  z[2 * h] = a2;
  z[3 * h] = a3;
}
__device__ __forceinline__ void dit4(uint32_t* z, int h, uint32_t p, uint2 u1, uint2 u2, uint2 u3) {
  uint32_t a0 = z[0], a1 = z[h], a2 = z[2 * h], a3 = z[3 * h];
  dit4v(a0, a1, a2, a3, p, u1, u2, u3);
  z[0] = a0;
  z[h] = a1;
  z[2 * h] = a2;
  z[3 * h] = a3;
}

// One radix-4 forward pass over stages lm and lm - 1 (lm >= 1) of Z0 and Z1,
// or one inverse pass over stages lm and lm + 1 of Z, each thread a group of
// four residues at stride h.
__device__ __forceinline__ void dif_pass2(const Blk& b, uint32_t* Z0, uint32_t* Z1, int logn, int lm, uint32_t p,
                                          const uint2* fw) {
  const int m = 1 << lm, h = m >> 1, quarter = (1 << logn) >> 2;
#pragma unroll 2
  for (int g = b.tid; g < quarter; g += b.nt) {
    const int i = g & (h - 1);
    const int base = ((g >> (lm - 1)) << (lm + 1)) + i;
    const uint2 w1 = __ldg(fw + m + i), w2 = __ldg(fw + m + h + i), w3 = __ldg(fw + h + i);
    dif4(Z0 + base, h, p, w1, w2, w3);
    dif4(Z1 + base, h, p, w1, w2, w3);
  }
}
__device__ __forceinline__ void dit_pass(const Blk& b, uint32_t* Z, int logn, int lm, uint32_t p, const uint2* iw) {
  const int h = 1 << lm, m = 2 * h, quarter = (1 << logn) >> 2;
#pragma unroll 2
  for (int g = b.tid; g < quarter; g += b.nt) {
    const int i = g & (h - 1);
    const int base = ((g >> lm) << (lm + 2)) + i;
    dit4(Z + base, h, p, __ldg(iw + h + i), __ldg(iw + m + i), __ldg(iw + m + h + i));
  }
}

// Z = N 2^-32 (X * Y) modulo prime j, the cyclic convolution of length
// N = 2^logn (logn >= 3, nx, ny <= N) through the transforms: the forward
// transforms of X and Y (into Z and T) run from the longest stage down and
// read the operands' digits, reduced, in their first pass; the last forward
// pass, the pointwise Montgomery product and the first inverse pass are one
// pass over contiguous groups (4 residues when logn is even, 2 when odd), read
// and written as vectors; the remaining inverse passes run upward. One barrier
// per pass.
template <bool WHOLE>
__device__ __forceinline__ void ntt_conv_prime(const Blk& b, uint32_t* Z, uint32_t* T, const uint32_t* X, int nx,
                                               const uint32_t* Y, int ny, int logn, const uint32_t* tab, int j) {
  const uint32_t p = __ldg(tab + mp_ntt::kP + j), pinv = __ldg(tab + mp_ntt::kPinv + j);
  const uint2* fw = reinterpret_cast<const uint2*>(tab + j * mp_ntt::kPerPrime + mp_ntt::kFw);
  const uint2* iw = reinterpret_cast<const uint2*>(tab + j * mp_ntt::kPerPrime + mp_ntt::kIw);
  const int N = 1 << logn, quarter = N >> 2;
  {  // stages logn - 1 and logn - 2 from the operands (one block of N: base = i = g)
    const int m = N >> 1, h = quarter;
#pragma unroll 2
    for (int g = b.tid; g < quarter; g += b.nt) {
      const uint2 w1 = __ldg(fw + m + g), w2 = __ldg(fw + m + h + g), w3 = __ldg(fw + h + g);
      uint32_t x0 = g < nx ? mod_red(X[g], p) : 0u, x1 = g + h < nx ? mod_red(X[g + h], p) : 0u;
      uint32_t x2 = g + 2 * h < nx ? mod_red(X[g + 2 * h], p) : 0u;
      uint32_t x3 = g + 3 * h < nx ? mod_red(X[g + 3 * h], p) : 0u;
      dif4v(x0, x1, x2, x3, p, w1, w2, w3);
      Z[g] = x0;
      Z[g + h] = x1;
      Z[g + 2 * h] = x2;
      Z[g + 3 * h] = x3;
      uint32_t y0 = g < ny ? mod_red(Y[g], p) : 0u, y1 = g + h < ny ? mod_red(Y[g + h], p) : 0u;
      uint32_t y2 = g + 2 * h < ny ? mod_red(Y[g + 2 * h], p) : 0u;
      uint32_t y3 = g + 3 * h < ny ? mod_red(Y[g + 3 * h], p) : 0u;
      dif4v(y0, y1, y2, y3, p, w1, w2, w3);
      T[g] = y0;
      T[g + h] = y1;
      T[g + 2 * h] = y2;
      T[g + 3 * h] = y3;
    }
    group_sync<WHOLE>(b);
  }
  int lm = logn - 3;
  for (; lm >= 2; lm -= 2) {
    dif_pass2(b, Z, T, logn, lm, p, fw);
    group_sync<WHOLE>(b);
  }
  if (lm == 1) {  // stages 1 and 0 forward, pointwise, stages 0 and 1 inverse: 4 contiguous residues
    const uint2 w1 = __ldg(fw + 2), w2 = __ldg(fw + 3), w3 = __ldg(fw + 1);
    const uint2 u1 = __ldg(iw + 1), u2 = __ldg(iw + 2), u3 = __ldg(iw + 3);
    uint4* Z4 = reinterpret_cast<uint4*>(Z);
    const uint4* T4 = reinterpret_cast<const uint4*>(T);
    for (int g = b.tid; g < quarter; g += b.nt) {
      uint4 z = Z4[g], t = T4[g];
      dif4v(z.x, z.y, z.z, z.w, p, w1, w2, w3);
      dif4v(t.x, t.y, t.z, t.w, p, w1, w2, w3);
      z.x = mod_mont(z.x, t.x, p, pinv);
      z.y = mod_mont(z.y, t.y, p, pinv);
      z.z = mod_mont(z.z, t.z, p, pinv);
      z.w = mod_mont(z.w, t.w, p, pinv);
      dit4v(z.x, z.y, z.z, z.w, p, u1, u2, u3);
      Z4[g] = z;
    }
  } else {  // stage 0 forward, pointwise, stage 0 inverse: pairs (twiddle 1)
    uint2* Z2 = reinterpret_cast<uint2*>(Z);
    const uint2* T2 = reinterpret_cast<const uint2*>(T);
    for (int g = b.tid; g < (N >> 1); g += b.nt) {
      const uint2 z = Z2[g], t = T2[g];
      const uint32_t y0 = mod_mont(mod_add(z.x, z.y, p), mod_add(t.x, t.y, p), p, pinv);
      const uint32_t y1 = mod_mont(mod_sub(z.x, z.y, p), mod_sub(t.x, t.y, p), p, pinv);
      Z2[g] = make_uint2(mod_add(y0, y1, p), mod_sub(y0, y1, p));
    }
  }
  group_sync<WHOLE>(b);
  for (lm = (logn & 1) ? 1 : 2; lm < logn; lm += 2) {
    dit_pass(b, Z, logn, lm, p, iw);
    group_sync<WHOLE>(b);
  }
}

// The same for N = 2 or 4 (logn 1 or 2): a load pass, then the stages one by
// one on the residues in shared memory.
template <bool WHOLE>
__device__ __forceinline__ void ntt_conv_prime_small(const Blk& b, uint32_t* Z, uint32_t* T, const uint32_t* X,
                                                     int nx, const uint32_t* Y, int ny, int logn,
                                                     const uint32_t* tab, int j) {
  const uint32_t p = __ldg(tab + mp_ntt::kP + j), pinv = __ldg(tab + mp_ntt::kPinv + j);
  const uint2* fw = reinterpret_cast<const uint2*>(tab + j * mp_ntt::kPerPrime + mp_ntt::kFw);
  const uint2* iw = reinterpret_cast<const uint2*>(tab + j * mp_ntt::kPerPrime + mp_ntt::kIw);
  const int N = 1 << logn;
  if (b.tid == 0) {  // at most 4 residues: one thread
    uint32_t z[4], t[4];
    for (int i = 0; i < N; i++) {
      z[i] = i < nx ? mod_red(X[i], p) : 0u;
      t[i] = i < ny ? mod_red(Y[i], p) : 0u;
    }
    if (logn == 2) {
      dif4v(z[0], z[1], z[2], z[3], p, __ldg(fw + 2), __ldg(fw + 3), __ldg(fw + 1));
      dif4v(t[0], t[1], t[2], t[3], p, __ldg(fw + 2), __ldg(fw + 3), __ldg(fw + 1));
      for (int i = 0; i < 4; i++) z[i] = mod_mont(z[i], t[i], p, pinv);
      dit4v(z[0], z[1], z[2], z[3], p, __ldg(iw + 1), __ldg(iw + 2), __ldg(iw + 3));
    } else {
      const uint32_t y0 = mod_mont(mod_add(z[0], z[1], p), mod_add(t[0], t[1], p), p, pinv);
      const uint32_t y1 = mod_mont(mod_sub(z[0], z[1], p), mod_sub(t[0], t[1], p), p, pinv);
      z[0] = mod_add(y0, y1, p);
      z[1] = mod_sub(y0, y1, p);
    }
    for (int i = 0; i < N; i++) Z[i] = z[i];
  }
  group_sync<WHOLE>(b);
}

// The product below is a called function (one copy per group kind serves
// every call site); it takes the group's scalars rather than a reference to
// the caller's group, which would otherwise have to live in local memory.
// WHOLE: the group is the whole block (its barriers are the block's own).
template <bool WHOLE>
static __device__ __noinline__ int ntt_mul_group(int tid, int nw, int bar, int* red, uint32_t* C, int npos,
                                                 const uint32_t* X, int nx, const uint32_t* Y, int ny, uint32_t* S,
                                                 const uint32_t* tab, int plo, bool compact) {
  Blk b;
  b.tid = tid;
  b.lane = tid & 31;
  b.warp = tid >> 5;
  b.nw = nw;
  b.nt = 32 * nw;
  b.bar = bar;
  b.red = red;
  b.work = nullptr;
  b.tcols = 5;
  b.kcut = 0;
  const int first = mul_first_column(npos, plo);
  const int n = nx + ny;
  const int len = min(npos, n);  // digits at n and above are zero
  if (nx <= 0 || ny <= 0 || len <= first) {
    for (int c = first + b.tid; c < npos; c += b.nt) C[compact ? c - first : c] = 0u;
    group_sync<WHOLE>(b);
    return first;
  }
  const int logn = ntt_log(n), N = 1 << logn;
  uint32_t* T = S + 3 * N;
  for (int j = 0; j < 3; j++) {
    if (logn >= 3)
      ntt_conv_prime<WHOLE>(b, S + j * N, T, X, nx, Y, ny, logn, tab, j);
    else
      ntt_conv_prime_small<WHOLE>(b, S + j * N, T, X, nx, Y, ny, logn, tab, j);
  }
  // Garner: c_k = x1 + p1 x2 + p1 p2 x3 with x_j < p_j, written as three words
  {
    const uint32_t p1 = __ldg(tab + mp_ntt::kP), p2 = __ldg(tab + mp_ntt::kP + 1), p3 = __ldg(tab + mp_ntt::kP + 2);
    const uint32_t* sc = tab + mp_ntt::kScale;
    const int s1 = 2 * logn, s2 = 2 * ((NTT_LOG_MAX + 1) + logn), s3 = 2 * (2 * (NTT_LOG_MAX + 1) + logn);
    const uint32_t c1 = __ldg(sc + s1), c1s = __ldg(sc + s1 + 1);
    const uint32_t c2 = __ldg(sc + s2), c2s = __ldg(sc + s2 + 1);
    const uint32_t c3 = __ldg(sc + s3), c3s = __ldg(sc + s3 + 1);
    const uint32_t i12 = __ldg(tab + mp_ntt::kInv12), i12s = __ldg(tab + mp_ntt::kInv12 + 1);
    const uint32_t p1m3 = __ldg(tab + mp_ntt::kP1m3), p1m3s = __ldg(tab + mp_ntt::kP1m3 + 1);
    const uint32_t i123 = __ldg(tab + mp_ntt::kInv123), i123s = __ldg(tab + mp_ntt::kInv123 + 1);
    const uint64_t p12 = (uint64_t)__ldg(tab + mp_ntt::kP12) | ((uint64_t)__ldg(tab + mp_ntt::kP12 + 1) << 32);
    uint32_t *Z1 = S, *Z2 = S + N, *Z3 = S + 2 * N;
    for (int k = b.tid; k < len; k += b.nt) {
      const uint32_t x1 = mod_shoup(Z1[k], c1, c1s, p1);
      const uint32_t r2 = mod_shoup(Z2[k], c2, c2s, p2);
      const uint32_t r3 = mod_shoup(Z3[k], c3, c3s, p3);
      const uint32_t x2 = mod_shoup(mod_sub(r2, x1 >= p2 ? x1 - p2 : x1, p2), i12, i12s, p2);
      const uint32_t y3 = mod_add(x1 >= p3 ? x1 - p3 : x1, mod_shoup(x2, p1m3, p1m3s, p3), p3);  // (x1 + p1 x2) mod p3
      const uint32_t x3 = mod_shoup(mod_sub(r3, y3, p3), i123, i123s, p3);
      const uint64_t y = (uint64_t)x1 + (uint64_t)p1 * x2;  // < p1 p2 < 2^62
      const uint64_t lo = (uint64_t)(uint32_t)p12 * x3 + (uint32_t)y;
      const uint64_t hi = (uint64_t)(uint32_t)(p12 >> 32) * x3 + (y >> 32) + (lo >> 32);
      Z1[k] = (uint32_t)lo;
      Z2[k] = (uint32_t)hi;
      Z3[k] = (uint32_t)(hi >> 32);
    }
  }
  group_sync<WHOLE>(b);
  // digit k of sum c_k B^k before carries: c_k's word 0, c_{k-1}'s word 1 and
  // c_{k-2}'s word 2; the sum's high word (at most 2) is carried to k + 1
  {
    uint32_t *Z1 = S, *Z2 = S + N, *Z3 = S + 2 * N;
    for (int k = b.tid; k < len; k += b.nt) {
      const uint64_t s = (uint64_t)Z1[k] + (k >= 1 ? Z2[k - 1] : 0u) + (k >= 2 ? Z3[k - 2] : 0u);
      Z1[k] = (uint32_t)s;
      T[k] = (uint32_t)(s >> 32);
    }
  }
  group_sync<WHOLE>(b);
  addsub<false, WHOLE>(b, S, len, [&](int i) { return S[i]; }, [&](int i) { return i > 0 ? T[i - 1] : 0u; }, 0u);
  for (int c = first + b.tid; c < npos; c += b.nt) C[compact ? c - first : c] = c < len ? S[c] : 0u;
  group_sync<WHOLE>(b);
  return first;
}

// Digits [p0, npos) of X * Y, exact (p0 = mul_first_column(npos, plo); with
// `compact` digit c is stored at C[c - p0], else at C[c]); returns p0.
// Requires nx + ny <= NTT_MAX. X and Y are read only (no pads needed); S is
// scratch of 4 * 2^ntt_log(nx + ny) words; tab is the table block of
// ntt_tables.h in global memory. C must not overlap S.
template <bool WHOLE>
__device__ __forceinline__ int ntt_mul(const Blk& b, uint32_t* C, int npos, const uint32_t* X, int nx,
                                       const uint32_t* Y, int ny, uint32_t* S, const uint32_t* tab, int plo,
                                       bool compact) {
  return ntt_mul_group<WHOLE>(b.tid, b.nw, b.bar, b.red, C, npos, X, nx, Y, ny, S, tab, plo, compact);
}

}  // namespace mp

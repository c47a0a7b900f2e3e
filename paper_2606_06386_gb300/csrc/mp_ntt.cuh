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

// Two stages of the forward transform on the four residues z[0], z[h], z[2h],
// z[3h] (a radix-4 pass): the stage of half-length m = 2h with twiddles w1 =
// omega_{2m}^i and w2 = omega_{2m}^(i+h), then the stage of half-length h with
// w3 = omega_m^i; (w, ws) pairs are a constant and its Shoup companion.
__device__ __forceinline__ void dif4(uint32_t* z, int h, uint32_t p, uint32_t w1, uint32_t w1s, uint32_t w2,
                                     uint32_t w2s, uint32_t w3, uint32_t w3s) {
  const uint32_t a0 = z[0], a1 = z[h], a2 = z[2 * h], a3 = z[3 * h];
  const uint32_t b0 = mod_add(a0, a2, p), b2 = mod_shoup(a0 + p - a2, w1, w1s, p);
  const uint32_t b1 = mod_add(a1, a3, p), b3 = mod_shoup(a1 + p - a3, w2, w2s, p);
  z[0] = mod_add(b0, b1, p);
  z[h] = mod_shoup(b0 + p - b1, w3, w3s, p);
  z[2 * h] = mod_add(b2, b3, p);
  z[3 * h] = mod_shoup(b2 + p - b3, w3, w3s, p);
}

// Two stages of the inverse transform on z[0], z[h], z[2h], z[3h]: the stage
// of half-length h with u1 = omega_{2h}^-i on both pairs, then the stage of
// half-length 2h with u2 = omega_{4h}^-i and u3 = omega_{4h}^-(i+h).
__device__ __forceinline__ void dit4(uint32_t* z, int h, uint32_t p, uint32_t u1, uint32_t u1s, uint32_t u2,
                                     uint32_t u2s, uint32_t u3, uint32_t u3s) {
  const uint32_t a0 = z[0], a1 = z[h], a2 = z[2 * h], a3 = z[3 * h];
  uint32_t t = mod_shoup(a1, u1, u1s, p);
  const uint32_t b0 = mod_add(a0, t, p), b1 = mod_sub(a0, t, p);
  t = mod_shoup(a3, u1, u1s, p);
  const uint32_t b2 = mod_add(a2, t, p), b3 = mod_sub(a2, t, p);
  t = mod_shoup(b2, u2, u2s, p);
  z[0] = mod_add(b0, t, p);
  z[2 * h] = mod_sub(b0, t, p);
  t = mod_shoup(b3, u3, u3s, p);
  z[h] = mod_add(b1, t, p);
  z[3 * h] = mod_sub(b1, t, p);
}

// The stage of half-length 1 (twiddle 1) on the pairs (z[2g], z[2g+1]),
// read and written as 8-byte words (Z 8-byte aligned).
__device__ __forceinline__ void ntt_pairs(const Blk& b, uint32_t* Z, int half, uint32_t p) {
  uint2* Z2 = reinterpret_cast<uint2*>(Z);
  for (int g = b.tid; g < half; g += b.nt) {
    const uint2 v = Z2[g];
    Z2[g] = make_uint2(mod_add(v.x, v.y, p), mod_sub(v.x, v.y, p));
  }
}

// Forward transforms of Z0 and Z1 (2^logn residues each) modulo prime j:
// radix-4 passes from the longest stage down, then the last radix-2 stage
// when logn is odd. One barrier per pass.
template <bool WHOLE>
__device__ __forceinline__ void ntt_forward2(const Blk& b, uint32_t* Z0, uint32_t* Z1, int logn, const uint32_t* tab,
                                             int j) {
  const uint32_t p = __ldg(tab + mp_ntt::kP + j);
  const uint2* fw = reinterpret_cast<const uint2*>(tab + j * mp_ntt::kPerPrime + mp_ntt::kFw);
  const int quarter = (1 << logn) >> 2;
  int lm = logn - 1;
  for (; lm >= 1; lm -= 2) {
    const int m = 1 << lm, h = m >> 1;
#pragma unroll 2
    for (int g = b.tid; g < quarter; g += b.nt) {
      const int i = g & (h - 1);
      const int base = ((g >> (lm - 1)) << (lm + 1)) + i;
      const uint2 w1 = __ldg(fw + m + i), w2 = __ldg(fw + m + h + i), w3 = __ldg(fw + h + i);
      dif4(Z0 + base, h, p, w1.x, w1.y, w2.x, w2.y, w3.x, w3.y);
      dif4(Z1 + base, h, p, w1.x, w1.y, w2.x, w2.y, w3.x, w3.y);
    }
    group_sync<WHOLE>(b);
  }
  if (lm == 0) {
    ntt_pairs(b, Z0, 1 << (logn - 1), p);
    ntt_pairs(b, Z1, 1 << (logn - 1), p);
    group_sync<WHOLE>(b);
  }
}

// Inverse transform of Z (bit-reversed order in, natural order out, times N):
// the radix-2 stage of half-length 1 first when logn is odd, then radix-4
// passes upward.
template <bool WHOLE>
__device__ __forceinline__ void ntt_inverse(const Blk& b, uint32_t* Z, int logn, const uint32_t* tab, int j) {
  const uint32_t p = __ldg(tab + mp_ntt::kP + j);
  const uint2* iw = reinterpret_cast<const uint2*>(tab + j * mp_ntt::kPerPrime + mp_ntt::kIw);
  const int quarter = (1 << logn) >> 2;
  int lm = 0;
  if (logn & 1) {
    ntt_pairs(b, Z, 1 << (logn - 1), p);
    group_sync<WHOLE>(b);
    lm = 1;
  }
  for (; lm < logn; lm += 2) {
    const int h = 1 << lm, m = 2 * h;
#pragma unroll 2
    for (int g = b.tid; g < quarter; g += b.nt) {
      const int i = g & (h - 1);
      const int base = ((g >> lm) << (lm + 2)) + i;
      const uint2 u1 = __ldg(iw + h + i), u2 = __ldg(iw + m + i), u3 = __ldg(iw + m + h + i);
      dit4(Z + base, h, p, u1.x, u1.y, u2.x, u2.y, u3.x, u3.y);
    }
    group_sync<WHOLE>(b);
  }
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
    const uint32_t p = __ldg(tab + mp_ntt::kP + j), pinv = __ldg(tab + mp_ntt::kPinv + j);
    uint32_t* Z = S + j * N;
    for (int i = b.tid; i < N; i += b.nt) {
      Z[i] = i < nx ? mod_red(X[i], p) : 0u;
      T[i] = i < ny ? mod_red(Y[i], p) : 0u;
    }
    group_sync<WHOLE>(b);
    ntt_forward2<WHOLE>(b, Z, T, logn, tab, j);
    for (int i = b.tid; i < N; i += b.nt) Z[i] = mod_mont(Z[i], T[i], p, pinv);
    group_sync<WHOLE>(b);
    ntt_inverse<WHOLE>(b, Z, logn, tab, j);
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

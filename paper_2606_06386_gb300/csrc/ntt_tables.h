// Constants of the number-theoretic-transform product: three primes
// p = c 2^k + 1 below 2^31 (so that a sum of two residues fits a 32-bit word)
// whose multiplicative groups hold roots of unity of every power-of-two order
// up to kMax, and the tables the device reads (twiddle factors with their
// Shoup companions, Montgomery and Garner constants), built on the host.
// Host-only code apart from the constants; no CUDA types.
#pragma once
#include <cstdint>

namespace mp_ntt {

constexpr int kLogMax = 13;
constexpr int kMax = 1 << kLogMax;  // longest transform: products of up to 8192 digits

// 63*2^25+1, 15*2^27+1, 27*2^26+1, with a primitive root of each
constexpr uint32_t kPrime[3] = {2113929217u, 2013265921u, 1811939329u};
constexpr uint32_t kRoot[3] = {5u, 31u, 13u};

// Table layout (32-bit words). For prime j at j*4*kMax: the forward twiddles
// w_k = omega_{2m}^i for k = m + i (m = 1, 2, 4, ..., kMax/2; i < m;
// omega_{2m} a primitive 2m-th root of unity), each followed by its Shoup
// companion floor(w 2^32 / p) (the pair for k at kFw + 2k, one 8-byte load);
// then the inverse twiddles omega_{2m}^-i with companions at kIw + 2k.
constexpr int kFw = 0, kIw = 2 * kMax;
constexpr int kPerPrime = 4 * kMax;
// Constants after the three prime blocks:
constexpr int kConst = 3 * kPerPrime;
constexpr int kP = kConst + 0;      // p_j
constexpr int kPinv = kConst + 3;   // -p_j^-1 mod 2^32 (Montgomery)
constexpr int kScale = kConst + 8;  // [j][t]: (2^32 / 2^t) mod p_j and companion, t = 0..kLogMax
constexpr int kGarner = kScale + 2 * 3 * (kLogMax + 1);
// Garner's constants (with Shoup companions): p1^-1 mod p2, p1 mod p3,
// (p1 p2)^-1 mod p3; then p1 p2 as two words.
constexpr int kInv12 = kGarner + 0, kP1m3 = kGarner + 2, kInv123 = kGarner + 4, kP12 = kGarner + 6;
constexpr int kWords = kGarner + 8;

inline uint32_t mulmod(uint32_t a, uint32_t b, uint32_t p) { return (uint32_t)((uint64_t)a * b % p); }

inline uint32_t powmod(uint32_t a, uint64_t e, uint32_t p) {
  uint32_t r = 1u % p, x = a % p;
  for (; e; e >>= 1) {
    if (e & 1) r = mulmod(r, x, p);
    x = mulmod(x, x, p);
  }
  return r;
}

inline uint32_t invmod(uint32_t a, uint32_t p) { return powmod(a, p - 2u, p); }  // p prime, a != 0 mod p

inline uint32_t shoup_companion(uint32_t w, uint32_t p) { return (uint32_t)(((uint64_t)w << 32) / p); }

// Fill t[0..kWords).
inline void build_tables(uint32_t* t) {
  for (int j = 0; j < 3; j++) {
    const uint32_t p = kPrime[j];
    uint32_t* b = t + j * kPerPrime;
    b[kFw] = b[kFw + 1] = b[kIw] = b[kIw + 1] = 0u;  // pair 0 is not used
    for (int m = 1; m < kMax; m *= 2) {
      const uint32_t w = powmod(kRoot[j], (p - 1u) / (2u * (uint32_t)m), p);
      const uint32_t wi = invmod(w, p);
      uint32_t f = 1u, g = 1u;
      for (int i = 0; i < m; i++) {
        b[kFw + 2 * (m + i)] = f;
        b[kFw + 2 * (m + i) + 1] = shoup_companion(f, p);
        b[kIw + 2 * (m + i)] = g;
        b[kIw + 2 * (m + i) + 1] = shoup_companion(g, p);
        f = mulmod(f, w, p);
        g = mulmod(g, wi, p);
      }
    }
    t[kP + j] = p;
    uint32_t inv = 1u;  // p^-1 mod 2^32 by Newton's iteration on the 2-adic inverse
    for (int k = 0; k < 5; k++) inv *= 2u - p * inv;
    t[kPinv + j] = 0u - inv;
    const uint32_t r = (uint32_t)((1ull << 32) % p);
    for (int s = 0; s <= kLogMax; s++) {
      const uint32_t c = mulmod(r, invmod(powmod(2u, (uint64_t)s, p), p), p);
      t[kScale + 2 * (j * (kLogMax + 1) + s)] = c;
      t[kScale + 2 * (j * (kLogMax + 1) + s) + 1] = shoup_companion(c, p);
    }
  }
  for (int i = kPinv + 3; i < kScale; i++) t[i] = 0u;
  const uint32_t p1 = kPrime[0], p2 = kPrime[1], p3 = kPrime[2];
  const uint32_t i12 = invmod(p1 % p2, p2), p1m3 = p1 % p3;
  const uint32_t i123 = invmod(mulmod(p1 % p3, p2 % p3, p3), p3);
  t[kInv12] = i12;
  t[kInv12 + 1] = shoup_companion(i12, p2);
  t[kP1m3] = p1m3;
  t[kP1m3 + 1] = shoup_companion(p1m3, p3);
  t[kInv123] = i123;
  t[kInv123 + 1] = shoup_companion(i123, p3);
  const uint64_t p12 = (uint64_t)p1 * p2;
  t[kP12] = (uint32_t)p12;
  t[kP12 + 1] = (uint32_t)(p12 >> 32);
}

}  // namespace mp_ntt

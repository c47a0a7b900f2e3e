// CPU check of the transform product's constants (csrc/ntt_tables.h): the
// primes, the roots of unity and their orders, the Shoup companions, the
// Montgomery, scaling and Garner constants, the bound that makes three primes
// enough, and an exact product through the tables (a transform written here
// from the textbook definitions) against the schoolbook product.
#include <cstdio>
#include <cstdlib>
#include <random>
#include <vector>

#include "ntt_tables.h"

using namespace mp_ntt;
typedef unsigned __int128 u128;

static int fails = 0;
#define CHECK(c)                                                   \
  do {                                                             \
    if (!(c)) {                                                    \
      std::printf("FAIL %s:%d %s\n", __FILE__, __LINE__, #c);      \
      if (++fails > 20) std::exit(1);                              \
    }                                                              \
  } while (0)

static bool is_prime(uint32_t p) {
  if (p < 2) return false;
  for (uint64_t d = 2; d * d <= p; d++)
    if (p % d == 0) return false;
  return true;
}

// x^e mod p by square and multiply, independent of the header's helper
static uint32_t pw(uint32_t x, uint64_t e, uint32_t p) {
  uint64_t r = 1, b = x % p;
  for (; e; e >>= 1, b = b * b % p)
    if (e & 1) r = r * b % p;
  return (uint32_t)r;
}

// Exact product of a and b by the cyclic convolution modulo each prime
// (the DFT by its defining sum would be too slow at 8192 points; this is the
// radix-2 recursion of the DFT, evaluated with the table's roots) and the
// Chinese remainder theorem on 128-bit integers.
static void dft(std::vector<uint32_t>& a, uint32_t p, const uint32_t* fw, bool inv, const uint32_t* iw) {
  // fw, iw: (twiddle, companion) pairs; twiddle k at index 2k
  const size_t n = a.size();
  if (n == 1) return;
  std::vector<uint32_t> ev(n / 2), od(n / 2);
  for (size_t i = 0; i < n / 2; i++) {
    ev[i] = a[2 * i];
    od[i] = a[2 * i + 1];
  }
  dft(ev, p, fw, inv, iw);
  dft(od, p, fw, inv, iw);
  const size_t m = n / 2;  // omega_n^k = twiddle m + k for k < m
  for (size_t k = 0; k < m; k++) {
    const uint32_t w = inv ? iw[2 * (m + k)] : fw[2 * (m + k)];
    const uint32_t t = (uint32_t)((uint64_t)w * od[k] % p);
    a[k] = (uint32_t)(((uint64_t)ev[k] + t) % p);
    a[k + m] = (uint32_t)(((uint64_t)ev[k] + p - t) % p);
  }
}

static std::vector<uint32_t> product_by_tables(const std::vector<uint32_t>& a, const std::vector<uint32_t>& b,
                                               const std::vector<uint32_t>& tab) {
  const size_t n = a.size() + b.size();
  size_t N = 2;
  while (N < n) N *= 2;
  std::vector<std::vector<uint32_t>> res(3);
  for (int j = 0; j < 3; j++) {
    const uint32_t p = kPrime[j];
    const uint32_t* base = tab.data() + j * kPerPrime;
    std::vector<uint32_t> x(N, 0), y(N, 0);
    for (size_t i = 0; i < a.size(); i++) x[i] = a[i] % p;
    for (size_t i = 0; i < b.size(); i++) y[i] = b[i] % p;
    dft(x, p, base + kFw, false, base + kIw);
    dft(y, p, base + kFw, false, base + kIw);
    for (size_t i = 0; i < N; i++) x[i] = (uint32_t)((uint64_t)x[i] * y[i] % p);
    dft(x, p, base + kFw, true, base + kIw);
    const uint32_t ninv = pw((uint32_t)(N % p), p - 2, p);
    for (size_t i = 0; i < N; i++) x[i] = (uint32_t)((uint64_t)x[i] * ninv % p);
    res[j] = x;
  }
  const u128 p1 = kPrime[0], p2 = kPrime[1], p3 = kPrime[2], M = p1 * p2 * p3;
  std::vector<uint32_t> out(n + 3, 0);
  u128 carry = 0;
  std::vector<u128> coef(N);
  // the unique value below M with the three residues (textbook CRT: sum of
  // r_j (M / p_j) ((M / p_j)^-1 mod p_j), reduced mod M; inverses by Fermat)
  u128 e[3];
  const u128 pj[3] = {p1, p2, p3};
  for (int j = 0; j < 3; j++) {
    const u128 mj = M / pj[j];
    e[j] = mj * pw((uint32_t)(mj % pj[j]), (uint64_t)pj[j] - 2, (uint32_t)pj[j]);  // < M p_j < 2^124
  }
  for (size_t k = 0; k < N; k++) {
    u128 y = 0;
    for (int j = 0; j < 3; j++) y = (y + (e[j] % M) * res[j][k] % M) % M;
    coef[k] = y;
  }
  for (size_t k = 0; k < n + 3; k++) {
    u128 s = carry + (k < N ? coef[k] : 0);
    out[k] = (uint32_t)s;
    carry = s >> 32;
  }
  out.resize(n);
  return out;
}

static std::vector<uint32_t> schoolbook(const std::vector<uint32_t>& a, const std::vector<uint32_t>& b) {
  std::vector<uint32_t> c(a.size() + b.size(), 0);
  for (size_t i = 0; i < a.size(); i++) {
    uint64_t carry = 0;
    for (size_t j = 0; j < b.size(); j++) {
      const uint64_t t = (uint64_t)a[i] * b[j] + c[i + j] + carry;
      c[i + j] = (uint32_t)t;
      carry = t >> 32;
    }
    c[i + b.size()] = (uint32_t)carry;
  }
  return c;
}

int main() {
  std::vector<uint32_t> tab(kWords, 0xdeadbeefu);
  build_tables(tab.data());
  // primes below 2^31 (sums of two residues fit a word), 2^32 < 3p (two
  // conditional subtractions reduce a word), roots of every order up to kMax
  for (int j = 0; j < 3; j++) {
    const uint32_t p = kPrime[j];
    CHECK(is_prime(p));
    CHECK(p < (1u << 31));
    CHECK(3ull * p > (1ull << 32));
    CHECK((p - 1) % (uint32_t)kMax == 0);
    CHECK(pw(kRoot[j], (p - 1) / 2, p) == p - 1);  // a non-residue: its 2-power part has full order
    CHECK(tab[kP + j] == p);
    CHECK((uint32_t)(tab[kPinv + j] * p) == 0xffffffffu);  // -p^-1 * p = -1 mod 2^32
    const uint32_t* b = tab.data() + j * kPerPrime;
    for (int m = 1; m < kMax; m *= 2) {
      const uint32_t w = (m >= 2) ? b[kFw + 2 * (m + 1)] : p - 1;  // omega_{2m}
      CHECK(pw(w, (uint64_t)m, p) == p - 1);                       // order exactly 2m
      if (m >= 2) CHECK(pw(w, 2, p) == (m >= 4 ? b[kFw + 2 * (m / 2 + 1)] : p - 1));
      for (int i = 0; i < m; i++) {
        const uint32_t f = b[kFw + 2 * (m + i)], g = b[kIw + 2 * (m + i)];
        CHECK(f == pw(w, (uint64_t)i, p));
        CHECK((uint64_t)f * g % p == 1);
        CHECK(b[kFw + 2 * (m + i) + 1] == (uint32_t)(((uint64_t)f << 32) / p));
        CHECK(b[kIw + 2 * (m + i) + 1] == (uint32_t)(((uint64_t)g << 32) / p));
      }
    }
    for (int s = 0; s <= kLogMax; s++) {
      const uint32_t c = tab[kScale + 2 * (j * (kLogMax + 1) + s)];
      CHECK((uint64_t)c * pw(2, (uint64_t)s, p) % p == (1ull << 32) % p);  // c 2^s = 2^32 mod p
      CHECK(tab[kScale + 2 * (j * (kLogMax + 1) + s) + 1] == (uint32_t)(((uint64_t)c << 32) / p));
    }
  }
  const uint64_t p1 = kPrime[0], p2 = kPrime[1], p3 = kPrime[2];
  CHECK(tab[kInv12] * p1 % p2 == 1);
  CHECK(tab[kP1m3] == p1 % p3);
  CHECK((u128)tab[kInv123] * (p1 * p2 % p3) % p3 == 1);
  CHECK(((uint64_t)tab[kP12 + 1] << 32 | tab[kP12]) == p1 * p2);
  for (int i : {kInv12, kP1m3, kInv123}) {
    const uint32_t p = (i == kInv12) ? (uint32_t)p2 : (uint32_t)p3;
    CHECK(tab[i + 1] == (uint32_t)(((uint64_t)tab[i] << 32) / p));
  }
  // three primes hold every coefficient of a product of nx + ny <= kMax digits
  const u128 bmax = (u128)0xffffffffu * 0xffffffffu * (kMax / 2);
  CHECK((u128)p1 * p2 * p3 > bmax);
  // Shoup's estimate is at most one short for any 32-bit x
  std::mt19937_64 rng(12345);
  for (int it = 0; it < 200000; it++) {
    const int j = it % 3;
    const uint32_t p = kPrime[j];
    const int idx = 1 + (int)(rng() % (kMax - 1));
    const uint32_t w = tab[j * kPerPrime + kFw + 2 * idx], ws = tab[j * kPerPrime + kFw + 2 * idx + 1];
    const uint32_t x = (uint32_t)rng();
    const uint32_t q = (uint32_t)(((uint64_t)x * ws) >> 32);
    const uint32_t r = x * w - q * p;
    CHECK(r < 2 * p);
    CHECK(r % p == (uint64_t)x * w % p);
  }
  // exact products through the tables
  struct Case {
    int na, nb, kind;
  } cases[] = {{1, 1, 0}, {3, 5, 0}, {17, 30, 1}, {100, 100, 0}, {64, 1, 1},
               {1000, 24, 2}, {2048, 2048, 1}, {4096, 4096, 1}, {4096, 4096, 0}, {7000, 1192, 2}};
  for (const Case& c : cases) {
    std::vector<uint32_t> a(c.na), b(c.nb);
    for (auto& d : a) d = c.kind == 1 ? 0xffffffffu : c.kind == 2 ? (uint32_t)(rng() % 3 == 0 ? 0 : 0xffffffffu) : (uint32_t)rng();
    for (auto& d : b) d = c.kind == 1 ? 0xffffffffu : c.kind == 2 ? (uint32_t)(rng() % 2 ? 1 : 0xffffffffu) : (uint32_t)rng();
    CHECK(product_by_tables(a, b, tab) == schoolbook(a, b));
  }
  if (fails) return 1;
  std::printf("ok\n");
  return 0;
}

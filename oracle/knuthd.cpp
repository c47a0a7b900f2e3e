// Test oracle for batched multi-precision division (test infrastructure).
//
// Only the test-suite, the smoke check and the benchmark's CPU-baseline leg may
// load this library; the product path never does, and this file shares no code,
// header, table or helper with the CUDA path.
//
// What it computes is the plain definition the paper states for Div(u, v)
// (Section 2, Algorithm 3's output; Definition 1 for shinv):
//     q = floor(u / v),  r = u - q v,  so  u = q v + r  with  0 <= r < v,
//     shinv_h(v) = floor(B^h / v)  with  B = 2^32.
// It gets there by the classical long division of Knuth, TAOCP Vol. 2,
// Section 4.3.1, Algorithm D (normalise, estimate each quotient digit from the
// top two remainder digits and the top divisor digit, correct the estimate at
// most twice with the second divisor digit, multiply-and-subtract, add back on
// a negative result, unnormalise the remainder), written from the textbook's
// description. One-digit divisors use short division.
//
// The template is instantiated for 8-, 16- and 32-bit digits. The narrow
// digits exist only so that tests can drive the rare add-back step (its
// probability is about 2/B per quotient digit) against native 128-bit
// division; ``oracle_addback_count`` reports how often it ran.
//
// A second, independent routine (``oracle_check_u32``) verifies a claimed
// (q, r) by schoolbook multiplication: u == q v + r and r < v.

#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>
#include <atomic>
#include <algorithm>

namespace {

std::atomic<long long> g_addback{0};

template <typename L>
struct Digits {
  static constexpr int bits = 8 * (int)sizeof(L);
  static constexpr uint64_t base = 1ull << bits;
};

// number of significant digits (0 for zero)
template <typename L>
int sig_len(const L* x, int n) {
  while (n > 0 && x[n - 1] == 0) n--;
  return n;
}

template <typename L>
int count_leading_zero_bits(L x) {
  int s = 0;
  const int bits = Digits<L>::bits;
  while (s < bits && !((x >> (bits - 1 - s)) & 1)) s++;
  return s;
}

// Algorithm D. u has un digits, v has vn digits; q gets qn digits (zero-padded),
// r gets rn digits (zero-padded). Returns 0, or 1 when v == 0. The output
// buffers must hold at least max(un - vn + 1, 1) and vn significant digits
// respectively; otherwise returns 2.
template <typename L>
int divmod(const L* u_in, int un, const L* v_in, int vn, L* q, int qn, L* r, int rn) {
  const int bits = Digits<L>::bits;
  const uint64_t B = Digits<L>::base;
  const uint64_t mask = B - 1;
  int m_all = sig_len(u_in, un);
  int n = sig_len(v_in, vn);
  if (q && qn > 0) std::memset(q, 0, sizeof(L) * (size_t)qn);
  if (r && rn > 0) std::memset(r, 0, sizeof(L) * (size_t)rn);
  if (n == 0) return 1;
  // u < v: q = 0, r = u
  bool u_lt_v = false;
  if (m_all < n) {
    u_lt_v = true;
  } else if (m_all == n) {
    int i = n - 1;
    while (i >= 0 && u_in[i] == v_in[i]) i--;
    u_lt_v = (i >= 0 && u_in[i] < v_in[i]);
  }
  if (u_lt_v) {
    if (m_all > rn) return 2;
    for (int i = 0; i < m_all; i++) r[i] = u_in[i];
    return 0;
  }
  const int m = m_all - n;  // quotient has m + 1 digits
  if (m + 1 > qn || n > rn) return 2;
  if (n == 1) {
    // short division, most significant digit first
    uint64_t d = v_in[0], rem = 0;
    for (int i = m_all - 1; i >= 0; i--) {
      uint64_t cur = (rem << bits) | u_in[i];
      q[i] = (L)(cur / d);
      rem = cur % d;
    }
    r[0] = (L)rem;
    return 0;
  }
  // D1: normalise so that the top divisor digit has its high bit set
  const int s = count_leading_zero_bits<L>(v_in[n - 1]);
  std::vector<L> vv(n), uu(m_all + 1);
  for (int i = n - 1; i > 0; i--)
    vv[i] = (L)(((uint64_t)v_in[i] << s | (s ? (uint64_t)v_in[i - 1] >> (bits - s) : 0)) & mask);
  vv[0] = (L)(((uint64_t)v_in[0] << s) & mask);
  uu[m_all] = (L)(s ? ((uint64_t)u_in[m_all - 1] >> (bits - s)) : 0);
  for (int i = m_all - 1; i > 0; i--)
    uu[i] = (L)(((uint64_t)u_in[i] << s | (s ? (uint64_t)u_in[i - 1] >> (bits - s) : 0)) & mask);
  uu[0] = (L)(((uint64_t)u_in[0] << s) & mask);
  const uint64_t vtop = vv[n - 1], vnext = vv[n - 2];
  // D2..D7: one quotient digit per step, from the top
  for (int j = m; j >= 0; j--) {
    // D3: estimate qhat from the top two digits of the current remainder
    uint64_t num = ((uint64_t)uu[j + n] << bits) | uu[j + n - 1];
    uint64_t qhat = num / vtop;
    uint64_t rhat = num % vtop;
    while (qhat >= B || qhat * vnext > ((rhat << bits) | uu[j + n - 2])) {
      qhat--;
      rhat += vtop;
      if (rhat >= B) break;
    }
    // D4: multiply and subtract qhat * v from uu[j .. j+n]
    uint64_t carry = 0;
    int64_t borrow = 0;
    for (int i = 0; i < n; i++) {
      uint64_t p = qhat * vv[i] + carry;
      carry = p >> bits;
      int64_t t = (int64_t)uu[i + j] - (int64_t)(p & mask) - borrow;
      borrow = t < 0 ? 1 : 0;
      uu[i + j] = (L)((uint64_t)t & mask);
    }
    int64_t t = (int64_t)uu[j + n] - (int64_t)carry - borrow;
    uu[j + n] = (L)((uint64_t)t & mask);
    // D5/D6: a negative result means qhat was one too large: add v back
    if (t < 0) {
      g_addback.fetch_add(1, std::memory_order_relaxed);
      qhat--;
      uint64_t c = 0;
      for (int i = 0; i < n; i++) {
        uint64_t sum = (uint64_t)uu[i + j] + vv[i] + c;
        uu[i + j] = (L)(sum & mask);
        c = sum >> bits;
      }
      uu[j + n] = (L)(((uint64_t)uu[j + n] + c) & mask);
    }
    q[j] = (L)qhat;
  }
  // D8: unnormalise the remainder
  for (int i = 0; i < n - 1; i++)
    r[i] = (L)((((uint64_t)uu[i] >> s) | (s ? ((uint64_t)uu[i + 1] << (bits - s)) : 0)) & mask);
  r[n - 1] = (L)((uint64_t)uu[n - 1] >> s);
  return 0;
}

}  // namespace

extern "C" {

int oracle_divmod_u32(const uint32_t* u, int un, const uint32_t* v, int vn, uint32_t* q, int qn, uint32_t* r,
                      int rn) {
  return divmod<uint32_t>(u, un, v, vn, q, qn, r, rn);
}
int oracle_divmod_u16(const uint16_t* u, int un, const uint16_t* v, int vn, uint16_t* q, int qn, uint16_t* r,
                      int rn) {
  return divmod<uint16_t>(u, un, v, vn, q, qn, r, rn);
}
int oracle_divmod_u8(const uint8_t* u, int un, const uint8_t* v, int vn, uint8_t* q, int qn, uint8_t* r, int rn) {
  return divmod<uint8_t>(u, un, v, vn, q, qn, r, rn);
}

long long oracle_addback_count(void) { return g_addback.load(); }
void oracle_addback_reset(void) { g_addback.store(0); }

// shinv_h(v) = floor(B^h / v), B = 2^32 (Definition 1), as the quotient of
// B^h by v. out gets outn digits. Returns 0, 1 for v == 0, 2 if outn is short.
int oracle_shinv_u32(const uint32_t* v, int vn, int h, uint32_t* out, int outn) {
  std::vector<uint32_t> bh((size_t)h + 1, 0u);
  bh[h] = 1u;
  int n = sig_len(v, vn);
  std::vector<uint32_t> rem((size_t)std::max(n, 1), 0u);
  return divmod<uint32_t>(bh.data(), h + 1, v, vn, out, outn, rem.data(), std::max(n, 1));
}

// Independent verification of a claimed division: returns 0 when
// u == q*v + r and r < v (all little-endian 32-bit digits), 1 when the identity
// fails, 2 when r >= v, 3 when v == 0.
int oracle_check_u32(const uint32_t* u, int un, const uint32_t* v, int vn, const uint32_t* q, int qn,
                     const uint32_t* r, int rn) {
  int vs = sig_len(v, vn);
  if (vs == 0) return 3;
  int qs = sig_len(q, qn), rs = sig_len(r, rn), us = sig_len(u, un);
  // r < v
  if (rs > vs) return 2;
  if (rs == vs) {
    int i = vs - 1;
    while (i >= 0 && r[i] == v[i]) i--;
    if (i < 0 || r[i] > v[i]) return 2;
  }
  // t = q * v (schoolbook, row by row), then t += r
  std::vector<uint32_t> t((size_t)qs + vs + 2, 0u);
  for (int i = 0; i < qs; i++) {
    uint64_t c = 0;
    for (int j = 0; j < vs; j++) {
      uint64_t p = (uint64_t)q[i] * v[j] + t[i + j] + c;
      t[i + j] = (uint32_t)p;
      c = p >> 32;
    }
    int k = i + vs;
    while (c) {
      uint64_t s = (uint64_t)t[k] + c;
      t[k] = (uint32_t)s;
      c = s >> 32;
      k++;
    }
  }
  uint64_t c = 0;
  for (size_t i = 0; i < t.size(); i++) {
    uint64_t s = (uint64_t)t[i] + (i < (size_t)rs ? r[i] : 0u) + c;
    t[i] = (uint32_t)s;
    c = s >> 32;
  }
  if (c) return 1;
  int ts = sig_len(t.data(), (int)t.size());
  if (ts != us) return 1;
  for (int i = 0; i < us; i++)
    if (t[i] != u[i]) return 1;
  return 0;
}

// Batched form for timing and bulk parity: item i reads u + i*us, v + i*vs and
// writes q + i*qs, r + i*rs (strides in digits), with the digit counts given.
// Items are split into contiguous ranges over nthreads host threads
// (nthreads <= 0: all hardware threads). status[i] gets the per-item code.
// Returns the number of threads used.
int oracle_divmod_batch_u32(long long n_items, const uint32_t* u, int un, long long us, const uint32_t* v, int vn,
                            long long vs, uint32_t* q, int qn, long long qs, uint32_t* r, int rn, long long rs,
                            int32_t* status, int nthreads) {
  if (nthreads <= 0) nthreads = (int)std::max(1u, std::thread::hardware_concurrency());
  if (n_items < nthreads) nthreads = (int)std::max(1ll, n_items);
  auto work = [&](long long b, long long e) {
    for (long long i = b; i < e; i++)
      status[i] = divmod<uint32_t>(u + i * us, un, v + i * vs, vn, q + i * qs, qn, r + i * rs, rn);
  };
  if (nthreads == 1) {
    work(0, n_items);
    return 1;
  }
  std::vector<std::thread> th;
  for (int t = 0; t < nthreads; t++) {
    long long b = n_items * t / nthreads, e = n_items * (t + 1) / nthreads;
    th.emplace_back(work, b, e);
  }
  for (auto& x : th) x.join();
  return nthreads;
}

// Ragged batched form: per-item digit offsets and counts.
int oracle_divmod_ragged_u32(long long n_items, const uint32_t* u, const long long* u_off, const int* u_len,
                             const uint32_t* v, const long long* v_off, const int* v_len, uint32_t* q,
                             const long long* q_off, const int* q_len, uint32_t* r, const long long* r_off,
                             const int* r_len, int32_t* status, int nthreads) {
  if (nthreads <= 0) nthreads = (int)std::max(1u, std::thread::hardware_concurrency());
  if (n_items < nthreads) nthreads = (int)std::max(1ll, n_items);
  auto work = [&](long long b, long long e) {
    for (long long i = b; i < e; i++)
      status[i] = divmod<uint32_t>(u + u_off[i], u_len[i], v + v_off[i], v_len[i], q + q_off[i], q_len[i],
                                   r + r_off[i], r_len[i]);
  };
  if (nthreads == 1) {
    work(0, n_items);
    return 1;
  }
  std::vector<std::thread> th;
  for (int t = 0; t < nthreads; t++) {
    long long b = n_items * t / nthreads, e = n_items * (t + 1) / nthreads;
    th.emplace_back(work, b, e);
  }
  for (auto& x : th) x.join();
  return nthreads;
}

}  // extern "C"

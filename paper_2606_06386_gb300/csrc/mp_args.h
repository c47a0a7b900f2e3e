// Kernel argument blocks, shared by the kernels and the host runtime.
#pragma once
#include <cstdint>

namespace mp {

struct UniformArgs {
  const uint32_t* u;
  const uint32_t* v;
  uint32_t* q;
  uint32_t* r;
  int32_t* status;
  int32_t* iters;
  int64_t* products;  // per item: algorithmic digit products (may be null)
  int64_t n, us, vs, qs, rs;
  int un, vn, qn, rn;
  int smem_words;
  int flags;
  int tcols;  // columns per lane of the strip multiply
  int kcut;   // Karatsuba cutoff for full products (0: schoolbook only)
  const uint32_t* ntt;  // transform tables for full products (null: strip products only)
  int ntt_cut;          // the transform for products of at least this many digits
  // Item list of a ragged batch (null: item i at the strides and digit counts
  // above): the launch's i-th division is item list[i], whose operands and
  // results are at the offsets and digit counts of the arrays below, and
  // whose status (iterations, products) go to index list[i].
  const int32_t* list;
  const int64_t *u_off, *v_off, *q_off, *r_off;
  const int32_t *u_len, *v_len, *q_len, *r_len;
  // 0: one pass. 1: the fit pass, whose shared memory covers the items whose
  // operands' effective lengths are their buffers' (an item whose plan is
  // larger gets the internal retry status); 2: the retry pass, which divides
  // only the items with that status, in shared memory for any item.
  int pass;
};

struct RaggedArgs {
  const uint32_t* u;
  const int64_t* u_off;
  const int32_t* u_len;
  const uint32_t* v;
  const int64_t* v_off;
  const int32_t* v_len;
  uint32_t* q;
  const int64_t* q_off;
  const int32_t* q_len;
  uint32_t* r;
  const int64_t* r_off;
  const int32_t* r_len;
  int32_t* status;
  int32_t* iters;
  int64_t* products;
  const int32_t* order;  // item indices, most expensive first
  int32_t* head;         // queue head, zero at launch
  int64_t n;
  int smem_words;
  int flags;
  int tcols;            // columns per lane (0 in k_div_persistent: chosen per item)
  // k_div_persistent, per size class of the dividend (<= 1024, 2048, 4096,
  // 8192 and more digits, see class_of): columns per lane, Karatsuba cutoff
  // (when kcut < 0) and the warps a division of that class wants
  int tcols_class[5];
  int kcut;  // Karatsuba cutoff for full products (0: schoolbook only)
  int kcut_class[5];
  int want_class[5];
  const uint32_t* ntt;  // transform tables for full products (null: strip products only)
  int ntt_cut;
};

// Size class of a dividend of ul digits in the persistent kernel's tables.
__host__ __device__ __forceinline__ int class_of(int ul) {
  return ul <= 1024 ? 0 : ul <= 2048 ? 1 : ul <= 4096 ? 2 : ul <= 8192 ? 3 : 4;
}

struct ShinvArgs {
  const uint32_t* v;
  const int32_t* h;
  uint32_t* out;
  int32_t* iters;
  int32_t* status;
  int64_t n, vs, os;
  int vn, on;
  int smem_words;
  int tcols;
  int kcut;
  int flags;  // MPDIV_FLAG_FULL_PRODUCTS is honoured; the others are ignored
  const uint32_t* ntt;  // transform tables for full products (null: strip products only)
  int ntt_cut;
};

// Test entry: one group primitive per item (mpdiv_debug_primitive).
struct PrimArgs {
  const uint32_t* x;
  const uint32_t* y;
  uint32_t* out;
  int32_t* result;
  int64_t n;
  int nx, ny, cap;
  int op, arg;
  int tcols;
  int smem_words;
  const uint32_t* ntt;  // transform tables (op 9)
};

}  // namespace mp

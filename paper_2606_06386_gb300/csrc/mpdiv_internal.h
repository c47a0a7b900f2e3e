// Internal state and launch descriptors shared by the host-side sources.
#pragma once
#include <atomic>
#include <condition_variable>
#include <cstdint>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "mp_args.h"
#include "mpdiv.h"

struct MpServer;  // mpdiv_serve.cu

// Forms of a ragged launch: one plain launch per size class over its item
// list (forked, or one graph), the self-splitting persistent kernel, or the
// one-block-per-item queue kernel (16-warp blocks).
enum RaggedForm { RF_CLASSES = 0, RF_SPLIT = 1, RF_QUEUE = 2 };
constexpr int kMaxRuns = 5;  // size classes of a ragged batch (mp::class_of)

struct mpdiv_ctx {
  int device = 0;
  int num_sms = 0;
  int max_smem = 0;
  int smem_per_sm = 0;  // shared memory of one SM (all resident blocks)
  mpdiv_config cfg{0, 0, 0, 0, 0, 0, 0};
  uint32_t* d_ntt = nullptr;  // transform tables (ntt_tables.h), built at init
  mutable std::mutex err_mu;
  std::string err;
  // tuning table: size class (digits, power of two >= 128) -> launch shape
  std::mutex tune_mu;
  struct Shape {
    int warps, tcols, kcut;
    int regs;  // registers per thread of the plain kernel: 64, 128, or 0 (chosen by occupancy)
  };
  std::map<int, Shape> tuned;
  // persistent launch: queue head, cached order, cached graph
  std::mutex ragged_mu;
  // occupancies by (kernel, threads, shared memory)
  std::mutex attr_mu;
  std::map<std::tuple<void*, int, int>, int> occupancy;
  int32_t* d_head = nullptr;
  int32_t* d_order = nullptr;
  size_t order_cap = 0;
  std::vector<int32_t> order_u_len, order_v_len;  // the shape list the cached order was made for
  std::vector<int32_t> order_host;                // the cached order
  int order_form = -1;                            // and its form
  int64_t order_n = -1;
  // class form: forked streams, their events, and the captured graph
  cudaStream_t side[kMaxRuns] = {};
  cudaEvent_t fork_ev = nullptr, join_ev[kMaxRuns] = {};
  cudaGraphExec_t cgexec = nullptr;
  std::vector<char> c_desc;
  cudaEvent_t ragged_ev = nullptr;  // the last launch on the context's queue head and order array
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t gexec = nullptr;
  mp::RaggedArgs g_args{};
  int64_t g_grid = 0;
  int g_warps = 0, g_smem = 0;
  int64_t graph_captures = 0, graph_replays = 0;
  // serving
  MpServer* server = nullptr;
};

struct UniformLaunch {
  const uint32_t *u, *v;
  uint32_t *q, *r;
  int32_t *status, *iters;
  int64_t* products;
  int64_t n, us, vs, qs, rs;
  int un, vn, qn, rn;
  int warps;  // 0: from the tuning table
  int tcols;  // 0: from the tuning table
  int kcut;   // -1: from the tuning table; 0: schoolbook only
  int regs;   // registers per thread: 64, 128 (4, 8 and 16 warps), 0: from the tuning table, else by occupancy
  // item list of a ragged batch's size class (null: the strided uniform
  // batch); un is then the largest dividend of the list
  const int32_t* list;
  const int64_t *u_off, *v_off, *q_off, *r_off;
  const int32_t *u_len, *v_len, *q_len, *r_len;
  // host copies of the list and of the items' digit counts (with list): the
  // fit pass's shared memory covers the largest plan of the listed items
  const int32_t *list_host, *u_len_host, *v_len_host;
};

// A plain launch ready to go: kernel, arguments, grid, threads, shared memory;
// with retry_grid > 0 a fit pass (args.pass = 1, shared memory for the batch's
// own operand lengths, so more blocks fit on an SM) followed by a retry pass
// (grid retry_grid, shared memory retry_smem) for the items whose effective
// lengths need a larger plan.
struct PreparedLaunch {
  void* kernel = nullptr;
  mp::UniformArgs args{};
  int64_t grid = 0;
  int threads = 0, smem = 0;
  int64_t retry_grid = 0;
  int retry_smem = 0;
};

struct RaggedLaunch {
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
  int32_t *status, *iters;
  int64_t* products;
  const int32_t *u_len_host, *v_len_host;
  const int32_t* order;       // device order array (nullptr: computed and cached here)
  const int32_t* order_host;  // its host copy (with order)
  int32_t* head;              // device queue head of the queue forms (nullptr: the context's)
  int64_t n;
  bool use_graph;   // capture/replay as a CUDA graph
  bool grid_items;  // queue forms: one block per item instead of one wave of resident blocks
  int form;         // RaggedForm
};

int mpdiv_set_error(mpdiv_ctx* ctx, int code, const char* fmt, ...);
int mpdiv_cuda_check(mpdiv_ctx* ctx, cudaError_t e, const char* what);
int mpdiv_smem_bytes(int max_digits, int flags, int tcols);
// Raise kernel k's dynamic shared memory limit on the current device to at
// least smem bytes (never lowers it; shared by every context and entry point).
cudaError_t mpdiv_open_kernel_smem(void* k, int smem);
int mpdiv_size_class(int digits);
int mpdiv_default_warps(mpdiv_ctx* ctx, int max_digits);
int mpdiv_default_tcols(mpdiv_ctx* ctx, int max_digits);
int mpdiv_default_kcut(mpdiv_ctx* ctx, int max_digits);
int mpdiv_default_regs(mpdiv_ctx* ctx, int max_digits);
int mpdiv_ragged_form(const mpdiv_ctx* ctx);  // RF_SPLIT with MPDIV_FLAG_PERSISTENT_QUEUE, else RF_CLASSES
int mpdiv_launch_uniform(mpdiv_ctx* ctx, const UniformLaunch& L, cudaStream_t stream);
int mpdiv_prepare_uniform(mpdiv_ctx* ctx, const UniformLaunch& L, PreparedLaunch* P);
int mpdiv_launch_prepared(mpdiv_ctx* ctx, const PreparedLaunch& P, cudaStream_t stream);
int mpdiv_launch_ragged(mpdiv_ctx* ctx, const RaggedLaunch& L, cudaStream_t stream);
void mpdiv_tune_load(mpdiv_ctx* ctx, const char* path);
void mpdiv_serve_shutdown(mpdiv_ctx* ctx);

// A named NVTX range over a scope (batch, queue, tuning and serving phases);
// free unless a profiler is attached.
struct MpdivRange {
  explicit MpdivRange(const char* name) { nvtxRangePushA(name); }
  ~MpdivRange() { nvtxRangePop(); }
  MpdivRange(const MpdivRange&) = delete;
  MpdivRange& operator=(const MpdivRange&) = delete;
};

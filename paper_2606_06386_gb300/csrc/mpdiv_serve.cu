// Continuous-batching server for divisions of mixed precision.
//
// A scheduler thread owns a device operand pool and a pinned host mirror of
// it. Requests are admitted first-in first-out into batches: each batch takes
// one contiguous range of the pool holding its operands, its per-item
// offsets, lengths and queue order (largest first), its queue head and its
// results. A batch is one host-to-device copy, one launch of the persistent
// division kernel with one block per item (so blocks of the next batch fill
// SMs as blocks of the current one retire), and one device-to-host copy, on
// its own stream. Up to max_inflight batches run at once; requests that arrive
// meanwhile wait for the next free slot and pool range. The kernel is the
// same division path as the plain launch, so a result does not depend on the
// batch an item lands in.
#include <algorithm>
#include <atomic>
#include <map>
#include <chrono>
#include <cstring>
#include <deque>
#include <memory>
#include <numeric>
#include <thread>
#include <unordered_map>
#include <vector>

#include "mpdiv_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

int64_t now_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(Clock::now().time_since_epoch()).count();
}

enum ReqState { RQ_QUEUED = 0, RQ_RUNNING = 1, RQ_DONE = 2 };

struct Request {
  uint64_t ticket;
  int32_t u_len, v_len, q_len, r_len;
  std::vector<uint32_t> u, v;  // operands until launch
  std::vector<uint32_t> q, r;  // results once done
  int32_t status = 0;
  int state = RQ_QUEUED;
  int64_t t_submit = 0, t_done = 0;
};

// first-fit allocator over [0, size) in digit units; ranges are 4-digit aligned
struct RangeAlloc {
  std::map<int64_t, int64_t> free_;  // offset -> length
  explicit RangeAlloc(int64_t size = 0) {
    if (size > 0) free_[0] = size;
  }
  int64_t largest() const {
    int64_t m = 0;
    for (auto& kv : free_) m = std::max(m, kv.second);
    return m;
  }
  int64_t alloc(int64_t n) {
    n = (n + 3) & ~int64_t(3);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= n) {
        const int64_t off = it->first, len = it->second;
        free_.erase(it);
        if (len > n) free_[off + n] = len - n;
        return off;
      }
    }
    return -1;
  }
  void release(int64_t off, int64_t n) {
    n = (n + 3) & ~int64_t(3);
    auto it = free_.emplace(off, n).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
};

// digits needed by a batch of requests: operands, metadata (int64 offsets as
// two digits), head, results
int64_t batch_layout(const std::vector<Request*>& rs, std::vector<int64_t>& offs) {
  const int64_t n = (int64_t)rs.size();
  int64_t a = 0;
  offs.assign(16, 0);
  offs[0] = a;  // u digits
  for (auto* r : rs) a += r->u_len;
  a = (a + 3) & ~3;
  offs[1] = a;  // v digits
  for (auto* r : rs) a += r->v_len;
  a = (a + 3) & ~3;
  offs[2] = a;  // u_off, v_off, q_off, r_off: int64 each
  a += 4 * 2 * n;
  offs[3] = a;  // u_len, v_len, q_len, r_len, order: int32 each
  a += 5 * n;
  offs[4] = a;  // head (+ padding)
  a += 4;
  offs[5] = a;  // end of what is copied to the device
  a = (a + 3) & ~3;
  offs[6] = a;  // status
  a += n;
  a = (a + 3) & ~3;
  offs[7] = a;  // q digits
  for (auto* r : rs) a += r->q_len;
  a = (a + 3) & ~3;
  offs[8] = a;  // r digits
  for (auto* r : rs) a += r->r_len;
  offs[9] = a;  // total
  return a;
}

}  // namespace

struct MpServer {
  mpdiv_ctx* ctx;
  mpdiv_serve_config cfg;
  uint32_t* d_pool = nullptr;
  uint32_t* h_pool = nullptr;  // pinned mirror
  RangeAlloc alloc;
  std::mutex mu;
  std::condition_variable cv_sched, cv_done;
  std::deque<Request*> queue;
  std::unordered_map<uint64_t, std::unique_ptr<Request>> reqs;
  uint64_t next_ticket = 1;
  int64_t pending = 0;  // queued + running
  bool stopping = false, quit = false;
  std::thread th;
  int64_t completed = 0, launches = 0, batched_items = 0;
  struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t ev = nullptr;
    bool busy = false;
    int64_t range_off = 0, range_len = 0;
    std::vector<Request*> reqs;
    std::vector<int64_t> offs;
  };
  std::vector<Slot> slots;
  int sched_error = 0;

  void run();
  bool launch(Slot& s, std::vector<Request*>& batch, int64_t off, int64_t len);
  void finish(Slot& s);
};

bool MpServer::launch(Slot& s, std::vector<Request*>& batch, int64_t off, int64_t len) {
  const int64_t n = (int64_t)batch.size();
  std::vector<int64_t> o;
  batch_layout(batch, o);
  uint32_t* H = h_pool + off;
  uint32_t* D = d_pool + off;
  int64_t* h_off = reinterpret_cast<int64_t*>(H + o[2]);
  int32_t* h_len = reinterpret_cast<int32_t*>(H + o[3]);
  int64_t pu = o[0], pv = o[1], pq = o[7], pr = o[8];
  std::vector<double> cost(n);
  for (int64_t i = 0; i < n; i++) {
    Request* r = batch[i];
    std::memcpy(H + pu, r->u.data(), 4 * (size_t)r->u_len);
    std::memcpy(H + pv, r->v.data(), 4 * (size_t)r->v_len);
    h_off[0 * n + i] = pu - o[0];
    h_off[1 * n + i] = pv - o[1];
    h_off[2 * n + i] = pq - o[7];
    h_off[3 * n + i] = pr - o[8];
    h_len[0 * n + i] = r->u_len;
    h_len[1 * n + i] = r->v_len;
    h_len[2 * n + i] = r->q_len;
    h_len[3 * n + i] = r->r_len;
    pu += r->u_len;
    pv += r->v_len;
    pq += r->q_len;
    pr += r->r_len;
    const double a = std::max(1, r->u_len - r->v_len + 1);
    cost[i] = a * (r->u_len + r->v_len) + 2.0 * a * std::min<double>(a, r->v_len);
    r->u.clear();
    r->u.shrink_to_fit();
    r->v.clear();
    r->v.shrink_to_fit();
    r->state = RQ_RUNNING;
  }
  int32_t* order = h_len + 4 * n;
  std::iota(order, order + n, 0);
  std::stable_sort(order, order + n, [&](int32_t a, int32_t b) { return cost[a] > cost[b]; });
  std::memset(H + o[4], 0, 16);  // queue head
  cudaError_t e = cudaMemcpyAsync(D, H, 4 * (size_t)o[5], cudaMemcpyHostToDevice, s.stream);
  std::vector<int32_t> ulh(n), vlh(n);
  for (int64_t i = 0; i < n; i++) {
    ulh[i] = batch[i]->u_len;
    vlh[i] = batch[i]->v_len;
  }
  RaggedLaunch L{};
  const int64_t* d_off = reinterpret_cast<const int64_t*>(D + o[2]);
  const int32_t* d_len = reinterpret_cast<const int32_t*>(D + o[3]);
  L.u = D + o[0];
  L.u_off = d_off;
  L.u_len = d_len;
  L.v = D + o[1];
  L.v_off = d_off + n;
  L.v_len = d_len + n;
  L.q = D + o[7];
  L.q_off = d_off + 2 * n;
  L.q_len = d_len + 2 * n;
  L.r = D + o[8];
  L.r_off = d_off + 3 * n;
  L.r_len = d_len + 3 * n;
  L.status = reinterpret_cast<int32_t*>(D + o[6]);
  L.iters = nullptr;
  L.u_len_host = ulh.data();
  L.v_len_host = vlh.data();
  L.order = d_len + 4 * n;
  L.head = reinterpret_cast<int32_t*>(D + o[4]);
  L.n = n;
  L.use_graph = false;
  L.grid_items = true;
  int rc = (e == cudaSuccess) ? mpdiv_launch_ragged(ctx, L, s.stream) : MPDIV_ECUDA;
  if (rc == MPDIV_OK)
    e = cudaMemcpyAsync(H + o[6], D + o[6], 4 * (size_t)(o[9] - o[6]), cudaMemcpyDeviceToHost, s.stream);
  if (rc == MPDIV_OK && e == cudaSuccess) e = cudaEventRecord(s.ev, s.stream);
  if (rc != MPDIV_OK || e != cudaSuccess) {
    // the operands are consumed: fail these requests instead of requeueing them
    sched_error = rc != MPDIV_OK ? rc : MPDIV_ECUDA;
    const int64_t t = now_ns();
    for (Request* r : batch) {
      r->q.assign(r->q_len, 0u);
      r->r.assign(r->r_len, 0u);
      r->status = MPDIV_ST_INTERNAL;
      r->state = RQ_DONE;
      r->t_done = t;
    }
    pending -= n;
    cv_done.notify_all();
    return false;
  }
  s.busy = true;
  s.range_off = off;
  s.range_len = len;
  s.reqs = batch;
  s.offs = o;
  launches++;
  batched_items += n;
  return true;
}

void MpServer::finish(Slot& s) {
  const std::vector<int64_t>& o = s.offs;
  const uint32_t* H = h_pool + s.range_off;
  const int32_t* st = reinterpret_cast<const int32_t*>(H + o[6]);
  int64_t pq = o[7], pr = o[8];
  const int64_t t = now_ns();
  for (size_t i = 0; i < s.reqs.size(); i++) {
    Request* r = s.reqs[i];
    r->q.assign(H + pq, H + pq + r->q_len);
    r->r.assign(H + pr, H + pr + r->r_len);
    pq += r->q_len;
    pr += r->r_len;
    r->status = st[i];
    r->state = RQ_DONE;
    r->t_done = t;
  }
  completed += (int64_t)s.reqs.size();
  pending -= (int64_t)s.reqs.size();
  alloc.release(s.range_off, s.range_len);
  s.reqs.clear();
  s.busy = false;
}

void MpServer::run() {
  cudaSetDevice(ctx->device);
  std::unique_lock<std::mutex> lk(mu);
  while (true) {
    bool progressed = false;
    int busy = 0;
    for (auto& s : slots) {
      if (!s.busy) continue;
      if (cudaEventQuery(s.ev) == cudaSuccess) {
        finish(s);
        progressed = true;
      } else {
        busy++;
      }
    }
    if (progressed) cv_done.notify_all();
    // admit the next batch into a free slot
    Slot* free_slot = nullptr;
    for (auto& s : slots)
      if (!s.busy) {
        free_slot = &s;
        break;
      }
    if (free_slot && !queue.empty() && sched_error == 0) {
      std::vector<Request*> batch;
      std::vector<int64_t> o;
      const int64_t room = alloc.largest();
      while (!queue.empty() && (int)batch.size() < cfg.max_batch) {
        batch.push_back(queue.front());
        if (batch_layout(batch, o) > room) {
          batch.pop_back();
          break;
        }
        queue.pop_front();
      }
      if (!batch.empty()) {
        const int64_t len = batch_layout(batch, o);
        const int64_t off = alloc.alloc(len);
        if (off < 0) {
          for (auto it = batch.rbegin(); it != batch.rend(); ++it) queue.push_front(*it);
        } else if (launch(*free_slot, batch, off, len)) {
          progressed = true;
          busy++;
        } else {
          alloc.release(off, len);
          progressed = true;
        }
      }
    }
    if (quit && busy == 0 && (queue.empty() || sched_error)) break;
    if (!progressed) {
      if (busy > 0)
        cv_sched.wait_for(lk, std::chrono::microseconds(20));
      else
        cv_sched.wait_for(lk, std::chrono::milliseconds(5));
    }
  }
}

// ------------------------------------------------------------------ C ABI
extern "C" int mpdiv_serve_start(mpdiv_ctx* ctx, const mpdiv_serve_config* cfg) {
  if (!ctx) return MPDIV_EINVAL;
  if (ctx->server) {
    bool stopped;
    {
      std::lock_guard<std::mutex> g(ctx->server->mu);
      stopped = ctx->server->stopping;
    }
    if (!stopped) return mpdiv_set_error(ctx, MPDIV_ESTATE, "server already running");
    mpdiv_serve_shutdown(ctx);  // a stopped server is released: its unpolled results are dropped
  }
  cudaSetDevice(ctx->device);
  auto* S = new MpServer();
  S->ctx = ctx;
  S->cfg = cfg ? *cfg : mpdiv_serve_config{0, 0, 0, 0};
  if (S->cfg.pool_digits <= 0) S->cfg.pool_digits = 64ll << 20;
  if (S->cfg.max_batch <= 0) S->cfg.max_batch = 4096;
  if (S->cfg.max_inflight <= 0) S->cfg.max_inflight = 3;
  if (S->cfg.max_pending <= 0) S->cfg.max_pending = 1 << 20;
  int rc = mpdiv_cuda_check(ctx, cudaMalloc(&S->d_pool, 4 * (size_t)S->cfg.pool_digits), "server pool");
  if (rc == MPDIV_OK)
    rc = mpdiv_cuda_check(ctx, cudaMallocHost(&S->h_pool, 4 * (size_t)S->cfg.pool_digits), "server host pool");
  if (rc != MPDIV_OK) {
    cudaFree(S->d_pool);
    delete S;
    return rc;
  }
  S->alloc = RangeAlloc(S->cfg.pool_digits);
  S->slots.resize(S->cfg.max_inflight);
  for (auto& s : S->slots) {
    cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking);
    cudaEventCreateWithFlags(&s.ev, cudaEventDisableTiming);
  }
  ctx->server = S;
  S->th = std::thread([S] { S->run(); });
  return MPDIV_OK;
}

static int64_t footprint(int32_t u_len, int32_t v_len) {
  return 2 * (int64_t)u_len + 2 * (int64_t)v_len + 16 + 16;
}

extern "C" int mpdiv_serve_submit(mpdiv_ctx* ctx, const uint32_t* u_host, int32_t u_len, const uint32_t* v_host,
                                  int32_t v_len, uint64_t* ticket) {
  if (!ctx || !u_host || !v_host || !ticket) return MPDIV_EINVAL;
  MpServer* S = ctx->server;
  if (!S) return mpdiv_set_error(ctx, MPDIV_ESTATE, "server not running");
  if (u_len < 1 || v_len < 1) return mpdiv_set_error(ctx, MPDIV_EINVAL, "digit counts must be positive");
  if (u_len > MPDIV_MAX_LIMBS || v_len > MPDIV_MAX_LIMBS)
    return mpdiv_set_error(ctx, MPDIV_EUNSUPPORTED, "at most %d digits", MPDIV_MAX_LIMBS);
  if (footprint(u_len, v_len) > S->cfg.pool_digits)
    return mpdiv_set_error(ctx, MPDIV_EBUSY, "request larger than the device pool");
  auto r = std::make_unique<Request>();
  r->u_len = u_len;
  r->v_len = v_len;
  r->q_len = u_len;  // enough for any quotient
  r->r_len = v_len;
  r->u.assign(u_host, u_host + u_len);
  r->v.assign(v_host, v_host + v_len);
  {
    std::lock_guard<std::mutex> g(S->mu);
    if (S->stopping) return mpdiv_set_error(ctx, MPDIV_ESTATE, "server stopping");
    if (S->pending >= S->cfg.max_pending) return MPDIV_EBUSY;
    r->ticket = S->next_ticket++;
    r->t_submit = now_ns();
    *ticket = r->ticket;
    S->queue.push_back(r.get());
    S->reqs.emplace(r->ticket, std::move(r));
    S->pending++;
  }
  S->cv_sched.notify_one();
  return MPDIV_OK;
}

static int poll_impl(mpdiv_ctx* ctx, uint64_t ticket, uint32_t* q_host, int32_t q_cap, uint32_t* r_host,
                     int32_t r_cap, int32_t* status, int64_t timeout_us, int64_t* t_done) {
  MpServer* S = ctx->server;
  if (!S) return mpdiv_set_error(ctx, MPDIV_ESTATE, "server not running");
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) return mpdiv_set_error(ctx, MPDIV_EINVAL, "unknown ticket");
  Request* r = it->second.get();
  if (r->state != RQ_DONE) {
    if (timeout_us <= 0) return MPDIV_PENDING;
    const auto until = Clock::now() + std::chrono::microseconds(timeout_us);
    while (r->state != RQ_DONE) {
      if (S->sched_error && r->state == RQ_QUEUED)
        return mpdiv_set_error(ctx, S->sched_error, "the server stopped after a failed launch");
      if (S->cv_done.wait_until(lk, until) == std::cv_status::timeout && r->state != RQ_DONE)
        return MPDIV_ETIMEDOUT;
    }
  }
  int qs = (int)r->q.size();
  while (qs > 0 && r->q[qs - 1] == 0u) qs--;
  if (q_host) {
    if (qs > q_cap) return mpdiv_set_error(ctx, MPDIV_EINVAL, "q_cap too small (%d digits needed)", qs);
    for (int i = 0; i < q_cap; i++) q_host[i] = i < qs ? r->q[i] : 0u;
  }
  if (r_host) {
    int rs = (int)r->r.size();
    while (rs > 0 && r->r[rs - 1] == 0u) rs--;
    if (rs > r_cap) return mpdiv_set_error(ctx, MPDIV_EINVAL, "r_cap too small");
    for (int i = 0; i < r_cap; i++) r_host[i] = i < rs ? r->r[i] : 0u;
  }
  if (status) *status = r->status;
  if (t_done) *t_done = r->t_done;
  S->reqs.erase(it);
  return MPDIV_OK;
}

extern "C" int mpdiv_serve_poll(mpdiv_ctx* ctx, uint64_t ticket, uint32_t* q_host, int32_t q_cap, uint32_t* r_host,
                                int32_t r_cap, int32_t* status, int64_t timeout_us) {
  if (!ctx) return MPDIV_EINVAL;
  return poll_impl(ctx, ticket, q_host, q_cap, r_host, r_cap, status, timeout_us, nullptr);
}

static void stop_impl(MpServer* S) {
  {
    std::lock_guard<std::mutex> g(S->mu);
    S->stopping = true;
    S->quit = true;
  }
  S->cv_sched.notify_all();
  if (S->th.joinable()) S->th.join();
}

extern "C" int mpdiv_serve_stop(mpdiv_ctx* ctx) {
  if (!ctx) return MPDIV_EINVAL;
  MpServer* S = ctx->server;
  if (!S) return mpdiv_set_error(ctx, MPDIV_ESTATE, "server not running");
  stop_impl(S);
  return S->sched_error ? mpdiv_set_error(ctx, S->sched_error, "a batch failed to launch") : MPDIV_OK;
}

extern "C" int mpdiv_serve_stats(mpdiv_ctx* ctx, int64_t* completed, int64_t* launches, int64_t* batched_items) {
  if (!ctx || !ctx->server) return MPDIV_EINVAL;
  MpServer* S = ctx->server;
  std::lock_guard<std::mutex> g(S->mu);
  if (completed) *completed = S->completed;
  if (launches) *launches = S->launches;
  if (batched_items) *batched_items = S->batched_items;
  return MPDIV_OK;
}

void mpdiv_serve_shutdown(mpdiv_ctx* ctx) {
  MpServer* S = ctx->server;
  if (!S) return;
  stop_impl(S);
  cudaSetDevice(ctx->device);
  for (auto& s : S->slots) {
    if (s.stream) cudaStreamSynchronize(s.stream);
    if (s.ev) cudaEventDestroy(s.ev);
    if (s.stream) cudaStreamDestroy(s.stream);
  }
  cudaFree(S->d_pool);
  cudaFreeHost(S->h_pool);
  delete S;
  ctx->server = nullptr;
}

// Open-loop replay of an arrival stream against the running server (the
// serving measurement): request i is submitted at t0 + arrival_ns[i]; its
// latency is the time from that scheduled arrival until its result is
// pollable on the host. Operands come from flat host arrays with offsets;
// quotients (q_len[i] digits) and remainders (r_len[i] digits) are written to
// host arrays. Returns MPDIV_OK or the first error; *rejected counts EBUSY
// retries.
extern "C" int mpdiv_serve_replay(mpdiv_ctx* ctx, int64_t n, const int64_t* arrival_ns, const uint32_t* u,
                                  const int64_t* u_off, const int32_t* u_len, const uint32_t* v,
                                  const int64_t* v_off, const int32_t* v_len, uint32_t* q, const int64_t* q_off,
                                  const int32_t* q_len, uint32_t* r, const int64_t* r_off, const int32_t* r_len,
                                  int32_t* status, int64_t* latency_ns, int64_t* rejected) {
  if (!ctx || !ctx->server || n < 0) return MPDIV_EINVAL;
  std::vector<uint64_t> tickets((size_t)n);
  std::vector<int64_t> t_arr((size_t)n);
  int64_t rej = 0;
  int err = MPDIV_OK;
  const int64_t t0 = now_ns();
  std::atomic<int64_t> submitted{0};
  std::thread submitter([&] {
    for (int64_t i = 0; i < n; i++) {
      const int64_t due = t0 + arrival_ns[i];
      while (now_ns() < due) {
        const int64_t gap = due - now_ns();
        if (gap > 200000) std::this_thread::sleep_for(std::chrono::nanoseconds(gap - 100000));
      }
      t_arr[i] = due;
      while (true) {
        const int rc = mpdiv_serve_submit(ctx, u + u_off[i], u_len[i], v + v_off[i], v_len[i], &tickets[i]);
        if (rc == MPDIV_OK) break;
        if (rc != MPDIV_EBUSY) {
          err = rc;
          tickets[i] = 0;
          break;
        }
        rej++;
        std::this_thread::sleep_for(std::chrono::microseconds(20));
      }
      submitted.store(i + 1, std::memory_order_release);
    }
  });
  for (int64_t i = 0; i < n; i++) {
    while (submitted.load(std::memory_order_acquire) <= i) std::this_thread::sleep_for(std::chrono::microseconds(5));
    if (tickets[i] == 0) {
      status[i] = -1;
      latency_ns[i] = -1;
      continue;
    }
    int64_t td = 0;
    int rc;
    while ((rc = poll_impl(ctx, tickets[i], q + q_off[i], q_len[i], r + r_off[i], r_len[i], &status[i], 1000000,
                           &td)) == MPDIV_ETIMEDOUT) {
    }
    if (rc != MPDIV_OK && err == MPDIV_OK) err = rc;
    latency_ns[i] = td - t_arr[i];
  }
  submitter.join();
  if (rejected) *rejected = rej;
  return err;
}

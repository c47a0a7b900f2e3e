// Continuous-batching server for divisions of mixed precision.
//
// Requests are admitted by footprint: each belongs to the footprint class of
// its dividend (at most 1024, 2048, 4096, 8192 digits, or more: the size
// classes whose shared-memory plan and block shape the launches are tuned
// for), and a batch holds requests of one class only, so that a large request
// never sets the block shape and shared memory of a batch of small ones.
// Operands travel through two pinned host rings mirrored on the device: an
// input ring (u and v of every request, in arrival order) and an output ring
// (q and r of every launched request). mpdiv_serve_submit reserves the
// request's digits at the tail of the input ring and copies its operands there
// itself, outside the server lock. A scheduler thread turns the oldest ready
// requests of a class into a batch: the run of the input ring from its first
// request to its last (one host-to-device copy on the server's copy stream; the
// run may hold requests of other classes and requests still being copied in,
// see copy_stream), per-item
// offsets and a most-expensive-first order (one more copy), one plain launch
// over the batch with the class's tuned shape (or, with
// MPDIV_FLAG_PERSISTENT_QUEUE, one launch of the self-splitting persistent
// kernel), and one device-to-host copy of the batch's results, all on the
// batch's own stream; batches of different classes overlap on the GPU.
// Up to max_inflight batches run at once. The class whose oldest ready request
// is oldest goes first. While fewer than low_water requests are on the GPU,
// the queued requests of a class launch as soon as there are at least
// batch_step of them for every batch of that class already in flight (so an
// idle class launches each request at once, and a busy one launches fewer,
// larger batches instead of being bound by the launch path); otherwise they
// gather into larger batches (up to max_batch, or until the oldest has waited
// max_wait_us).
// The kernel is the division path of the plain launch, so a result does not
// depend on the batch a request lands in.
//
// A batch whose launch fails fails its requests and every queued one (status
// MPDIV_ST_INTERNAL, and poll returns MPDIV_ECUDA for them), and the server
// refuses further work until it is stopped.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <numeric>
#include <thread>
#include <vector>

#include "mpdiv_internal.h"
#include "serve_ring.h"

namespace {

// Requests a launch needs per batch already in flight while the GPU is below
// its low-water mark (see the header comment), unless configured.
constexpr int kBatchStep = 8;

// Footprint classes: the dividend's size class (mp::class_of).
constexpr int kClasses = MPDIV_SERVE_CLASSES;

using Clock = std::chrono::steady_clock;

int64_t now_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(Clock::now().time_since_epoch()).count();
}

enum ReqState { RQ_QUEUED = 0, RQ_RUNNING = 1, RQ_DONE = 2 };

// The output-ring allocation of one batch; released when every request of
// the batch has been polled.
struct OutBatch {
  int64_t seq = -1;
  std::atomic<int> remaining{0};
};

struct Request {
  uint64_t ticket = 0;
  int32_t u_len = 0, v_len = 0, q_len = 0, r_len = 0;
  int cls = 0;                    // footprint class
  bool failed = false;            // its batch could not be launched
  int64_t in_off = -1;            // u at in_off, v at in_off + u_len (input ring digits)
  int64_t in_seq = -1;            // its input-ring allocation
  int64_t out_off = -1;           // q at out_off, r at out_off + q_len (output ring digits)
  std::shared_ptr<OutBatch> out;  // the batch's output allocation
  std::atomic<int> ready{0};      // operands copied into the ring
  int32_t status = 0;
  std::atomic<int> state{RQ_QUEUED};  // RQ_DONE is published with release order
  int64_t t_submit = 0, t_done = 0;
};

}  // namespace

struct MpServer {
  mpdiv_ctx* ctx = nullptr;
  mpdiv_serve_config cfg{};
  uint32_t *d_in = nullptr, *h_in = nullptr, *d_out = nullptr, *h_out = nullptr;
  mp_serve::Ring in_ring, out_ring;
  std::mutex mu;
  std::condition_variable cv_sched, cv_done;
  std::deque<Request*> queue[kClasses];
  int64_t queued = 0;  // requests in all queues
  // request of ticket t at by_ticket[t & ticket_mask], owned there until it is
  // polled (a poller claims it by swapping the slot to null, without the lock)
  std::unique_ptr<std::atomic<Request*>[]> by_ticket;
  uint64_t ticket_mask = 0;
  uint64_t next_ticket = 1;
  int64_t pending = 0, inflight_items = 0;
  bool stopping = false, quit = false;
  int sched_error = 0;
  int64_t completed = 0, launches = 0, batched_items = 0;
  int64_t class_launches[kClasses] = {}, class_items[kClasses] = {};  // by the batch's largest dividend
  int64_t fail_launch = -1;  // test hook: the launch with this index fails on the host (-1: none)
  std::thread th;
  // operand copies of every batch, in admission order: a batch's copy may
  // span ring space of requests still being written by their submitters
  // (skipped, to be taken by a later batch), and the later batch's own copy of
  // that space must land after this stale one
  cudaStream_t copy_stream = nullptr;
  struct Slot {
    MpServer* server = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev = nullptr;
    cudaEvent_t copied = nullptr;  // the batch's operand copy is done
    // set by a host function the slot's stream runs after the batch's results
    // are on the host, so that the scheduler reads a flag per slot instead of
    // querying an event
    std::atomic<int> done{0};
    uint32_t *h_meta = nullptr, *d_meta = nullptr;  // offsets, lengths, order, heads, status
    bool busy = false;
    int cls = 0;  // footprint class of the batch in flight
    int64_t out_off = -1, out_seq = -1;
    std::vector<Request*> reqs;
  };
  std::vector<Slot> slots;
  int64_t meta_words = 0;

  std::vector<Request*> skipped;  // scheduler scratch: requests a batch passed over

  void run();
  bool launch(Slot& s);
  static void CUDART_CB slot_done(void* p);
  void fail(Request* r, int64_t t);
};

// Mark a request failed (no results; status MPDIV_ST_INTERNAL) and release its
// input-ring space. Called with the lock held.
void MpServer::fail(Request* r, int64_t t) {
  r->out.reset();
  r->out_off = -1;
  r->failed = true;
  r->status = MPDIV_ST_INTERNAL;
  r->t_done = t;
  r->state.store(RQ_DONE, std::memory_order_release);
  in_ring.release(r->in_seq);
}

// metadata layout of a slot for n items: int64 offsets (u, v, q, r) as digit
// pairs, int32 lengths (u, v, q, r), order, queue heads, status
static int64_t meta_words_for(int64_t n) { return 8 * n + 5 * n + 8 + n + 8; }

bool MpServer::launch(Slot& s) {
  MpdivRange nvtx_range("mpdiv.serve.batch");
  const int64_t n = (int64_t)s.reqs.size();
  uint32_t* H = s.h_meta;
  int64_t* h_off = reinterpret_cast<int64_t*>(H);
  int32_t* h_len = reinterpret_cast<int32_t*>(H + 8 * n);
  int32_t* order = h_len + 4 * n;
  int32_t* heads = order + n;
  const int64_t status_w = 13 * n + 8;  // status after the heads
  std::vector<double> cost(n);
  int64_t pq = s.out_off;
  auto ob = std::make_shared<OutBatch>();
  ob->seq = s.out_seq;
  ob->remaining = (int)n;
  for (int64_t i = 0; i < n; i++) {
    Request* r = s.reqs[i];
    r->out_off = pq;
    r->out = ob;
    h_off[i] = r->in_off;
    h_off[n + i] = r->in_off + r->u_len;
    h_off[2 * n + i] = pq;
    h_off[3 * n + i] = pq + r->q_len;
    pq += r->q_len + r->r_len;
    h_len[i] = r->u_len;
    h_len[n + i] = r->v_len;
    h_len[2 * n + i] = r->q_len;
    h_len[3 * n + i] = r->r_len;
    const double a = std::max(1, r->u_len - r->v_len + 1);
    cost[i] = a * (r->u_len + r->v_len) + 2.0 * a * std::min<double>(a, r->v_len);
  }
  // the order of the context's ragged form: most expensive first (a batch is
  // one footprint class), or, for the self-splitting kernel, largest dividend
  // first (the shared memory a group must hold), then most expensive
  const int form = mpdiv_ragged_form(ctx);
  std::iota(order, order + n, 0);
  std::stable_sort(order, order + n, [&](int32_t a, int32_t b) {
    if (form == RF_SPLIT && s.reqs[a]->u_len != s.reqs[b]->u_len) return s.reqs[a]->u_len > s.reqs[b]->u_len;
    return cost[a] > cost[b];
  });
  std::memset(heads, 0, 8 * sizeof(int32_t));
  // operands: one contiguous run of the input ring
  // operands: one run of the input ring, from the first request of the batch
  // to the end of its last (a class's requests are in ring order), on the copy
  // stream
  const int64_t in_lo = s.reqs.front()->in_off;
  const int64_t in_hi = s.reqs.back()->in_off + s.reqs.back()->u_len + s.reqs.back()->v_len;
  cudaError_t e = cudaMemcpyAsync(d_in + in_lo, h_in + in_lo, 4 * (size_t)(in_hi - in_lo), cudaMemcpyHostToDevice,
                                  copy_stream);
  if (e == cudaSuccess) e = cudaEventRecord(s.copied, copy_stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s.stream, s.copied, 0);
  if (e == cudaSuccess) e = cudaMemcpyAsync(s.d_meta, H, 4 * (size_t)status_w, cudaMemcpyHostToDevice, s.stream);
  const int64_t* d_off = reinterpret_cast<const int64_t*>(s.d_meta);
  const int32_t* d_len = reinterpret_cast<const int32_t*>(s.d_meta + 8 * n);
  int32_t* d_status = reinterpret_cast<int32_t*>(s.d_meta + status_w);
  int rc = (e == cudaSuccess) ? MPDIV_OK : MPDIV_ECUDA;
  if (rc == MPDIV_OK) {
    // one launch over the batch in the context's ragged form
    std::vector<int32_t> ulh(n), vlh(n);
    for (int64_t i = 0; i < n; i++) {
      ulh[i] = s.reqs[i]->u_len;
      vlh[i] = s.reqs[i]->v_len;
    }
    RaggedLaunch L{};
    L.u = d_in;
    L.u_off = d_off;
    L.u_len = d_len;
    L.v = d_in;
    L.v_off = d_off + n;
    L.v_len = d_len + n;
    L.q = d_out;
    L.q_off = d_off + 2 * n;
    L.q_len = d_len + 2 * n;
    L.r = d_out;
    L.r_off = d_off + 3 * n;
    L.r_len = d_len + 3 * n;
    L.status = d_status;
    L.u_len_host = ulh.data();
    L.v_len_host = vlh.data();
    L.order = d_len + 4 * n;
    L.order_host = order;
    L.head = const_cast<int32_t*>(d_len + 5 * n);
    L.n = n;
    L.use_graph = false;
    L.form = form;
    rc = mpdiv_launch_ragged(ctx, L, s.stream);
  }
  if (rc == MPDIV_OK)
    e = cudaMemcpyAsync(h_out + s.out_off, d_out + s.out_off, 4 * (size_t)(pq - s.out_off), cudaMemcpyDeviceToHost,
                        s.stream);
  if (rc == MPDIV_OK && e == cudaSuccess)
    e = cudaMemcpyAsync(H + status_w, d_status, 4 * (size_t)n, cudaMemcpyDeviceToHost, s.stream);
  if (rc == MPDIV_OK && e == cudaSuccess) e = cudaLaunchHostFunc(s.stream, slot_done, &s);
  return rc == MPDIV_OK && e == cudaSuccess;
}

// Host function run by a slot's stream once its batch's results and statuses
// are on the host: flags the slot and wakes the scheduler (no CUDA call).
void CUDART_CB MpServer::slot_done(void* p) {
  Slot* s = static_cast<Slot*>(p);
  s->done.store(1, std::memory_order_release);
  s->server->cv_sched.notify_one();
}

void MpServer::run() {
  cudaSetDevice(ctx->device);
  std::vector<Slot*> finished;
  while (true) {
    // ---- completions: results stay in the pinned output ring until polled
    finished.clear();
    for (auto& s : slots)
      if (s.busy && s.done.load(std::memory_order_acquire)) finished.push_back(&s);
    std::unique_lock<std::mutex> lk(mu);
    const int64_t t = now_ns();
    for (Slot* s : finished) {
      const int64_t n = (int64_t)s->reqs.size();
      const int32_t* st = reinterpret_cast<const int32_t*>(s->h_meta + 13 * n + 8);
      for (int64_t i = 0; i < n; i++) {
        Request* r = s->reqs[i];
        r->status = st[i];
        r->t_done = t;
        r->state.store(RQ_DONE, std::memory_order_release);
        in_ring.release(r->in_seq);
      }
      completed += n;
      pending -= n;
      inflight_items -= n;
      s->reqs.clear();
      s->done.store(0, std::memory_order_relaxed);
      s->busy = false;
    }
    if (!finished.empty()) cv_done.notify_all();
    int busy = 0, busy_c[kClasses] = {};
    Slot* free_slot = nullptr;
    for (auto& s : slots) {
      if (s.busy) {
        busy++;
        busy_c[s.cls]++;
      } else if (!free_slot) {
        free_slot = &s;
      }
    }
    // ---- admission: the class whose oldest ready request is oldest among
    // those whose admission condition holds
    int adm = -1;
    if (free_slot && sched_error == 0) {
      int64_t oldest = INT64_MAX;
      for (int c = 0; c < kClasses; c++) {
        if (queue[c].empty() || !queue[c].front()->ready.load(std::memory_order_acquire)) continue;
        const Request* f = queue[c].front();
        const int64_t waited_us = (t - f->t_submit) / 1000;
        const bool go = (inflight_items < cfg.low_water && (int64_t)queue[c].size() >= (int64_t)cfg.batch_step * busy_c[c]) ||
                        (int64_t)queue[c].size() >= cfg.max_batch || waited_us >= cfg.max_wait_us || quit;
        if (go && f->t_submit < oldest) {
          oldest = f->t_submit;
          adm = c;
        }
      }
    }
    if (adm >= 0) {
      // the oldest ready requests of the class, in ring order and short of the
      // ring's wrap, within the output ring; requests whose submitters are
      // still copying their operands are skipped and stay queued in order
      std::deque<Request*>& qc = queue[adm];
      std::vector<Request*>& b = free_slot->reqs;
      int64_t out_need = 0;
      const int64_t out_room = out_ring.cap - out_ring.used - 4;
      skipped.clear();
      while (!qc.empty() && (int64_t)b.size() < cfg.max_batch) {
        Request* r = qc.front();
        if (!b.empty() && r->in_off < b.back()->in_off) break;  // the ring wrapped
        if (!r->ready.load(std::memory_order_acquire)) {
          skipped.push_back(r);
          qc.pop_front();
          continue;
        }
        const int64_t need = r->q_len + r->r_len;
        if (out_need + need > out_room) break;
        out_need += need;
        b.push_back(r);
        qc.pop_front();
      }
      for (auto it = skipped.rbegin(); it != skipped.rend(); ++it) qc.push_front(*it);
      queued -= (int64_t)b.size();
      int64_t oseq = -1;
      const int64_t off = b.empty() ? -1 : out_ring.alloc(out_need, &oseq);
      if (off < 0) {
        // put the batch back in ring order among the skipped requests
        for (auto it = b.rbegin(); it != b.rend(); ++it) qc.push_front(*it);
        std::stable_sort(qc.begin(), qc.begin() + (ptrdiff_t)(b.size() + skipped.size()),
                         [](const Request* x, const Request* y) { return x->in_off < y->in_off; });
        queued += (int64_t)b.size();
        b.clear();
      } else {
        free_slot->out_off = off;
        free_slot->out_seq = oseq;
        free_slot->busy = true;
        free_slot->cls = adm;
        int bcls = 0;
        for (Request* r : b) {
          r->state.store(RQ_RUNNING, std::memory_order_relaxed);
          bcls = std::max(bcls, mp::class_of(r->u_len));
        }
        const int64_t nb = (int64_t)b.size();
        const bool inject = launches == fail_launch;
        inflight_items += nb;
        launches++;
        batched_items += nb;
        class_launches[bcls]++;
        class_items[bcls] += nb;
        lk.unlock();
        const bool ok = !inject && launch(*free_slot);
        lk.lock();
        if (!ok) {  // fail these requests and every queued one, and refuse further work
          sched_error = MPDIV_ECUDA;
          const int64_t tf = now_ns();
          for (Request* r : b) fail(r, tf);
          out_ring.release(oseq);
          pending -= nb;
          inflight_items -= nb;
          b.clear();
          free_slot->busy = false;
          for (auto& qq : queue) {
            for (Request* r : qq) fail(r, tf);
            pending -= (int64_t)qq.size();
            qq.clear();
          }
          queued = 0;
          cv_done.notify_all();
        }
        continue;
      }
    }
    if (quit && busy == 0 && (queued == 0 || sched_error)) break;
    cv_sched.wait_for(lk, (busy > 0 || queued > 0) ? std::chrono::microseconds(20)
                                                  : std::chrono::microseconds(5000));
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
  if (cfg) S->cfg = *cfg;
  if (S->cfg.pool_digits <= 0) S->cfg.pool_digits = 64ll << 20;
  if (S->cfg.max_batch <= 0) S->cfg.max_batch = 4096;
  if (S->cfg.max_inflight <= 0) S->cfg.max_inflight = 32;
  if (S->cfg.max_pending <= 0) S->cfg.max_pending = 1 << 20;
  if (S->cfg.low_water <= 0) S->cfg.low_water = 2048;
  if (S->cfg.max_wait_us <= 0) S->cfg.max_wait_us = 2000;
  if (S->cfg.batch_step <= 0) S->cfg.batch_step = kBatchStep;
  const int64_t half = (S->cfg.pool_digits / 2) & ~int64_t(3);
  S->in_ring.cap = half;
  S->out_ring.cap = half;
  S->meta_words = meta_words_for(S->cfg.max_batch);
  {
    uint64_t cap = 1024;
    while (cap < 2 * (uint64_t)S->cfg.max_pending) cap *= 2;
    S->by_ticket.reset(new std::atomic<Request*>[cap]);
    for (uint64_t i = 0; i < cap; i++) S->by_ticket[i].store(nullptr, std::memory_order_relaxed);
    S->ticket_mask = cap - 1;
  }
  int rc = mpdiv_cuda_check(ctx, cudaMalloc(&S->d_in, 4 * (size_t)half), "server input ring");
  if (!rc) rc = mpdiv_cuda_check(ctx, cudaMalloc(&S->d_out, 4 * (size_t)half), "server output ring");
  if (!rc) rc = mpdiv_cuda_check(ctx, cudaMallocHost(&S->h_in, 4 * (size_t)half), "server pinned input ring");
  if (!rc) rc = mpdiv_cuda_check(ctx, cudaMallocHost(&S->h_out, 4 * (size_t)half), "server pinned output ring");
  if (!rc)
    rc = mpdiv_cuda_check(ctx, cudaStreamCreateWithFlags(&S->copy_stream, cudaStreamNonBlocking), "server copy stream");
  S->slots = std::vector<MpServer::Slot>(S->cfg.max_inflight);
  for (auto& s : S->slots) {
    s.server = S;
    if (rc) break;
    rc = mpdiv_cuda_check(ctx, cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking), "server stream");
    if (!rc) rc = mpdiv_cuda_check(ctx, cudaEventCreateWithFlags(&s.ev, cudaEventDisableTiming), "server event");
    if (!rc) rc = mpdiv_cuda_check(ctx, cudaEventCreateWithFlags(&s.copied, cudaEventDisableTiming), "server event");
    if (!rc) rc = mpdiv_cuda_check(ctx, cudaMallocHost(&s.h_meta, 4 * (size_t)S->meta_words), "server metadata");
    if (!rc) rc = mpdiv_cuda_check(ctx, cudaMalloc(&s.d_meta, 4 * (size_t)S->meta_words), "server metadata");
  }
  ctx->server = S;
  if (rc) {
    mpdiv_serve_shutdown(ctx);
    return rc;
  }
  S->th = std::thread([S] { S->run(); });
  return MPDIV_OK;
}

extern "C" int mpdiv_serve_submit(mpdiv_ctx* ctx, const uint32_t* u_host, int32_t u_len, const uint32_t* v_host,
                                  int32_t v_len, uint64_t* ticket) {
  if (!ctx || !u_host || !v_host || !ticket) return MPDIV_EINVAL;
  MpServer* S = ctx->server;
  if (!S) return mpdiv_set_error(ctx, MPDIV_ESTATE, "server not running");
  if (u_len < 1 || v_len < 1) return mpdiv_set_error(ctx, MPDIV_EINVAL, "digit counts must be positive");
  if (u_len > MPDIV_MAX_LIMBS || v_len > MPDIV_MAX_LIMBS)
    return mpdiv_set_error(ctx, MPDIV_EUNSUPPORTED, "at most %d digits", MPDIV_MAX_LIMBS);
  const int cls = mp::class_of(u_len);
  if (2 * (int64_t)(u_len + v_len) + 8 > S->in_ring.cap)
    return mpdiv_set_error(ctx, MPDIV_EBUSY, "request larger than the server's rings");
  auto r = std::make_unique<Request>();
  r->u_len = u_len;
  r->v_len = v_len;
  r->q_len = u_len;  // enough for any quotient
  r->r_len = v_len;
  r->cls = cls;
  Request* rp = r.get();
  bool wake = false;
  {
    std::lock_guard<std::mutex> g(S->mu);
    if (S->stopping) return mpdiv_set_error(ctx, MPDIV_ESTATE, "server stopping");
    if (S->sched_error) return mpdiv_set_error(ctx, S->sched_error, "the server stopped after a failed launch");
    if (S->pending >= S->cfg.max_pending) return MPDIV_EBUSY;
    // the ticket's slot still holds an unpolled result from ticket - capacity
    if (S->by_ticket[S->next_ticket & S->ticket_mask].load(std::memory_order_acquire) != nullptr) return MPDIV_EBUSY;
    int64_t seq = -1;
    const int64_t off = S->in_ring.alloc(u_len + v_len, &seq);
    if (off < 0) return MPDIV_EBUSY;  // input ring full: retry later
    r->in_off = off;
    r->in_seq = seq;
    r->ticket = S->next_ticket++;
    r->t_submit = now_ns();
    *ticket = r->ticket;
    // the scheduler re-checks a non-empty queue every few microseconds by
    // itself; only a request into an empty queue needs to wake it
    wake = S->queued == 0;
    S->queue[cls].push_back(rp);
    S->queued++;
    S->by_ticket[rp->ticket & S->ticket_mask].store(r.release(), std::memory_order_release);
    S->pending++;
  }
  // the operands go straight into the pinned ring; the scheduler waits for `ready`
  std::memcpy(S->h_in + rp->in_off, u_host, 4 * (size_t)u_len);
  std::memcpy(S->h_in + rp->in_off + u_len, v_host, 4 * (size_t)v_len);
  rp->ready.store(1, std::memory_order_release);
  if (wake) S->cv_sched.notify_one();
  return MPDIV_OK;
}

static int poll_impl(mpdiv_ctx* ctx, uint64_t ticket, uint32_t* q_host, int32_t q_cap, uint32_t* r_host,
                     int32_t r_cap, int32_t* status, int64_t timeout_us, int64_t* t_done) {
  MpServer* S = ctx->server;
  if (!S) return mpdiv_set_error(ctx, MPDIV_ESTATE, "server not running");
  std::atomic<Request*>& slot = S->by_ticket[ticket & S->ticket_mask];
  Request* r = slot.load(std::memory_order_acquire);
  if (r == nullptr || r->ticket != ticket) return mpdiv_set_error(ctx, MPDIV_EINVAL, "unknown ticket");
  if (r->state.load(std::memory_order_acquire) != RQ_DONE) {
    if (timeout_us <= 0) return MPDIV_PENDING;
    std::unique_lock<std::mutex> lk(S->mu);
    const auto until = Clock::now() + std::chrono::microseconds(timeout_us);
    while (r->state.load(std::memory_order_acquire) != RQ_DONE) {
      if (S->sched_error && r->state.load(std::memory_order_relaxed) == RQ_QUEUED)
        return mpdiv_set_error(ctx, S->sched_error, "the server stopped after a failed launch");
      if (S->cv_done.wait_until(lk, until) == std::cv_status::timeout &&
          r->state.load(std::memory_order_acquire) != RQ_DONE)
        return MPDIV_ETIMEDOUT;
    }
  }
  const uint32_t* qd = (r->out_off >= 0 && !r->failed) ? S->h_out + r->out_off : nullptr;
  if (qd && ((q_host && q_cap < r->q_len) || (r_host && r_cap < r->r_len))) {
    // a short buffer is fine when the digits it drops are zero
    int qs = r->q_len, rs = r->r_len;
    while (qs > 0 && qd[qs - 1] == 0u) qs--;
    while (rs > 0 && qd[r->q_len + rs - 1] == 0u) rs--;
    if (q_host && qs > q_cap) return mpdiv_set_error(ctx, MPDIV_EINVAL, "q_cap too small (%d digits needed)", qs);
    if (r_host && rs > r_cap) return mpdiv_set_error(ctx, MPDIV_EINVAL, "r_cap too small");
  }
  // claim the request: a concurrent poll of the same ticket finds it gone
  Request* expect = r;
  if (!slot.compare_exchange_strong(expect, nullptr, std::memory_order_acq_rel))
    return mpdiv_set_error(ctx, MPDIV_EINVAL, "unknown ticket");
  std::unique_ptr<Request> done(r);
  // the digits stay valid until this request's share of its batch is released below
  if (q_host) {
    const int n = qd ? std::min(q_cap, r->q_len) : 0;
    if (n) std::memcpy(q_host, qd, 4 * (size_t)n);
    for (int i = n; i < q_cap; i++) q_host[i] = 0u;
  }
  if (r_host) {
    const int n = qd ? std::min(r_cap, r->r_len) : 0;
    if (n) std::memcpy(r_host, qd + r->q_len, 4 * (size_t)n);
    for (int i = n; i < r_cap; i++) r_host[i] = 0u;
  }
  if (status) *status = r->status;
  if (t_done) *t_done = r->t_done;
  if (r->out && r->out->remaining.fetch_sub(1, std::memory_order_acq_rel) == 1) {
    std::lock_guard<std::mutex> g(S->mu);
    S->out_ring.release(r->out->seq);
  }
  if (r->failed) return mpdiv_set_error(ctx, MPDIV_ECUDA, "ticket %llu failed: its batch could not be launched",
                                        (unsigned long long)ticket);
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

extern "C" int mpdiv_serve_stats(mpdiv_ctx* ctx, int64_t* completed, int64_t* launches, int64_t* batched_items,
                                 int64_t* class_launches, int64_t* class_items) {
  if (!ctx || !ctx->server) return MPDIV_EINVAL;
  MpServer* S = ctx->server;
  std::lock_guard<std::mutex> g(S->mu);
  if (completed) *completed = S->completed;
  if (launches) *launches = S->launches;
  if (batched_items) *batched_items = S->batched_items;
  for (int c = 0; c < kClasses; c++) {
    if (class_launches) class_launches[c] = S->class_launches[c];
    if (class_items) class_items[c] = S->class_items[c];
  }
  return MPDIV_OK;
}

extern "C" int mpdiv_debug_serve_fail_launch(mpdiv_ctx* ctx, int64_t launch_index) {
  if (!ctx || launch_index < -1) return MPDIV_EINVAL;
  MpServer* S = ctx->server;
  if (!S) return mpdiv_set_error(ctx, MPDIV_ESTATE, "server not running");
  std::lock_guard<std::mutex> g(S->mu);
  S->fail_launch = launch_index;
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
    if (s.copied) cudaEventDestroy(s.copied);
    if (s.stream) cudaStreamDestroy(s.stream);
    if (s.h_meta) cudaFreeHost(s.h_meta);
    if (s.d_meta) cudaFree(s.d_meta);
  }
  if (S->by_ticket)
    for (uint64_t i = 0; i <= S->ticket_mask; i++) delete S->by_ticket[i].exchange(nullptr);
  if (S->copy_stream) {
    cudaStreamSynchronize(S->copy_stream);
    cudaStreamDestroy(S->copy_stream);
  }
  cudaFree(S->d_in);
  cudaFree(S->d_out);
  if (S->h_in) cudaFreeHost(S->h_in);
  if (S->h_out) cudaFreeHost(S->h_out);
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
  std::atomic<int64_t> rej{0};
  std::atomic<int> err{MPDIV_OK};
  const int64_t t0 = now_ns();
  // several submitter threads (request i goes to thread i mod kSub) so that
  // the offered rate is not capped by one thread's operand copies
  constexpr int kSub = 4;
  std::vector<std::atomic<int64_t>> sub_next(kSub);
  for (auto& x : sub_next) x.store(0);
  auto submitter_fn = [&](int tid) {
    for (int64_t i = tid; i < n; i += kSub) {
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
          int expect = MPDIV_OK;
          err.compare_exchange_strong(expect, rc);
          tickets[i] = 0;
          break;
        }
        rej++;
        std::this_thread::sleep_for(std::chrono::microseconds(20));
      }
      sub_next[tid].store(i + kSub, std::memory_order_release);
    }
  };
  std::vector<std::thread> submitters;
  for (int t = 0; t < kSub; t++) submitters.emplace_back(submitter_fn, t);
  // several pollers too (request i is polled by thread i mod kPoll); each
  // copies its results straight from the server's pinned output ring
  constexpr int kPoll = 4;
  auto poller_fn = [&](int tid) {
    for (int64_t i = tid; i < n; i += kPoll) {
      while (sub_next[i % kSub].load(std::memory_order_acquire) <= i)
        std::this_thread::sleep_for(std::chrono::microseconds(5));
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
      if (rc != MPDIV_OK) {
        int expect = MPDIV_OK;
        err.compare_exchange_strong(expect, rc);
        status[i] = -1;
        latency_ns[i] = -1;
        continue;
      }
      latency_ns[i] = td - t_arr[i];
    }
  };
  std::vector<std::thread> pollers;
  for (int t = 0; t < kPoll; t++) pollers.emplace_back(poller_fn, t);
  for (auto& th : pollers) th.join();
  for (auto& th : submitters) th.join();
  if (rejected) *rejected = rej.load();
  return err.load();
}

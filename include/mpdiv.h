/* mpdiv -- batched exact division of midsize unsigned integers on GB300 (sm_103a).
 *
 * Each division computes (q, r) with u = q*v + r and 0 <= r < v by the
 * whole-shifted-inverse method of arXiv 2606.06386: the shifted inverse
 * shinv_h(v) = floor(B^h / v) (Definition 1, B = 2^32, h = prec(u)) is refined
 * by an all-integer Newton iteration (Algorithm 1 with PowDiff, Algorithm 2),
 * the quotient is shift_{-h}(u * shinv_h(v)), and one-step corrections
 * (Algorithm 3, Theorem 2) make the remainder exact. One thread block runs one
 * division; operands and intermediates live in shared memory.
 *
 * Conventions for every entry point below:
 *  - Integers are little-endian arrays of uint32 digits. Digit counts may
 *    include leading zero digits; effective precisions are found on the device.
 *  - "Device" pointers are CUDA global-memory pointers of the context's device
 *    (for instance the data pointers of torch tensors); the caller owns them and
 *    they must stay valid until the work on `stream` completes. The library
 *    never frees caller memory.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream). Calls are asynchronous; results are valid after the stream is
 *    synchronised.
 *  - Sizes: 1 <= u_limbs, v_limbs <= MPDIV_MAX_LIMBS (16384 digits = 2^19 bits;
 *    dividends of more than 8192 digits need the default clipped products: with
 *    MPDIV_FLAG_FULL_PRODUCTS their working set exceeds a block's shared memory
 *    and the call returns MPDIV_EUNSUPPORTED).
 *    q_limbs >= 1 and r_limbs >= v_limbs. A quotient needs at most
 *    u_limbs - prec(v) + 1 digits; with q_limbs = u_limbs every quotient fits.
 *  - Return codes: MPDIV_OK (0) or a negative MPDIV_E* code; the text of the
 *    last error of a context is available from mpdiv_last_error().
 *  - Per-item status (int32 array, device): MPDIV_ST_*.
 */
#ifndef MPDIV_H
#define MPDIV_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MPDIV_MAX_LIMBS 16384

/* return codes */
#define MPDIV_OK 0
#define MPDIV_PENDING 1
#define MPDIV_EINVAL (-1)
#define MPDIV_EUNSUPPORTED (-2)
#define MPDIV_ENOMEM (-3)
#define MPDIV_ECUDA (-4)
#define MPDIV_EBUSY (-5)
#define MPDIV_ETIMEDOUT (-6)
#define MPDIV_ESTATE (-7)

/* per-item status */
#define MPDIV_ST_OK 0
#define MPDIV_ST_DIV_BY_ZERO 1          /* v == 0: q and r are written as zero */
#define MPDIV_ST_CORRECTION_OVERFLOW 2  /* more corrections than the bound (2 each way with full
                                           products, 4 with clipped ones) */
#define MPDIV_ST_Q_OVERFLOW 3           /* the quotient does not fit in q_limbs (low digits written) */
#define MPDIV_ST_INTERNAL 4             /* an internal working-buffer bound was exceeded */

/* flags of mpdiv_config.flags */
#define MPDIV_FLAG_INJECT_LAMBDA 1 /* test only: use shinv + 1, forcing Theorem 2's delta = -1 path */
#define MPDIV_FLAG_FULL_PRODUCTS 2 /* Algorithms 1-3 with the paper's full products w*x in Step,
                                      u*shinv and v*q (default: clipped products, Section 5: Step's
                                      w*x from the columns at or above the dropped ones less two,
                                      PowDiff's close product from the columns that can move the
                                      Step result by a unit or more, the quotient from the
                                      columns at or above h-2 of u*shinv,
                                      the remainder from v*q mod B^(prec(v)+1); same q and r,
                                      fewer products; the shifted inverse itself can then differ
                                      from Algorithm 1's by one unit) */
#define MPDIV_FLAG_NTT_PRODUCTS 4  /* full products (implies MPDIV_FLAG_FULL_PRODUCTS) by a
                                      number-theoretic transform over three primes where the
                                      block's spare shared memory holds it (transforms of up to
                                      8192 points, four words per point), the strip product
                                      elsewhere: the FFT multiplication the paper names for larger
                                      sizes (Section 6); same digits, fewer instructions for
                                      long operands */

#define MPDIV_FLAG_PERSISTENT_QUEUE 8 /* ragged batches and serving run the self-splitting
                                         persistent kernel over one size-sorted queue (blocks
                                         split into halves and quarters for smaller items);
                                         default: one plain launch per size class of the
                                         batch, each with that class's tuned shape over its
                                         items in cost order, the launches forked as
                                         branches of one CUDA graph. Same q and r. */

typedef struct mpdiv_ctx mpdiv_ctx; /* opaque; owned by the library */

typedef struct mpdiv_config {
  int warps_per_block; /* 0: per size class from the tuning table (mpdiv_autotune) */
  int blocks_per_sm;   /* persistent kernels: resident blocks per SM; 0: from occupancy */
  int flags;           /* MPDIV_FLAG_* */
  int mul_columns;     /* output columns per lane of the strip multiply: 3, 5 or 7; 0: per
                          size class from the tuning table */
  int karatsuba_cutoff; /* one Karatsuba level for the Newton step's full products (only with
                           MPDIV_FLAG_FULL_PRODUCTS) whose shorter operand has at least this
                           many digits (> 0); -1: never; 0: per size class from the tuning
                           table (never if untuned) */
  int transform_cutoff; /* with MPDIV_FLAG_NTT_PRODUCTS: products whose operands have at least
                           this many digits together use the transform (0: 4096) */
  int registers;        /* registers per thread of the plain kernel: 64, or 128 (block sizes of
                           4, 8 and 16 warps, which have such a build); 0: per size class
                           from the tuning table, else 64 */
} mpdiv_config;

/* Create a context on CUDA device `device` (cfg may be NULL for defaults).
 * The context owns its device workspace, queue buffers, captured CUDA graphs,
 * tuning table and serving pools. Returns MPDIV_OK or MPDIV_ECUDA/EINVAL. */
int mpdiv_init(mpdiv_ctx **ctx, int device, const mpdiv_config *cfg);

/* Release everything the context owns (stops a running server first). */
void mpdiv_destroy(mpdiv_ctx *ctx);

/* Text of the last error recorded on ctx ("" if none). Valid until the next call. */
const char *mpdiv_last_error(const mpdiv_ctx *ctx);

/* Uniform batch, the plain launch (one thread block per division; Section 3 of
 * the paper): item i reads u + i*u_stride (u_limbs digits) and v + i*v_stride
 * (v_limbs digits), writes q + i*q_stride (q_limbs digits, zero-padded),
 * r + i*r_stride (r_limbs digits, zero-padded) and status[i]. iters may be NULL;
 * otherwise iters[i] gets the number of Newton (Refine) iterations run.
 * products may be NULL; otherwise products[i] gets the digit products of the
 * multiplications of Algorithms 1-3 for item i at their operand precisions
 * (a close product modulo B^L counts only the digit pairs below L): the unit
 * of the paper's multiplication cost model (Section 2.3).
 * Strides are in digits. All pointers are device pointers.
 * Errors: MPDIV_EINVAL (null pointer, non-positive size, r_limbs < v_limbs,
 * stride shorter than the digit count), MPDIV_EUNSUPPORTED (more than
 * MPDIV_MAX_LIMBS digits, or a working set beyond the device's shared memory
 * per block), MPDIV_ECUDA (launch failure). */
int mpdiv_batch(mpdiv_ctx *ctx, int64_t n_items, const uint32_t *u, int32_t u_limbs, int64_t u_stride,
                const uint32_t *v, int32_t v_limbs, int64_t v_stride, uint32_t *q, int32_t q_limbs,
                int64_t q_stride, uint32_t *r, int32_t r_limbs, int64_t r_stride, int32_t *status, int32_t *iters,
                int64_t *products, void *stream);

/* Ragged batch of mixed precisions in one call. By default the items are
 * grouped by the size class of their dividend (at most 1024, 2048, 4096, 8192
 * digits, more), ordered most expensive first within each class, and each
 * class runs as one plain launch with that class's tuned shape; the class
 * launches are independent branches of one CUDA graph, so that the blocks of
 * one class fill the last wave of another. With MPDIV_FLAG_PERSISTENT_QUEUE
 * the batch is one launch of the self-splitting persistent kernel, whose
 * resident blocks take items largest-first from a size-sorted queue. Item i reads
 * u + u_off[i] (u_len[i] digits), v + v_off[i] (v_len[i] digits) and writes
 * q + q_off[i] (q_len[i] digits), r + r_off[i] (r_len[i] digits), status[i],
 * iters[i] and products[i] (each may be NULL). Offsets are in digits. u_off..r_len and status
 * are device arrays; the host-side copies of u_len and v_len (u_len_host,
 * v_len_host, n_items entries each) are used to size and order the work.
 * Requirements as for mpdiv_batch, per item (r_len[i] >= v_len[i]).
 * When the same shape list is submitted again (both length lists equal entry
 * for entry), the launch replays a captured CUDA graph. The context's queue
 * head and order array serve every call: the calls of one context run on the
 * GPU one after another, whatever their streams, and a call with a new shape
 * list first waits on the host for the previous call's launch to finish. */
int mpdiv_batch_ragged(mpdiv_ctx *ctx, int64_t n_items, const uint32_t *u, const int64_t *u_off,
                       const int32_t *u_len, const uint32_t *v, const int64_t *v_off, const int32_t *v_len,
                       uint32_t *q, const int64_t *q_off, const int32_t *q_len, uint32_t *r, const int64_t *r_off,
                       const int32_t *r_len, int32_t *status, int32_t *iters, int64_t *products,
                       const int32_t *u_len_host, const int32_t *v_len_host, void *stream);

/* Kernel launches mpdiv_batch makes for n_items items of u_limbs and v_limbs
 * digits on this context: 1, or 2 when the launch is split into a fit pass
 * (shared memory for the batch's own digit counts, so that more blocks share
 * an SM) and a retry pass (the items whose effective lengths need more). A
 * negative error code for shapes mpdiv_batch would refuse. */
int mpdiv_batch_launches(mpdiv_ctx *ctx, int64_t n_items, int32_t u_limbs, int32_t v_limbs);

/* Test entry: the shifted inverse of Algorithm 1 for each item, as the
 * division path computes it (16-warp blocks; the context's strip width, 5 if
 * unset, and its MPDIV_FLAG_FULL_PRODUCTS flag): out + i*out_stride gets
 * shinv_h(v_i) (out_limbs digits, zero-padded) with h = h_digits[i] (device
 * int32 array), iters[i] the Refine iteration count. With full products the
 * value is floor(B^h/v) or one more (Theorem 2); with the default clipped
 * Newton steps it can differ from that by one more unit either way. Requires
 * v_i != 0 and h_i >= prec(v_i); otherwise status[i] is set. */
int mpdiv_debug_shinv(mpdiv_ctx *ctx, int64_t n_items, const uint32_t *v, int32_t v_limbs, int64_t v_stride,
                      const int32_t *h_digits, uint32_t *out, int32_t out_limbs, int64_t out_stride,
                      int32_t *iters, int32_t *status, void *stream);

/* Test entry: one block-group primitive of the division path per item, on
 * item i's x (x + i*nx, nx digits) and y (y + i*ny, ny digits), with the
 * result digits at out + i*cap (cap >= 1; 3 for op 7) and an int32 at result[i]:
 *   op 0: out = (x + y) mod B^cap, result = carry out of digit cap-1
 *   op 1: out = (x - y) mod B^cap, result = borrow out
 *   op 2: result = -1, 0, 1 as x <, ==, > y
 *   op 3: result = prec(x), the significant digits of x
 *   op 4: out = x - B^arg (cap digits), result = 0 if x < B^arg (then out is x)
 *   op 5: out = x + B^arg mod B^cap, result = 0 on a carry out of cap
 *   op 6: out[arg..cap) = digits arg.. of the sum of the digit products
 *         x_i y_j B^(i+j) with i + j >= arg, mod B^cap (the clipped product;
 *         arg = 0: x y mod B^cap); out below arg is zero; result = arg
 *   op 7: out[0..3) = lowest nonzero digit, highest nonzero digit, highest
 *         digit that is not all ones of x (-1 where there is none)
 *   op 8: out = B^cap - x (x nonzero below cap)
 *   op 9: out[arg..cap) = digits arg.. of x y mod B^cap by the number-theoretic
 *         transform (MPDIV_FLAG_NTT_PRODUCTS), exact (the carries of the
 *         digits below arg included); out below arg is zero; result = arg;
 *         nx + ny <= 8192 (else MPDIV_EUNSUPPORTED)
 * with `warps` warps per block (rounded up to 1, 2, 4, 8, 16 or 32) and the
 * context's strip width (3 if unset). Device pointers; asynchronous. */
int mpdiv_debug_primitive(mpdiv_ctx *ctx, int32_t op, int64_t n_items, const uint32_t *x, int32_t nx,
                          const uint32_t *y, int32_t ny, int32_t arg, uint32_t *out, int32_t cap, int32_t *result,
                          int32_t warps, void *stream);

/* Tuning: time the plain kernel for the given (u_limbs, v_limbs) shape at each
 * candidate block size (1 and 2 warps for u_limbs <= 1024, then 4, 8, 16 and
 * 32 warps) and strip width (3, 5, 7 columns
 * per lane), then at Karatsuba cutoffs (never, 2048, 1024, 512 digits), on
 * `n_items` synthetic divisions and keep the fastest in the context's tuning
 * table for that size class (used where cfg leaves the
 * choice open). Returns the chosen warps per block (> 0) or a negative error
 * code. Synchronous. */
int mpdiv_autotune(mpdiv_ctx *ctx, int32_t u_limbs, int32_t v_limbs, int32_t n_items);

/* The launch shape the context uses for dividends of u_limbs digits: warps per
 * block, output columns per lane of the strip multiply, the Karatsuba cutoff
 * (0: never) and the registers per thread of the plain kernel (64 or 128;
 * 0: untuned, which runs 64), tuned, configured or default. Any pointer may be
 * NULL. */
int mpdiv_tuning(mpdiv_ctx *ctx, int32_t u_limbs, int32_t *warps, int32_t *mul_columns,
                 int32_t *karatsuba_cutoff, int32_t *regs);

/* Microbenchmark of the integer multiply pipe, the measured ceilings of the
 * roofline: kind 0 runs the strip multiply's digit product (mad.lo.cc /
 * madc.hi.cc / addc into independent in-register three-word accumulators)
 * and kind 1 independent 32-bit multiply-adds, with eight 256-thread blocks
 * per SM for `iters` rounds (0: 4096); kind 2 runs the strip multiply's inner
 * loop itself (5 columns per lane, the window digits and the row digits read
 * from shared memory) with two 256-thread blocks per SM, as the largest
 * divisions run, for `iters` passes over 4200 rows (0: 8). *rate gets digit
 * products (kinds 0 and 2) or multiply-adds (kind 1) per second over all SMs,
 * *ms the kernel time (CUDA events, after one warm-up launch). Synchronous;
 * uses a stream of its own. Errors: MPDIV_EINVAL (kind not 0, 1 or 2,
 * iters < 0, null pointer), MPDIV_ENOMEM, MPDIV_ECUDA. */
int mpdiv_measure_peak(mpdiv_ctx *ctx, int32_t kind, int32_t iters, double *rate, double *ms);

/* The cost unit of the paper's multiplication count (Section 2.3, Fig. 3 and
 * Table 1's "Our Mul"): out + i*out_stride gets (u_i * v_i) mod B^n, the
 * product of two n-digit numbers kept to n digits (the digit pairs below n),
 * one thread block per item, with the division path's strip multiply (with
 * MPDIV_FLAG_NTT_PRODUCTS, by the number-theoretic transform when 2 n_limbs is
 * at most 8192 and at least the transform cutoff). u_i, v_i at u + i*stride,
 * v + i*stride; all device pointers. Asynchronous on stream.
 * n_limbs <= 2 * MPDIV_MAX_LIMBS. */
int mpdiv_mul_batch(mpdiv_ctx *ctx, int64_t n_items, const uint32_t *u, const uint32_t *v, int32_t n_limbs,
                    int64_t stride, uint32_t *out, int64_t out_stride, void *stream);

/* ---------------------------------------------------------------- serving
 * Continuous batching: submitted requests are copied into a pinned input ring
 * that is mapped into the GPU's address space; a host scheduler thread
 * launches batches of them as slots free up, with several batches in flight
 * on separate streams; the kernels read the operands from the input ring and
 * write the results into a pinned, mapped output ring directly (host memory
 * over the CPU-GPU link: a batch makes no copy), and each batch's completion
 * publishes its results. With MPDIV_SERVE_DEVICE_POOLS the operands live in a
 * device-resident pool (HBM) instead, and each batch copies its operands in
 * before its launch; the results still go to the mapped output ring. Requests
 * that arrive while batches run
 * join the next launch. Admission is by footprint: a request's footprint
 * class is the size class of its dividend (class 0: at most 1024 digits,
 * 1: 2048, 2: 4096, 3: 8192, 4: more), which sets the shared memory and block
 * shape its division needs; each class has its own queue, and a batch holds
 * requests of one class only, so that a large request never sets the launch
 * shape of small ones. Batches of different classes run at once. */
#define MPDIV_SERVE_CLASSES 5
#define MPDIV_SERVE_DEVICE_POOLS 1 /* serve_config.flags: operands in a device pool (HBM) */
typedef struct mpdiv_serve_config {
  int64_t pool_digits;  /* digits of the operand and result rings, half each, on the host
                           (pinned); with MPDIV_SERVE_DEVICE_POOLS the operand half on the
                           device too (0: 64 Mi digits) */
  int32_t max_batch;    /* most requests per batch (0: 4096) */
  int32_t max_inflight; /* batches in flight at once, each on its own stream (0: 64) */
  int32_t max_pending;  /* submitted-but-unfinished requests before EBUSY (0: 1<<20) */
  int32_t low_water;    /* below this many requests on the GPU, queued requests launch as
                           soon as there are batch_step of them per batch in flight; above it
                           they gather into larger batches (0: 2048) */
  int32_t max_wait_us;  /* longest a queued request waits for its batch to grow (0: 2000) */
  int32_t batch_step;   /* below low_water, a class's queued requests launch once there are this
                           many per batch of that class in flight (0: 32) */
  int32_t flags;        /* MPDIV_SERVE_* */
} mpdiv_serve_config;

/* Start the server on ctx (cfg may be NULL). MPDIV_ESTATE if one is running.
 * Starting again after mpdiv_serve_stop releases the stopped server first, and
 * with it the results of tickets that were never polled. */
int mpdiv_serve_start(mpdiv_ctx *ctx, const mpdiv_serve_config *cfg);

/* Submit one division from host memory; the operands are copied before the
 * call returns. *ticket identifies the request. MPDIV_EBUSY when the request
 * would exceed max_pending, finds the pool full (retry later) or can never
 * fit it, or when the ticket 2*max_pending (rounded up to a power of two)
 * before it has not been polled yet; MPDIV_EUNSUPPORTED for
 * sizes beyond MPDIV_MAX_LIMBS; MPDIV_ECUDA once a batch has failed to launch
 * (the server then refuses work until it is stopped). Thread-safe. */
int mpdiv_serve_submit(mpdiv_ctx *ctx, const uint32_t *u_host, int32_t u_len, const uint32_t *v_host,
                       int32_t v_len, uint64_t *ticket);

/* Poll a ticket: MPDIV_PENDING while it is queued or running; MPDIV_OK once
 * done, after copying q (q_cap digits, zero-padded; q_cap >= u_len - prec(v) + 1
 * always suffices) and r (r_cap >= v_len digits) to host memory and the item
 * status to *status. A finished ticket can be polled once; afterwards it is
 * MPDIV_EINVAL. Thread-safe; a finished ticket is collected without the
 * server's lock. timeout_us > 0 waits up to that long for completion
 * (MPDIV_ETIMEDOUT after); 0 returns at once. A request whose batch failed to
 * launch, or that was still queued when a batch failed, finishes with status
 * MPDIV_ST_INTERNAL and zero digits: its poll collects it and returns
 * MPDIV_ECUDA. */
int mpdiv_serve_poll(mpdiv_ctx *ctx, uint64_t ticket, uint32_t *q_host, int32_t q_cap, uint32_t *r_host,
                     int32_t r_cap, int32_t *status, int64_t timeout_us);

/* Stop admitting, finish every admitted request, stop the scheduler. Results
 * of finished tickets stay pollable until mpdiv_destroy. */
int mpdiv_serve_stop(mpdiv_ctx *ctx);

/* Counters of the server: completed requests, launches, and the sum of
 * requests per launch (for the mean batch size); per footprint class of a
 * launch (the class of its largest dividend; MPDIV_SERVE_CLASSES entries
 * each), the launches and their requests. Any pointer may be NULL. */
int mpdiv_serve_stats(mpdiv_ctx *ctx, int64_t *completed, int64_t *launches, int64_t *batched_items,
                      int64_t *class_launches, int64_t *class_items);

/* Test entry: the server's launch with index launch_index (0 for the first
 * launch since mpdiv_serve_start; -1: none) fails on the host, before any of
 * its copies or kernels reach the GPU, as a failed launch would. This drives
 * the failure path (failed requests, MPDIV_ECUDA from poll and submit) without
 * a GPU fault. MPDIV_ESTATE if no server runs. */
int mpdiv_debug_serve_fail_launch(mpdiv_ctx *ctx, int64_t launch_index);

/* Open-loop replay of an arrival stream against the running server, for
 * latency measurement: request i (operands at u + u_off[i], v + v_off[i] in
 * host memory) is submitted at t0 + arrival_ns[i] from a submitter thread;
 * latency_ns[i] is the time from that scheduled arrival until its result was
 * pollable. Results go to host arrays q + q_off[i] (q_len[i] digits) and
 * r + r_off[i] (r_len[i] digits); status[i] per item (-1 if never admitted).
 * *rejected (may be NULL) counts MPDIV_EBUSY retries. phase_ns (may be NULL;
 * 3 n entries) splits each latency into the submitter's delay past the
 * scheduled arrival, the wait in the queue until its batch launched, and the
 * time from launch until the result was pollable (-1 for a request that never
 * completed). Synchronous. */
int mpdiv_serve_replay(mpdiv_ctx *ctx, int64_t n, const int64_t *arrival_ns, const uint32_t *u,
                       const int64_t *u_off, const int32_t *u_len, const uint32_t *v, const int64_t *v_off,
                       const int32_t *v_len, uint32_t *q, const int64_t *q_off, const int32_t *q_len, uint32_t *r,
                       const int64_t *r_off, const int32_t *r_len, int32_t *status, int64_t *latency_ns,
                       int64_t *rejected, int64_t *phase_ns);

/* ---------------------------------------------------------------- allocation-free form
 * The paper has no counterpart to this entry point; it exists for callers that
 * cannot allocate device memory when they divide (a memory pool that owns the
 * whole device, an allocator that forbids cudaMalloc after start-up, an
 * embedding with a fixed memory budget). It takes the same arguments as
 * mpdiv_batch_ragged and returns the same q, r and status (iters and products
 * are not produced), but runs without a context: it calls no cudaMalloc,
 * cudaFree or other allocating routine and captures no graph. It runs the
 * one-block-per-item queue kernel (16-warp blocks, 5 columns per lane, no
 * Karatsuba, no tuned per-class shapes) over items ordered by a cost bucket,
 * not mpdiv_batch_ragged's self-splitting persistent kernel, so its results
 * are the same but its throughput is lower. Its queue head and ordered item
 * list live in a fixed scratch array in the library image, on every GPU that
 * loads the library, until the process exits.
 *  - At most MPDIV_NOALLOC_MAX_ITEMS items per call (the scratch holds one
 *    order slot per item); more returns MPDIV_EUNSUPPORTED with nothing run.
 *  - Runs on the current CUDA device: every device pointer and the stream
 *    must belong to it. The first call on a device looks up the scratch
 *    array's device address (cudaGetSymbolAddress) once; make that first call
 *    outside any stream capture.
 *  - Every call reuses the same scratch and clears what must start at zero.
 *    Calls whose work overlaps on the GPU (for example on two streams at once)
 *    race on the scratch: serialise them, for instance on one stream.
 *  - Returns MPDIV_OK, MPDIV_EINVAL (null pointer, n_items < 0, a u_len_host
 *    entry < 1), MPDIV_EUNSUPPORTED (too many items or digits) or MPDIV_ECUDA.
 * All arrays except u_len_host (host) are device arrays, as in
 * mpdiv_batch_ragged; r_len[i] >= v_len[i] >= 1 is required. */
#define MPDIV_NOALLOC_MAX_ITEMS 65536
int mpdiv_batch_ragged_noalloc(int64_t n_items, const uint32_t *u, const int64_t *u_off, const int32_t *u_len,
                               const uint32_t *v, const int64_t *v_off, const int32_t *v_len, uint32_t *q,
                               const int64_t *q_off, const int32_t *q_len, uint32_t *r, const int64_t *r_off,
                               const int32_t *r_len, int32_t *status, const int32_t *u_len_host, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* MPDIV_H */

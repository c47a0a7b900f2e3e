"""Benchmark of batched exact division of midsize integers on GB300.

Default workload (the plain per-size batched sweep): dividends of 2^15, 2^16,
2^17 and 2^18 bits (1024/2048/4096/8192 uint32 digits, top digit nonzero)
divided by divisors of half their length, batches of 8192/4096/2048/1024
uniform random operands, one plain launch (one thread block per division) per
size. One step = the four launches (15,360 divisions). Prints one JSON line.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload sweep|mixed|serve|stress|paper] [--products clipped|full|ntt]

The sweep's line also carries: per_size (mean and median launch time, digit
products, the division/multiplication time ratio), roofline (the 2^18-bit
launch against the derived multiply-pipe peak, with the pipe measured on the
same GPU in roofline.measured), e2e (through host buffers), the same
divisions as one batched persistent launch (batched_single_launch), the
CPU oracle baseline and the SM clocks seen during the timed region. At its end
it carries compact results of the other configurations, each with its clocks
(--no-configs leaves them out): mixed (8192 mixed-precision divisions, the
batched launch against one plain launch per size class), serve (200,000
Poisson arrivals at 50/80/95 % of the plain capacity, 95 % three times: p50,
p99, sustained rate) and stress (the five 2^18-bit variants: rate, Newton
iterations, nonzero statuses).

--impl reference times the CPU oracle (Knuth's Algorithm D, C++) on this
machine's host cores over a bounded sample of the same workload per step.
Other workloads: mixed (one persistent launch of 8192 mixed-precision
divisions vs one plain launch per size class), serve (Poisson arrivals at
50/80/95% of the plain path's capacity through the serving loop), stress
(2^18-bit adversarial cases), paper (the paper's own Table 1 datasets,
2^13..2^18 bits, with the division/multiplication time ratio per dataset).
Under torchrun each rank runs the workload on
its own GPU (independent replicas); the value is the total over ranks divided
by the slowest rank's time.
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2606_06386_gb300 import inputs as I  # noqa: E402

SWEEP = I.SWEEP  # (u digits, v digits, batch)
METRIC = "divisions/sec at 2^15-2^18 bits, batched vs plain launch; p99 latency; % IMAD peak"
UNIT = "div/s"
# mpdiv_config.flags per product mode: clipped (Section 5's clipped products,
# the default), the paper's full products, full products by the
# number-theoretic transform where it fits (MPDIV_FLAG_NTT_PRODUCTS)
PRODUCT_FLAGS = {"clipped": 0, "full": 2, "ntt": 6}
PERSISTENT_QUEUE = 8  # MPDIV_FLAG_PERSISTENT_QUEUE: ragged batches by the self-splitting persistent kernel
SM_COUNT_GB300 = 152
PRODUCTS_PER_CLK_SM = 32  # 64 32-bit IMAD results/clk/SM, two (lo, hi) per 32x32->64 digit product
SM_MAX_MHZ = 2070.0
# DRAM bytes per 2^18-bit division of k_div_uniform, from one ncu capture of
# that kernel (dram__bytes_read.sum + dram__bytes_write.sum = 15,427,840 +
# 1,024 bytes over a 304-division launch, 8 warps, 5 columns per lane, 64
# registers, early Refine iterations on the first warp): the operands read
# once, the results held in L2; the roofline's traffic is this times the
# launch's divisions
DRAM_BYTES_PER_DIV_2E18 = (15427840 + 1024) / 304


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f)
    return {}


# ---------------------------------------------------------------- distributed
def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return None, 0, 1, 0
    import torch.distributed as dist

    rank = int(os.environ["RANK"])
    local = int(os.environ.get("LOCAL_RANK", rank))
    backend = "nccl" if os.environ.get("MPDIV_BENCH_BACKEND", "nccl") == "nccl" else "gloo"
    dist.init_process_group(backend=backend)
    return dist, rank, ws, local


def _barrier(dist, dev):
    import torch

    torch.cuda.synchronize(dev)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize(dev)


def _max_over_ranks(dist, x: float, dev) -> float:
    if dist is None:
        return x
    import torch

    t = torch.tensor([x], dtype=torch.float64, device=dev if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        # raw samples go to $MPDIV_CLOCKS_DIR (default: the temporary directory)
        out_dir = os.environ.get("MPDIV_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out_dir, f"mpdiv_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=self.f, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None:
            return None
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
                except ValueError:
                    continue
        if not rows:
            return None
        mx = max(r[1] for r in rows)
        loaded = [r for r in rows if r[0] > 0.5 * mx] or rows
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[2]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in loaded), "sm_max_mhz": mx, "reasons": reasons,
                "samples": len(rows)}


# ---------------------------------------------------------------- CPU baseline (oracle)
def cpu_baseline(items, nthreads=0):
    """Time the oracle (Knuth D) on host cores over a list of (U, V) batches."""
    import oracle

    oracle.lib()
    n = 0
    t0 = time.perf_counter()
    used = 1
    for U, V in items:
        _, _, _, used = oracle.divmod_batch_u32(U, V, U.shape[1] - V.shape[1] + 1, V.shape[1], nthreads)
        n += U.shape[0]
    dt = time.perf_counter() - t0
    return n / dt, used, dt, n


# ---------------------------------------------------------------- workloads
def _to_dev(a, dev):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).to(dev)


def run_sweep(args, dev, dist, rank, ws):
    import torch

    import paper_2606_06386_gb300 as mp

    mp.build()
    ctx = mp.mpdiv_init(dev.index or 0, flags=PRODUCT_FLAGS[args.products])
    host = [I.sweep(n, kl, b) for n, kl, b in SWEEP]
    sizes = []
    for (n, kl, b), (U, V) in zip(SWEEP, host):
        d = dict(n=n, kl=kl, b=b, U=U, V=V, u=_to_dev(U, dev), v=_to_dev(V, dev),
                 q=torch.empty((b, n - kl + 1), dtype=torch.int32, device=dev),
                 r=torch.empty((b, kl), dtype=torch.int32, device=dev),
                 st=torch.empty((b,), dtype=torch.int32, device=dev),
                 prod=torch.zeros((b,), dtype=torch.int64, device=dev))
        sizes.append(d)
    stream = torch.cuda.current_stream(dev)
    # the tuner picks warps per block for each size class (kept in the context)
    tuned = {d["n"]: mp.mpdiv_autotune(ctx, d["n"], d["kl"], d["b"]) for d in sizes}
    # one untimed pass that also records the algorithmic digit products per item
    for d in sizes:
        mp.mpdiv_batch(ctx, d["u"], d["v"], d["q"], d["r"], d["st"], None, d["prod"], stream)
    torch.cuda.synchronize(dev)
    for d in sizes:
        d["products"] = int(d["prod"].sum().item())
        bad = int((d["st"] != 0).sum().item())
        if bad:
            raise RuntimeError(f"{bad} items of size {d['n']} returned a nonzero status")

    def step(evs=None):
        for i, d in enumerate(sizes):
            if evs is not None:
                evs[i][0].record(stream)
            mp.mpdiv_batch(ctx, d["u"], d["v"], d["q"], d["r"], d["st"], None, None, stream)
            if evs is not None:
                evs[i][1].record(stream)

    for _ in range(args.warmup):
        step()
    K = args.steps
    evs = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in sizes]
           for _ in range(K)]
    _barrier(dist, dev)
    with ClockSampler(dev.index or 0) as clk:
        t_start = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        t_start.record(stream)
        for k in range(K):
            step(evs[k])
        t_end.record(stream)
        _barrier(dist, dev)
    total_ms = t_start.elapsed_time(t_end)
    total_ms = _max_over_ranks(dist, total_ms, dev)
    per_size_ms = [statistics.mean(evs[k][i][0].elapsed_time(evs[k][i][1]) for k in range(K))
                   for i in range(len(sizes))]
    per_size_median = [statistics.median(evs[k][i][0].elapsed_time(evs[k][i][1]) for k in range(K))
                       for i in range(len(sizes))]
    items_step = sum(d["b"] for d in sizes)
    value = items_step * K * ws / (total_ms / 1e3)
    # the paper's cost unit (Table 1, "Our Mul"): the n-digit product kept to n
    # digits, same batch and block shape, for the division/multiplication ratio
    mul_ms = []
    for d in sizes:
        vv = _to_dev(I.uniform_batch(d["b"], d["n"], seed=I.SEED_BASE + 5, stream=d["n"]), dev)
        out_m = torch.empty((d["b"], d["n"]), dtype=torch.int32, device=dev)
        mp.mpdiv_mul_batch(ctx, d["u"], vv, out_m, stream)
        mul_ms.append(_time(lambda: mp.mpdiv_mul_batch(ctx, d["u"], vv, out_m, stream), stream, 5))
        del vv, out_m

    # end to end through the C ABI with host buffers: H2D inputs, launches, D2H results
    pinned = []
    for d in sizes:
        pinned.append(dict(
            u=torch.from_numpy(d["U"].view(np.int32)).pin_memory(), v=torch.from_numpy(d["V"].view(np.int32)).pin_memory(),
            q=torch.empty(tuple(d["q"].shape), dtype=torch.int32).pin_memory(),
            r=torch.empty(tuple(d["r"].shape), dtype=torch.int32).pin_memory(),
            st=torch.empty(tuple(d["st"].shape), dtype=torch.int32).pin_memory()))
    h2d = sum(p["u"].numel() * 4 + p["v"].numel() * 4 for p in pinned)
    d2h = sum(p["q"].numel() * 4 + p["r"].numel() * 4 + p["st"].numel() * 4 for p in pinned)

    # copies overlap the divisions: size i's operands go up on one copy stream
    # once the previous step's division of size i has read them, and its
    # results come down on another as soon as its division is done
    h2d_s, d2h_s = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    ev = {k: [torch.cuda.Event() for _ in sizes] for k in ("h2d", "div", "d2h")}
    for k in ev:
        for e in ev[k]:
            e.record(stream)

    def e2e_step():
        with torch.cuda.stream(h2d_s):
            for i, (d, p) in enumerate(zip(sizes, pinned)):
                h2d_s.wait_event(ev["div"][i])
                d["u"].copy_(p["u"], non_blocking=True)
                d["v"].copy_(p["v"], non_blocking=True)
                ev["h2d"][i].record(h2d_s)
        for i, (d, p) in enumerate(zip(sizes, pinned)):
            stream.wait_event(ev["h2d"][i])
            stream.wait_event(ev["d2h"][i])  # the previous step's results of size i are down
            mp.mpdiv_batch(ctx, d["u"], d["v"], d["q"], d["r"], d["st"], None, None, stream)
            ev["div"][i].record(stream)
            with torch.cuda.stream(d2h_s):
                d2h_s.wait_event(ev["div"][i])
                p["q"].copy_(d["q"], non_blocking=True)
                p["r"].copy_(d["r"], non_blocking=True)
                p["st"].copy_(d["st"], non_blocking=True)
                ev["d2h"][i].record(d2h_s)

    for _ in range(max(1, args.warmup)):
        e2e_step()
    torch.cuda.synchronize(dev)
    Ke = max(3, K // 2)
    _barrier(dist, dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    h2d_s.wait_stream(stream)  # the copies start inside the timed region
    for _ in range(Ke):
        e2e_step()
    for e in ev["d2h"]:
        stream.wait_event(e)  # the last results are on the host
    e1.record(stream)
    _barrier(dist, dev)
    e2e_ms = _max_over_ranks(dist, e0.elapsed_time(e1), dev)
    e2e_value = items_step * Ke * ws / (e2e_ms / 1e3)

    # the batched form of the same work: the step's 15,360 divisions as one
    # persistent launch over the size-sorted queue, results checked against
    # the plain launches' digits
    u_len = np.concatenate([np.full(d["b"], d["n"], np.int32) for d in sizes])
    v_len = np.concatenate([np.full(d["b"], d["kl"], np.int32) for d in sizes])
    q_len, r_len = (u_len - v_len + 1).astype(np.int32), v_len.copy()
    offs = lambda ln: np.concatenate([[0], np.cumsum(ln)[:-1]]).astype(np.int64)  # noqa: E731
    td = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
    bq = torch.zeros(int(q_len.sum()), dtype=torch.int32, device=dev)
    br = torch.zeros(int(r_len.sum()), dtype=torch.int32, device=dev)
    bst = torch.full((len(u_len),), -1, dtype=torch.int32, device=dev)
    bu = torch.cat([d["u"].reshape(-1) for d in sizes])
    bv = torch.cat([d["v"].reshape(-1) for d in sizes])
    bargs = [bu, td(offs(u_len)), td(u_len), bv, td(offs(v_len)), td(v_len), bq, td(offs(q_len)), td(q_len), br,
             td(offs(r_len)), td(r_len), bst]
    q_plain = torch.cat([d["q"].reshape(-1) for d in sizes])
    r_plain = torch.cat([d["r"].reshape(-1) for d in sizes])

    def batched_form(c):
        """(ms, same digits as the plain launches) of the step's divisions in one call on context c."""
        run = lambda: mp.mpdiv_batch_ragged(c, *bargs, None, None, torch.from_numpy(u_len),  # noqa: E731
                                            torch.from_numpy(v_len), stream)
        bq.zero_()
        br.zero_()
        bst.fill_(-1)
        run()
        torch.cuda.synchronize(dev)
        ok = int((bst != 0).sum().item()) == 0 and torch.equal(bq, q_plain) and torch.equal(br, r_plain)
        for _ in range(2):
            run()
        return _time(run, stream, K), ok

    # the default form (one plain launch per size class, forked in one graph)
    # on the sweep's tuned context; the self-splitting persistent kernel on a
    # context tuned the same way
    ms_batched, same = batched_form(ctx)
    ctx_p = mp.mpdiv_init(dev.index or 0, flags=PRODUCT_FLAGS[args.products] | PERSISTENT_QUEUE)
    for d in sizes:
        mp.mpdiv_autotune(ctx_p, d["n"], d["kl"], d["b"])
    ms_persist, same_p = batched_form(ctx_p)
    mp.mpdiv_destroy(ctx_p)
    del bu, bv, bq, br, q_plain, r_plain

    # roofline of the dominant launch (2^18-bit dividends)
    big = max(range(len(sizes)), key=lambda i: per_size_ms[i])
    prod_big = sizes[big]["products"]
    achieved = prod_big / (per_size_ms[big] / 1e3) / 1e12
    peak = SM_COUNT_GB300 * PRODUCTS_PER_CLK_SM * SM_MAX_MHZ * 1e6 / 1e12
    # the multiply pipe measured on this GPU (after the timed regions): the
    # strip multiply's digit-product idiom in registers, and plain multiply-adds
    mac3_rate, _ = mp.mpdiv_measure_peak(ctx, 0)
    imad_rate, _ = mp.mpdiv_measure_peak(ctx, 1)
    strip_rate, _ = mp.mpdiv_measure_peak(ctx, 2)
    per_size = {}
    for i, d in enumerate(sizes):
        bits = 32 * d["n"]
        per_size[f"2^{bits.bit_length() - 1}"] = {
            "div_per_s": d["b"] / (per_size_ms[i] / 1e3), "ms": per_size_ms[i], "ms_median": per_size_median[i],
            "batch": d["b"],
            "digit_products_per_div": d["products"] / d["b"],
            "cost_units_per_div": d["products"] / d["b"] / (d["n"] * (d["n"] + 1) / 2),
            "Tprod_per_s": d["products"] / (per_size_ms[i] / 1e3) / 1e12,
            "mul_ms": mul_ms[i],
            "div_over_mul": per_size_ms[i] / mul_ms[i],
            "warps_per_block": tuned[d["n"]],
            "mul_columns": mp.mpdiv_tuning(ctx, d["n"])[1],
            "karatsuba_cutoff": mp.mpdiv_tuning(ctx, d["n"])[2],
            "registers": mp.mpdiv_tuning(ctx, d["n"])[3],
        }
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": K, "warmup": args.warmup,
        "ms_per_step": total_ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u32", "data": "synthetic",
        "config": {"workload": "plain per-size sweep: 2^15/2^16/2^17/2^18-bit dividends by half-length divisors, "
                               "batches 8192/4096/2048/1024, one plain launch per size (15360 divisions per step)",
                   "l2": "no flush: each step reads ~200 MB of operands (> 129 MB L2) before any reuse",
                   "products": args.products,
                   "parallelism": f"replicas x{ws}"},
        "per_size": per_size,
        "roofline": {"bound": "alu",
                     "kernel": f"k_div_uniform, 2^{(32 * sizes[big]['n']).bit_length() - 1}-bit launch "
                               f"({sizes[big]['b']} divisions)",
                     "achieved": achieved, "peak": peak, "unit": "Tprod/s", "frac": achieved / peak,
                     "traffic": (DRAM_BYTES_PER_DIV_2E18 * sizes[big]["b"]
                                 if sizes[big]["n"] == 8192 and args.products == "clipped" else None),
                     "traffic_unit": "bytes per launch: ncu dram__bytes_read.sum + dram__bytes_write.sum of a "
                                     "304-division launch, scaled by divisions; the writes are 1 KB (q and r stay "
                                     "in L2 within the launch), the reads are the operands once",
                     "peak_basis": "derived: 152 SMs x 32 digit products/clk/SM (64 IMAD/clk/SM, lo+hi per "
                                   "32x32->64 product) x 2070 MHz max SM clock",
                     "work_basis": "algorithmic 32x32-bit digit products of Algorithms 1-3 at operand precision, "
                                   "counted by the kernel",
                     "measured": {"digit_products_Tps": mac3_rate / 1e12, "imad_Tops": imad_rate / 1e12,
                                  "frac_of_measured_idiom": achieved / (mac3_rate / 1e12),
                                  "strip_loop_Tps": strip_rate / 1e12,
                                  "frac_of_strip_loop": achieved / (strip_rate / 1e12),
                                  "basis": "mpdiv_measure_peak on this GPU: in-register mad.lo.cc/madc.hi.cc/addc "
                                           "digit products and mad.lo.u32, 8 blocks x 256 threads per SM; the strip "
                                           "multiply's inner loop (5 columns per lane, digits from shared memory), "
                                           "2 blocks x 256 threads per SM"}},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "batched_single_launch": {"div_per_s": items_step * ws / (ms_batched / 1e3), "ms": ms_batched,
                                  "over_plain": (items_step * ws / (ms_batched / 1e3)) / value,
                                  "same_digits_as_plain": same,
                                  "how": "the step's divisions in one mpdiv_batch_ragged call, replayed as one CUDA "
                                         "graph: one plain launch per size class with its tuned shape, the four "
                                         "launches forked as graph branches; timed after the plain launches",
                                  "persistent_queue": {"div_per_s": items_step * ws / (ms_persist / 1e3),
                                                       "ms": ms_persist,
                                                       "over_plain": (items_step * ws / (ms_persist / 1e3)) / value,
                                                       "same_digits_as_plain": same_p,
                                                       "how": "MPDIV_FLAG_PERSISTENT_QUEUE: one launch of the "
                                                              "self-splitting persistent kernel over the size-sorted "
                                                              "queue"}},
        "gpu_launches": sum(mp.mpdiv_batch_launches(ctx, d["b"], d["n"], d["kl"]) for d in sizes) * K,
    }
    clocks = clk.summary()
    if clocks is not None:
        out["clocks"] = clocks
    if rank == 0 and not args.no_cpu_baseline:
        sample = [(d["U"][: d["b"] // 2], d["V"][: d["b"] // 2]) for d in sizes]
        v, cores, dt, n = cpu_baseline(sample)
        # one host thread on a sixteenth of that sample
        sample1 = [(d["U"][: d["b"] // 32], d["V"][: d["b"] // 32]) for d in sizes]
        v1, _, dt1, n1 = cpu_baseline(sample1, nthreads=1)
        out["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                               "sample": f"first half of each size's batch ({n} divisions, {dt:.1f} s), "
                                         "Knuth Algorithm D in C++ on all host threads",
                               "single_thread": {"value": v1, "unit": UNIT, "cores": 1,
                                                 "sample": f"first 1/32 of each size's batch ({n1} divisions, "
                                                           f"{dt1:.1f} s)"}}
    if not args.no_configs:
        out.update(other_configs_summary(mp, ctx, dev, stream, args))
    mp.mpdiv_destroy(ctx)
    return out


def _sig(x, digits=4):
    """x rounded to a few significant digits (compact JSON)."""
    if x is None or x == 0:
        return x
    return float(f"{x:.{digits}g}")


def _clk(c):
    return None if c is None else {"sm_mhz": c["sm_mhz"], "max": c["sm_max_mhz"], "reasons": c["reasons"]}


def other_configs_summary(mp, ctx, dev, stream, args):
    """Compact results of the mixed (config 3), serving (config 4) and stress
    (config 5) workloads on the sweep's context (shapes tuned per size class),
    each with the clocks seen while it ran; appended at the end of the sweep's
    JSON line."""
    m, _, _ = measure_mixed(mp, ctx, dev, stream, max(5, args.steps // 2), 3, per_n=False)
    mixed = {"div_s": _sig(m["div_per_s"]), "plain_class_div_s": _sig(m["plain_per_size_class"]["div_per_s"]),
             "over_plain": _sig(m["batched_over_plain_class"]), "n": m["n"], "clk": _clk(m["clocks"])}
    cap, sv = measure_serve(mp, ctx, dev, stream, args.requests, args.max_batch, args.max_inflight, args.low_water,
                            repeat_top=3, batch_step=args.batch_step, max_wait_us=args.max_wait_us)
    loads = {}
    for k, x in sv.items():
        d = {"div_s": _sig(x["sustained_div_per_s"]), "p50_ms": _sig(x["p50_ms"], 3), "p99_ms": _sig(x["p99_ms"], 3),
             "ok": x["ok"], "batch": _sig(x["mean_batch"], 3),
             "p99_phase_ms": {k2: _sig(v2, 3) for k2, v2 in x["p99_phase_ms"].items()}, "clk": _clk(x["clocks"])}
        if "runs" in x:
            d["p99_ms_runs"] = [_sig(r["p99_ms"], 3) for r in x["runs"]]
            d["ok"] = min(r["ok"] for r in x["runs"])
        loads[k] = d
    serve = {"requests": args.requests, "cap_div_s": _sig(cap), "pools": "pinned host rings mapped into the GPU",
             **loads}
    # the same with operands and results in device pools (HBM), copied per batch
    _, sm_ = measure_serve(mp, ctx, dev, stream, args.requests, args.max_batch, args.max_inflight, args.low_water,
                           batch_step=args.batch_step, max_wait_us=args.max_wait_us,
                           serve_flags=mp.MPDIV_SERVE_DEVICE_POOLS)
    serve["device_pools"] = {k: {"div_s": _sig(x["sustained_div_per_s"]), "p50_ms": _sig(x["p50_ms"], 3),
                                 "p99_ms": _sig(x["p99_ms"], 3), "ok": x["ok"]} for k, x in sm_.items()}
    st, _, _, sclk = measure_stress(mp, ctx, dev, stream, 3)
    stress = {k.split("_")[0]: {"div_s": _sig(x["div_per_s"]), "it": [x["newton_iters_min"], x["newton_iters_max"]],
                                "st_nz": x["status_nonzero"]} for k, x in st.items()}
    stress["clk"] = _clk(sclk)
    return {"mixed": mixed, "serve": serve, "stress": stress}


def _ragged_setup(u_len, v_len, seed, dev):
    import torch

    u_len = np.asarray(u_len, np.int32)
    v_len = np.asarray(v_len, np.int32)
    u_flat, u_off, v_flat, v_off = I.ragged_operands(u_len, v_len, seed=seed)
    q_len, r_len = u_len.copy(), v_len.copy()
    q_off = np.concatenate([[0], np.cumsum(q_len)[:-1]]).astype(np.int64)
    r_off = np.concatenate([[0], np.cumsum(r_len)[:-1]]).astype(np.int64)
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
    n = len(u_len)
    return dict(
        n=n, u_len=u_len, v_len=v_len, u_flat=u_flat, u_off=u_off, v_flat=v_flat, v_off=v_off, q_off=q_off,
        r_off=r_off, q_len=q_len, r_len=r_len,
        args=[d(u_flat.view(np.int32)), d(u_off), d(u_len), d(v_flat.view(np.int32)), d(v_off), d(v_len),
              torch.zeros(int(q_len.sum()), dtype=torch.int32, device=dev), d(q_off), d(q_len),
              torch.zeros(int(r_len.sum()), dtype=torch.int32, device=dev), d(r_off), d(r_len),
              torch.full((n,), -1, dtype=torch.int32, device=dev)],
        u_len_host=torch.from_numpy(u_len), v_len_host=torch.from_numpy(v_len),
    )


def _class_batches(R, classes, dev, key):
    """Group a ragged set into uniform zero-padded batches, one per group key."""
    import torch

    groups = {}
    for i in range(R["n"]):
        groups.setdefault(key(int(R["u_len"][i])), []).append(i)
    out = []
    for c, idx in sorted(groups.items()):
        idx = np.array(idx)
        vw = int(R["v_len"][idx].max())
        U = np.zeros((len(idx), c), np.uint32)
        V = np.zeros((len(idx), vw), np.uint32)
        for j, i in enumerate(idx):
            U[j, : R["u_len"][i]] = R["u_flat"][R["u_off"][i] : R["u_off"][i] + R["u_len"][i]]
            V[j, : R["v_len"][i]] = R["v_flat"][R["v_off"][i] : R["v_off"][i] + R["v_len"][i]]
        out.append(dict(u=_to_dev(U, dev), v=_to_dev(V, dev),
                        q=torch.zeros((len(idx), c), dtype=torch.int32, device=dev),
                        r=torch.zeros((len(idx), vw), dtype=torch.int32, device=dev),
                        st=torch.full((len(idx),), -1, dtype=torch.int32, device=dev)))
    return out


def _time(fn, stream, reps):
    import torch

    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / reps


def measure_mixed(mp, ctx, dev, stream, steps, warmup, per_n=True):
    """Config 3: one persistent launch of 8192 mixed-precision divisions
    (size-sorted queue, replayed as a CUDA graph) against one plain launch per
    padded size class (and, with per_n, one per distinct dividend length). The
    context's shapes should be tuned per size class first."""
    import torch

    u_len, v_len = I.mixed_sizes(8192)
    R = _ragged_setup(u_len, v_len, seed=I.SEED_BASE + 2, dev=dev)
    prod = torch.zeros(R["n"], dtype=torch.int64, device=dev)
    mp.mpdiv_batch_ragged(ctx, *R["args"], None, prod, R["u_len_host"], R["v_len_host"], stream)
    torch.cuda.synchronize(dev)
    if int((R["args"][12] != 0).sum().item()):
        raise RuntimeError("nonzero status in the mixed batch")
    products = int(prod.sum().item())
    persistent = lambda: mp.mpdiv_batch_ragged(ctx, *R["args"], None, None, R["u_len_host"], R["v_len_host"],  # noqa
                                               stream)
    for _ in range(warmup):
        persistent()
    classes = _class_batches(R, None, dev, key=lambda n: 1 << max(10, (n - 1).bit_length()))

    def plain(batches):
        for b in batches:
            mp.mpdiv_batch(ctx, b["u"], b["v"], b["q"], b["r"], b["st"], None, None, stream)

    plain(classes)
    torch.cuda.synchronize(dev)
    with ClockSampler(dev.index or 0) as clk:
        ms_persist = _time(persistent, stream, steps)
        ms_class = _time(lambda: plain(classes), stream, steps)
    n = R["n"]
    res = {"n": n, "ms": ms_persist, "div_per_s": n / (ms_persist / 1e3),
           "plain_per_size_class": {"div_per_s": n / (ms_class / 1e3), "launches": len(classes), "ms": ms_class},
           "batched_over_plain_class": ms_class / ms_persist,
           "digit_products_per_div": products / n, "Tprod_per_s": products / (ms_persist / 1e3) / 1e12,
           "clocks": clk.summary()}
    if per_n:
        per_n_b = _class_batches(R, None, dev, key=lambda m: m)
        plain(per_n_b)
        ms_n = _time(lambda: plain(per_n_b), stream, 2)
        res["plain_per_distinct_n"] = {"div_per_s": n / (ms_n / 1e3), "launches": len(per_n_b), "ms": ms_n}
    return res, R, classes


def measure_serve(mp, ctx, dev, stream, n_req, max_batch, max_inflight, low_water, loads=(0.5, 0.8, 0.95),
                  repeat_top=1, batch_step=0, max_wait_us=0, serve_flags=0):
    """Config 4: Poisson arrivals of mixed-precision requests through the
    serving loop at fractions of the plain path's measured capacity (one plain
    launch per size class); the last load is run repeat_top times."""
    u_len, v_len = I.mixed_sizes(8192)
    R = _ragged_setup(u_len, v_len, seed=I.SEED_BASE + 2, dev=dev)
    classes = _class_batches(R, None, dev, key=lambda n: 1 << max(10, (n - 1).bit_length()))

    def plain():
        for b in classes:
            mp.mpdiv_batch(ctx, b["u"], b["v"], b["q"], b["r"], b["st"], None, None, stream)

    plain()
    cap = R["n"] / (_time(plain, stream, 3) / 1e3)
    pick = np.arange(n_req) % R["n"]  # request i divides mixed item i mod 8192
    ul = R["u_len"][pick].astype(np.int32)
    vl = R["v_len"][pick].astype(np.int32)
    uo = R["u_off"][pick].astype(np.int64)
    vo = R["v_off"][pick].astype(np.int64)
    qo = R["q_off"][pick].astype(np.int64)  # results of repeated items land in the same slots
    ro = R["r_off"][pick].astype(np.int64)
    res = {}
    for li, frac in enumerate(loads):
        runs = []
        for rep in range(repeat_top if li == len(loads) - 1 else 1):
            rate = frac * cap
            arr = (I.poisson_arrivals(n_req, rate, seed=I.SEED_BASE + 3 + rep, stream=int(frac * 100)) * 1e9
                   ).astype(np.int64)
            q = np.zeros(int(R["q_len"].sum()), np.uint32)
            r = np.zeros(int(R["r_len"].sum()), np.uint32)
            st = np.full(n_req, -9, np.int32)
            lat = np.zeros(n_req, np.int64)
            ph = np.zeros(3 * n_req, np.int64)
            mp.mpdiv_serve_start(ctx, pool_digits=256 << 20, max_batch=max_batch, max_inflight=max_inflight,
                                 low_water=low_water, batch_step=batch_step, max_wait_us=max_wait_us,
                                 flags=serve_flags)
            with ClockSampler(dev.index or 0) as clk:
                t0 = time.perf_counter()
                rej = mp.mpdiv_serve_replay(ctx, arr, R["u_flat"], uo, ul, R["v_flat"], vo, vl, q, qo, ul.copy(), r,
                                            ro, vl.copy(), st, lat, ph)
                wall = time.perf_counter() - t0
            completed, launches, batched = mp.mpdiv_serve_stats(ctx)
            mp.mpdiv_serve_stop(ctx)
            span = ((arr + lat).max() - arr.min()) / 1e9
            runs.append({
                "offered_div_per_s": rate, "sustained_div_per_s": n_req / span,
                "p50_ms": float(np.percentile(lat, 50)) / 1e6, "p99_ms": float(np.percentile(lat, 99)) / 1e6,
                "max_ms": float(lat.max()) / 1e6, "ok": int((st == 0).sum()), "launches": launches,
                "mean_batch": batched / max(1, launches), "busy_retries": rej, "wall_s": wall,
                "p99_phase_ms": {k: float(np.percentile(ph[j::3], 99)) / 1e6
                                 for j, k in enumerate(("submit", "queue", "run"))},
                "clocks": clk.summary()})
        out = dict(runs[0])
        if len(runs) > 1:
            out["runs"] = [{k: x[k] for k in ("sustained_div_per_s", "p50_ms", "p99_ms", "ok")} for x in runs]
            out["p99_ms_median"] = float(np.median([x["p99_ms"] for x in runs]))
        res[f"{int(frac * 100)}%"] = out
    return cap, res


def measure_stress(mp, ctx, dev, stream, reps):
    """Config 5: the five 2^18-bit adversarial variants, 1024 divisions each,
    with Newton iteration counts and statuses."""
    import torch

    res = {}
    total_items, total_ms = 0, 0.0
    with ClockSampler(dev.index or 0) as clk:
        for variant in I.STRESS_VARIANTS:
            U, V = I.stress(variant)
            u, v = _to_dev(U, dev), _to_dev(V, dev)
            n = U.shape[0]
            q = torch.zeros((n, U.shape[1]), dtype=torch.int32, device=dev)
            r = torch.zeros((n, V.shape[1]), dtype=torch.int32, device=dev)
            st = torch.full((n,), -1, dtype=torch.int32, device=dev)
            it = torch.zeros(n, dtype=torch.int32, device=dev)
            pr = torch.zeros(n, dtype=torch.int64, device=dev)
            mp.mpdiv_batch(ctx, u, v, q, r, st, it, pr, stream)
            torch.cuda.synchronize(dev)
            bad = int((st != 0).sum().item())
            ms = _time(lambda: mp.mpdiv_batch(ctx, u, v, q, r, st, None, None, stream), stream, reps)
            its = it.cpu().numpy()
            res[variant] = {"div_per_s": n / (ms / 1e3), "ms": ms, "status_nonzero": bad,
                            "newton_iters_min": int(its.min()), "newton_iters_max": int(its.max()),
                            "digit_products_per_div": float(pr.sum().item()) / n,
                            "Tprod_per_s": float(pr.sum().item()) / (ms / 1e3) / 1e12}
            total_items += n
            total_ms += ms
            del u, v, q, r, st, it, pr
    return res, total_items, total_ms, clk.summary()


def _tune_classes(mp, ctx):
    for c in (1024, 2048, 4096, 8192):  # tuned shape per size class, for both launch forms
        mp.mpdiv_autotune(ctx, c, c // 2, 1024)


def run_mixed(args, dev, dist, rank, ws):
    """One persistent launch of 8192 mixed-precision divisions (size-sorted queue,
    CUDA graph replay) against plain launches per padded size class and per
    distinct dividend length."""
    import torch

    import paper_2606_06386_gb300 as mp

    mp.build()
    ctx = mp.mpdiv_init(dev.index or 0, flags=PERSISTENT_QUEUE if args.persistent_queue else 0)
    _tune_classes(mp, ctx)
    stream = torch.cuda.current_stream(dev)
    _barrier(dist, dev)
    m, _, _ = measure_mixed(mp, ctx, dev, stream, args.steps, args.warmup)
    ms_persist = _max_over_ranks(dist, m["ms"], dev)
    n = m["n"]
    out = {
        "metric": METRIC, "value": n * ws / (ms_persist / 1e3), "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_persist, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": "mixed precisions: 8192 divisions, dividends 2^(15+3x) bits (x uniform), divisors "
                               "(0.25+0.75y) x dividend length; one persistent launch over a size-sorted queue, "
                               "replayed as a CUDA graph",
                   "l2": "inputs 113 MB, re-read each step (compute-bound: ~1 MB/ms)"},
        "plain_per_size_class": m["plain_per_size_class"],
        "plain_per_distinct_n": m["plain_per_distinct_n"],
        "batched_over_plain_class": m["batched_over_plain_class"],
        "digit_products_per_div": m["digit_products_per_div"],
        "Tprod_per_s": m["Tprod_per_s"],
        "gpu_launches": args.steps,
    }
    if m["clocks"] is not None:
        out["clocks"] = m["clocks"]
    mp.mpdiv_destroy(ctx)
    return out


def run_serve(args, dev, dist, rank, ws):
    """Poisson arrivals of mixed-precision requests through the serving loop at
    50/80/95% of the plain path's measured capacity (per-size-class launches)."""
    import torch

    import paper_2606_06386_gb300 as mp

    mp.build()
    ctx = mp.mpdiv_init(dev.index or 0, flags=PERSISTENT_QUEUE if args.persistent_queue else 0)
    _tune_classes(mp, ctx)
    stream = torch.cuda.current_stream(dev)
    cap, res = measure_serve(mp, ctx, dev, stream, args.requests, args.max_batch, args.max_inflight, args.low_water,
                             repeat_top=3, batch_step=args.batch_step, max_wait_us=args.max_wait_us,
                             serve_flags=mp.MPDIV_SERVE_DEVICE_POOLS if args.device_pools else 0)
    n_req = args.requests
    out = {
        "metric": METRIC, "value": res["95%"]["sustained_div_per_s"], "unit": UNIT, "n_gpus": ws,
        "steps": 1, "warmup": 0, "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": f"serving: {n_req} Poisson-arrival requests, sizes as the mixed batch, offered at "
                               "50/80/95% of the plain per-size-class capacity (95% three times); latency from "
                               "scheduled arrival to result pollable on the host"},
        "plain_capacity_div_per_s": cap, "loads": res,
    }
    mp.mpdiv_destroy(ctx)
    return out


def run_stress(args, dev, dist, rank, ws):
    """Adversarial cases at 2^18 bits, 1024 divisions each, with Newton iteration counts."""
    import torch

    import paper_2606_06386_gb300 as mp

    mp.build()
    ctx = mp.mpdiv_init(dev.index or 0)
    stream = torch.cuda.current_stream(dev)
    res, total_items, total_ms, clocks = measure_stress(mp, ctx, dev, stream, max(3, args.steps // 4))
    out = {
        "metric": METRIC, "value": total_items / (total_ms / 1e3), "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": "stress at 2^18-bit dividends: 1024 divisions per variant (short divisor, just over "
                               "half, all ones, 1% sparse, v = B^k - 1)"},
        "variants": res,
    }
    if clocks is not None:
        out["clocks"] = clocks
    mp.mpdiv_destroy(ctx)
    return out


# Table 1 of the paper (A100, 64-bit digits): division time / multiplication
# time per dataset, quoted as context next to the same ratio measured here.
PAPER_DIV_OVER_MUL = {13: 15.46, 14: 14.74, 15: 9.73, 16: 6.94, 17: 6.66, 18: 6.77}


def run_paper(args, dev, dist, rank, ws):
    """The paper's own datasets (Section 4): 2^13..2^18-bit u of M - 2 digits,
    v of random precision in [2, M/2] (64-bit digits), 2^32 / bits instances,
    one plain launch each, and 2^19 bits built the same way; beside each the
    cost unit (an M-digit product kept to M digits) on the same instance count."""
    import torch

    import paper_2606_06386_gb300 as mp

    mp.build()
    ctx = mp.mpdiv_init(dev.index or 0)
    stream = torch.cuda.current_stream(dev)
    sets = []
    for bits, n_items in I.PAPER_TABLE + I.BEYOND_TABLE:
        U, V, v_len = I.paper_workload(bits, n_items)
        un, vn = U.shape[1], V.shape[1]
        d = dict(bits=bits, b=n_items, un=un, vn=vn, u=_to_dev(U, dev), v=_to_dev(V, dev),
                 q=torch.empty((n_items, un), dtype=torch.int32, device=dev),
                 r=torch.empty((n_items, vn), dtype=torch.int32, device=dev),
                 st=torch.empty((n_items,), dtype=torch.int32, device=dev),
                 prod=torch.zeros((n_items,), dtype=torch.int64, device=dev))
        del U, V
        d["warps"] = mp.mpdiv_autotune(ctx, un, vn, min(n_items, 8192))
        mp.mpdiv_batch(ctx, d["u"], d["v"], d["q"], d["r"], d["st"], None, d["prod"], stream)
        torch.cuda.synchronize(dev)
        bad = int((d["st"] != 0).sum().item())
        if bad:
            raise RuntimeError(f"{bad} items of the 2^{bits.bit_length() - 1}-bit dataset returned a nonzero status")
        d["products"] = int(d["prod"].sum().item())
        sets.append(d)
    reps = max(3, args.steps // 4)
    _barrier(dist, dev)
    with ClockSampler(dev.index or 0) as clk:
        for d in sets:
            d["ms"] = _time(lambda: mp.mpdiv_batch(ctx, d["u"], d["v"], d["q"], d["r"], d["st"], None, None,
                                                   stream), stream, reps)
    res, total_items, total_ms = {}, 0, 0.0
    for d in sets:
        m32 = d["bits"] // 32
        a = _to_dev(I.uniform_batch(d["b"], m32, seed=I.SEED_BASE + 7, stream=m32), dev)
        bb = _to_dev(I.uniform_batch(d["b"], m32, seed=I.SEED_BASE + 7, stream=m32 + 1), dev)
        out_m = torch.empty((d["b"], m32), dtype=torch.int32, device=dev)
        mp.mpdiv_mul_batch(ctx, a, bb, out_m, stream)
        mul_ms = _time(lambda: mp.mpdiv_mul_batch(ctx, a, bb, out_m, stream), stream, reps)
        del a, bb, out_m
        lg = d["bits"].bit_length() - 1
        res[f"2^{lg}"] = {"instances": d["b"], "u_digits": d["un"], "v_digits_max": d["vn"],
                          "div_ms": d["ms"], "div_per_s": d["b"] / (d["ms"] / 1e3), "mul_ms": mul_ms,
                          "div_over_mul": d["ms"] / mul_ms, "paper_div_over_mul_A100": PAPER_DIV_OVER_MUL.get(lg),
                          "digit_products_per_div": d["products"] / d["b"],
                          "Tprod_per_s": d["products"] / (d["ms"] / 1e3) / 1e12,
                          "warps_per_block": d["warps"], "mul_columns": mp.mpdiv_tuning(ctx, d["un"])[1]}
        if lg in PAPER_DIV_OVER_MUL:  # the value covers the paper's datasets only
            total_items += d["b"]
            total_ms += d["ms"]
    total_ms = _max_over_ranks(dist, total_ms, dev)
    out = {
        "metric": METRIC, "value": total_items * ws / (total_ms / 1e3), "unit": UNIT, "n_gpus": ws,
        "steps": reps, "warmup": 1, "ms_per_step": total_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": "the paper's Table 1 datasets: 2^13..2^18-bit dividends of M-2 64-bit digits, "
                               "divisors of random precision in [2, M/2] 64-bit digits, 2^32/bits instances, "
                               "one plain launch per dataset (the value covers these); 2^19 bits (2^13 instances) "
                               "built the same way is reported beside them, beyond the paper's table",
                   "l2": "no flush: every dataset's operands exceed the 129 MB L2"},
        "datasets": res,
    }
    clocks = clk.summary()
    if clocks is not None:
        out["clocks"] = clocks
    mp.mpdiv_destroy(ctx)
    return out


def run_reference(args, rank, ws):
    """The reference arm: the CPU oracle on this machine's host cores."""
    out_sample = []
    for n, kl, b in SWEEP:
        U, V = I.sweep(n, kl, b)
        m = max(1, b // 16)
        out_sample.append((U[:m], V[:m]))
    n_step = sum(U.shape[0] for U, _ in out_sample)
    for _ in range(args.warmup):
        cpu_baseline([(U[:1], V[:1]) for U, V in out_sample])
    t0 = time.perf_counter()
    used = 1
    for _ in range(args.steps):
        v, used, dt, n = cpu_baseline(out_sample)
    total = time.perf_counter() - t0
    value = n_step * args.steps / total
    sample = (f"1/16 of each size's batch per step ({n_step} divisions: "
              + ", ".join(f"{U.shape[0]}x{U.shape[1]}/{V.shape[1]} digits" for U, V in out_sample) + ")")
    return {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u32", "data": "synthetic", "impl": "reference",
        "config": {"workload": "plain per-size sweep (sampled): 2^15..2^18-bit dividends by half-length divisors"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": used, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=25)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="sweep", choices=["sweep", "mixed", "serve", "stress", "paper"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-configs", action="store_true", help="sweep workload: leave out the mixed, serving and "
                    "stress summaries at the end of the line")
    ap.add_argument("--products", default="clipped", choices=sorted(PRODUCT_FLAGS),
                    help="sweep workload: clipped products (default), the paper's full products, or full "
                    "products by the number-theoretic transform where it fits")
    ap.add_argument("--requests", type=int, default=200000, help="serve workload: number of requests")
    ap.add_argument("--max-batch", type=int, default=1024, help="serve workload: most requests per batch")
    ap.add_argument("--max-inflight", type=int, default=0, help="serve workload: batches in flight (0: the "
                    "server's default)")
    ap.add_argument("--low-water", type=int, default=2048, help="serve workload: requests on the GPU below "
                    "which queued requests launch at once")
    ap.add_argument("--batch-step", type=int, default=0, help="serve workload: queued requests of a class per "
                    "batch of that class in flight before a launch, below the low-water mark (0: 8)")
    ap.add_argument("--max-wait-us", type=int, default=0, help="serve workload: longest wait of a queued request "
                    "for its batch to grow (0: 2000)")
    ap.add_argument("--device-pools", action="store_true", help="serve workload: operands and results in device "
                    "pools copied per batch (MPDIV_SERVE_DEVICE_POOLS) instead of the mapped host rings")
    ap.add_argument("--persistent-queue", action="store_true", help="mixed and serve workloads: ragged batches by "
                    "the self-splitting persistent kernel (MPDIV_FLAG_PERSISTENT_QUEUE) instead of one plain launch "
                    "per size class")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    ws_env = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        rank = int(os.environ.get("RANK", "0"))
        if rank != 0:
            return
        print(json.dumps(run_reference(args, rank, ws_env)))
        return
    import torch

    dist, rank, ws, local = _dist()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    runner = {"sweep": run_sweep, "mixed": run_mixed, "serve": run_serve, "stress": run_stress,
              "paper": run_paper}[args.workload]
    out = runner(args, dev, dist, rank, ws)
    if rank == 0:
        print(json.dumps(out))
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

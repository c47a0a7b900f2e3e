"""mpdiv: batched exact division of midsize integers on GB300 (sm_103a).

A thin ctypes binding over the C ABI declared in include/mpdiv.h. Each
function here has the name of the C entry point it calls and only marshals
arguments: torch tensors (device memory) become pointers, a torch stream
becomes a cudaStream_t. Every step of the division runs in the CUDA kernels of
``csrc/``; there is no CPU fallback, and calling into the library without the
built extension raises ``RuntimeError``.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

_HERE = os.path.dirname(os.path.abspath(__file__))
_ROOT = os.path.dirname(_HERE)
_CSRC = os.path.join(_HERE, "csrc")
_BUILD = os.path.join(_HERE, "_build")
SO_PATH = os.path.join(_BUILD, "libmpdiv.so")
HEADER = os.path.join(_ROOT, "include", "mpdiv.h")
SOURCES = ["mpdiv_p.cu", "mpdiv_p16.cu", "mpdiv_q.cu", "mpdiv_t.cu", "mpdiv_k1.cu", "mpdiv_k2.cu", "mpdiv_k4.cu", "mpdiv_k8.cu", "mpdiv_k16.cu",
           "mpdiv_k4r.cu", "mpdiv_k8r.cu", "mpdiv_k16r.cu",
           "mpdiv_l1.cu", "mpdiv_l2.cu", "mpdiv_l4.cu", "mpdiv_l8.cu", "mpdiv_l16.cu", "mpdiv_l32.cu",
           "mpdiv_k32.cu", "mpdiv_n.cu", "mpdiv_n8.cu", "mpdiv_n16.cu", "mpdiv_n32.cu",
           "mpdiv_n2.cu", "mpdiv_n3.cu", "mpdiv_noalloc.cu", "mpdiv.cu", "mpdiv_tune.cu", "mpdiv_serve.cu"]
ARCH = "-gencode=arch=compute_103a,code=sm_103a"

# return codes and statuses (include/mpdiv.h)
MPDIV_OK, MPDIV_PENDING = 0, 1
MPDIV_EINVAL, MPDIV_EUNSUPPORTED, MPDIV_ENOMEM, MPDIV_ECUDA = -1, -2, -3, -4
MPDIV_EBUSY, MPDIV_ETIMEDOUT, MPDIV_ESTATE = -5, -6, -7
MPDIV_ST_OK, MPDIV_ST_DIV_BY_ZERO, MPDIV_ST_CORRECTION_OVERFLOW = 0, 1, 2
MPDIV_ST_Q_OVERFLOW, MPDIV_ST_INTERNAL = 3, 4
MPDIV_FLAG_INJECT_LAMBDA = 1
MPDIV_FLAG_FULL_PRODUCTS = 2
MPDIV_FLAG_NTT_PRODUCTS = 4
MPDIV_FLAG_PERSISTENT_QUEUE = 8
MPDIV_SERVE_DEVICE_POOLS = 1
MPDIV_MAX_LIMBS = 16384
MPDIV_NOALLOC_MAX_ITEMS = 65536
MPDIV_SERVE_CLASSES = 5

_lock = threading.Lock()
_lib = None


def _nvcc() -> str:
    for c in ("/usr/local/cuda/bin/nvcc", "nvcc"):
        if os.path.sep not in c or os.path.exists(c):
            return c
    return "nvcc"


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile csrc/*.cu for sm_103a into _build/libmpdiv.so (in-tree)."""
    os.makedirs(_BUILD, exist_ok=True)
    deps = [os.path.join(_CSRC, f) for f in os.listdir(_CSRC)] + [HEADER]
    newest = max(os.path.getmtime(p) for p in deps)
    if not force and os.path.exists(SO_PATH) and os.path.getmtime(SO_PATH) >= newest:
        return SO_PATH
    flags = [ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", os.path.join(_ROOT, "include")]

    def compile_one(src):
        obj = os.path.join(_BUILD, src.replace(".cu", ".o"))
        cmd = [_nvcc(), *flags, "-c", os.path.join(_CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    with ThreadPoolExecutor(len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = SO_PATH + f".tmp{os.getpid()}"
    r = subprocess.run([_nvcc(), ARCH, "-shared", *objs, "-o", tmp], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, SO_PATH)
    return SO_PATH


class mpdiv_config(ctypes.Structure):
    _fields_ = [("warps_per_block", ctypes.c_int), ("blocks_per_sm", ctypes.c_int), ("flags", ctypes.c_int),
                ("mul_columns", ctypes.c_int), ("karatsuba_cutoff", ctypes.c_int),
                ("transform_cutoff", ctypes.c_int), ("registers", ctypes.c_int)]


class mpdiv_serve_config(ctypes.Structure):
    _fields_ = [
        ("pool_digits", ctypes.c_int64),
        ("max_batch", ctypes.c_int32),
        ("max_inflight", ctypes.c_int32),
        ("max_pending", ctypes.c_int32),
        ("low_water", ctypes.c_int32),
        ("max_wait_us", ctypes.c_int32),
        ("batch_step", ctypes.c_int32),
        ("flags", ctypes.c_int32),
    ]


_P = ctypes.c_void_p
_I32, _I64, _U64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
_SIGS = {
    "mpdiv_init": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, ctypes.POINTER(mpdiv_config)]),
    "mpdiv_destroy": (None, [_P]),
    "mpdiv_last_error": (ctypes.c_char_p, [_P]),
    "mpdiv_batch": (ctypes.c_int, [_P, _I64, _P, _I32, _I64, _P, _I32, _I64, _P, _I32, _I64, _P, _I32, _I64, _P, _P, _P, _P]),
    "mpdiv_batch_ragged": (ctypes.c_int, [_P, _I64] + [_P] * 18),
    "mpdiv_debug_shinv": (ctypes.c_int, [_P, _I64, _P, _I32, _I64, _P, _P, _I32, _I64, _P, _P, _P]),
    "mpdiv_autotune": (ctypes.c_int, [_P, _I32, _I32, _I32]),
    "mpdiv_batch_launches": (ctypes.c_int, [_P, _I64, _I32, _I32]),
    "mpdiv_debug_primitive": (ctypes.c_int, [_P, _I32, _I64, _P, _I32, _P, _I32, _I32, _P, _I32, _P, _I32, _P]),
    "mpdiv_mul_batch": (ctypes.c_int, [_P, _I64, _P, _P, _I32, _I64, _P, _I64, _P]),
    "mpdiv_measure_peak": (ctypes.c_int, [_P, _I32, _I32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    "mpdiv_tuning": (ctypes.c_int, [_P, _I32] + [ctypes.POINTER(_I32)] * 4),
    "mpdiv_serve_start": (ctypes.c_int, [_P, ctypes.POINTER(mpdiv_serve_config)]),
    "mpdiv_serve_submit": (ctypes.c_int, [_P, _P, _I32, _P, _I32, ctypes.POINTER(_U64)]),
    "mpdiv_serve_poll": (ctypes.c_int, [_P, _U64, _P, _I32, _P, _I32, ctypes.POINTER(_I32), _I64]),
    "mpdiv_serve_stop": (ctypes.c_int, [_P]),
    "mpdiv_serve_stats": (ctypes.c_int, [_P] + [ctypes.POINTER(_I64)] * 5),
    "mpdiv_debug_serve_fail_launch": (ctypes.c_int, [_P, _I64]),
    "mpdiv_batch_ragged_noalloc": (ctypes.c_int, [_I64] + [_P] * 15),
    "mpdiv_serve_replay": (
        ctypes.c_int,
        [_P, _I64, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, ctypes.POINTER(_I64), _P],
    ),
}


def lib() -> ctypes.CDLL:
    """The loaded C library; raises RuntimeError when it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(SO_PATH):
                raise RuntimeError(
                    f"the CUDA library {SO_PATH} is not built: run paper_2606_06386_gb300.build() "
                    "(nvcc with sm_103a); there is no CPU fallback"
                )
            L = ctypes.CDLL(SO_PATH)
            for name, (res, args) in _SIGS.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


class MpdivError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"mpdiv error {code}: {msg}")
        self.code = code


def _check(ctx, rc: int) -> int:
    if rc < 0:
        msg = lib().mpdiv_last_error(ctx).decode() if ctx else ""
        raise MpdivError(rc, msg)
    return rc


def _ptr(t) -> int | None:
    if t is None:
        return None
    return t.data_ptr()


def _stream(stream) -> int | None:
    if stream is None:
        import torch

        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _check_dev(*ts):
    for t in ts:
        if t is not None and (not t.is_cuda or not t.is_contiguous()):
            raise ValueError("tensors must be contiguous CUDA tensors")


def _one_device(*ts):
    """The single CUDA device that every given tensor lives on (ValueError otherwise)."""
    devs = {t.device for t in ts if t is not None}
    if len(devs) != 1:
        raise ValueError(f"tensors must all live on one CUDA device, got {sorted(str(d) for d in devs)}")
    return devs.pop()


def _host_lengths(t, n: int, name: str):
    """A contiguous CPU int32 tensor of at least n digit counts (the C side reads n of them)."""
    import torch

    if t.device.type != "cpu" or t.dtype != torch.int32 or t.numel() < n:
        raise ValueError(f"{name} must be a CPU int32 tensor with at least {n} entries")
    return t.contiguous()


# ---------------------------------------------------------------- context
def mpdiv_init(device: int = 0, warps_per_block: int = 0, blocks_per_sm: int = 0, flags: int = 0,
               mul_columns: int = 0, karatsuba_cutoff: int = 0, transform_cutoff: int = 0, registers: int = 0):
    cfg = mpdiv_config(warps_per_block, blocks_per_sm, flags, mul_columns, karatsuba_cutoff, transform_cutoff,
                       registers)
    h = _P()
    _check(None, lib().mpdiv_init(ctypes.byref(h), device, ctypes.byref(cfg)))
    return h


def mpdiv_destroy(ctx) -> None:
    lib().mpdiv_destroy(ctx)


def mpdiv_last_error(ctx) -> str:
    return lib().mpdiv_last_error(ctx).decode()


def mpdiv_batch(ctx, u, v, q, r, status, iters=None, products=None, stream=None) -> None:
    """Uniform batch: u (items, u_limbs), v (items, v_limbs), q (items, q_limbs),
    r (items, r_limbs) uint32/int32 CUDA tensors; status (and iters) int32 (items,);
    products int64 (items,)."""
    _check_dev(u, v, q, r, status, iters, products)
    n = u.shape[0]
    _check(
        ctx,
        lib().mpdiv_batch(
            ctx, n, _ptr(u), u.shape[1], u.stride(0), _ptr(v), v.shape[1], v.stride(0), _ptr(q), q.shape[1],
            q.stride(0), _ptr(r), r.shape[1], r.stride(0), _ptr(status), _ptr(iters), _ptr(products), _stream(stream),
        ),
    )


def mpdiv_batch_ragged(ctx, u, u_off, u_len, v, v_off, v_len, q, q_off, q_len, r, r_off, r_len, status,
                       iters=None, products=None, u_len_host=None, v_len_host=None, stream=None) -> None:
    """Ragged batch over flat digit tensors with per-item int64 offsets and int32
    lengths (CUDA tensors); u_len_host / v_len_host are CPU int32 tensors."""
    _check_dev(u, u_off, u_len, v, v_off, v_len, q, q_off, q_len, r, r_off, r_len, status, iters, products)
    n = u_off.shape[0]
    u_len_host = _host_lengths(u_len.cpu() if u_len_host is None else u_len_host, n, "u_len_host")
    v_len_host = _host_lengths(v_len.cpu() if v_len_host is None else v_len_host, n, "v_len_host")
    _check(
        ctx,
        lib().mpdiv_batch_ragged(
            ctx, n, _ptr(u), _ptr(u_off), _ptr(u_len), _ptr(v), _ptr(v_off), _ptr(v_len), _ptr(q), _ptr(q_off),
            _ptr(q_len), _ptr(r), _ptr(r_off), _ptr(r_len), _ptr(status), _ptr(iters), _ptr(products), _ptr(u_len_host),
            _ptr(v_len_host), _stream(stream),
        ),
    )


def mpdiv_batch_ragged_noalloc(u, u_off, u_len, v, v_off, v_len, q, q_off, q_len, r, r_off, r_len, status,
                               u_len_host=None, stream=None) -> int:
    """The allocation-free ragged launch (no context): same arrays as
    mpdiv_batch_ragged, all on one CUDA device, on which the call runs (the C
    entry point launches on the current device). Returns the C return code
    (MPDIV_OK or a negative code)."""
    import torch

    _check_dev(u, u_off, u_len, v, v_off, v_len, q, q_off, q_len, r, r_off, r_len, status)
    device = _one_device(u, u_off, u_len, v, v_off, v_len, q, q_off, q_len, r, r_off, r_len, status)
    n = u_off.shape[0]
    u_len_host = _host_lengths(u_len.cpu() if u_len_host is None else u_len_host, n, "u_len_host")
    with torch.cuda.device(device):
        s = torch.cuda.current_stream(device).cuda_stream if stream is None else _stream(stream)
        return lib().mpdiv_batch_ragged_noalloc(
            n, _ptr(u), _ptr(u_off), _ptr(u_len), _ptr(v), _ptr(v_off), _ptr(v_len), _ptr(q), _ptr(q_off),
            _ptr(q_len), _ptr(r), _ptr(r_off), _ptr(r_len), _ptr(status), _ptr(u_len_host), s,
        )


def mpdiv_debug_shinv(ctx, v, h_digits, out, iters, status, stream=None) -> None:
    _check_dev(v, h_digits, out, iters, status)
    n = v.shape[0]
    _check(
        ctx,
        lib().mpdiv_debug_shinv(
            ctx, n, _ptr(v), v.shape[1], v.stride(0), _ptr(h_digits), _ptr(out), out.shape[1], out.stride(0),
            _ptr(iters), _ptr(status), _stream(stream),
        ),
    )


def mpdiv_debug_primitive(ctx, op: int, x, y, arg: int, out, result, warps: int, stream=None) -> None:
    """Test entry: one group primitive per row of the contiguous (items, nx) and
    (items, ny) CUDA tensors x, y into out (items, cap) and result (items,)."""
    _check_dev(x, y, out, result)
    for t in (x, y, out):
        if not t.is_contiguous():
            raise ValueError("contiguous tensors expected")
    _check(ctx, lib().mpdiv_debug_primitive(ctx, op, x.shape[0], _ptr(x), x.shape[1], _ptr(y), y.shape[1], arg,
                                            _ptr(out), out.shape[1], _ptr(result), warps, _stream(stream)))


def mpdiv_mul_batch(ctx, u, v, out, stream=None) -> None:
    """out[i] = (u[i] * v[i]) mod B^n for (items, n) CUDA tensors (the cost unit)."""
    _check_dev(u, v, out)
    if u.shape != v.shape or out.shape[0] != u.shape[0] or out.shape[1] < u.shape[1]:
        raise ValueError("shape mismatch")
    _check(ctx, lib().mpdiv_mul_batch(ctx, u.shape[0], _ptr(u), _ptr(v), u.shape[1], u.stride(0), _ptr(out),
                                      out.stride(0), _stream(stream)))


def mpdiv_measure_peak(ctx, kind: int = 0, iters: int = 0):
    """(rate per second, ms) of the multiply-pipe microbenchmark: kind 0 digit
    products of the strip multiply's idiom, kind 1 32-bit multiply-adds, kind 2
    digit products of the strip multiply's inner loop on shared-memory operands."""
    rate, ms = ctypes.c_double(), ctypes.c_double()
    _check(ctx, lib().mpdiv_measure_peak(ctx, kind, iters, ctypes.byref(rate), ctypes.byref(ms)))
    return rate.value, ms.value


def mpdiv_batch_launches(ctx, n_items: int, u_limbs: int, v_limbs: int) -> int:
    """Kernel launches mpdiv_batch makes for that shape on this context (1 or 2)."""
    return _check(ctx, lib().mpdiv_batch_launches(ctx, n_items, u_limbs, v_limbs))


def mpdiv_autotune(ctx, u_limbs: int, v_limbs: int, n_items: int) -> int:
    return _check(ctx, lib().mpdiv_autotune(ctx, u_limbs, v_limbs, n_items))


def mpdiv_tuning(ctx, u_limbs: int):
    """(warps per block, columns per lane, Karatsuba cutoff, registers per
    thread) used for dividends of u_limbs digits (registers 0: untuned, 64)."""
    w, t, k, g = _I32(), _I32(), _I32(), _I32()
    _check(ctx, lib().mpdiv_tuning(ctx, u_limbs, ctypes.byref(w), ctypes.byref(t), ctypes.byref(k), ctypes.byref(g)))
    return w.value, t.value, k.value, g.value


# ---------------------------------------------------------------- serving
def mpdiv_serve_start(ctx, pool_digits: int = 0, max_batch: int = 0, max_inflight: int = 0, max_pending: int = 0,
                      low_water: int = 0, max_wait_us: int = 0, batch_step: int = 0, flags: int = 0):
    cfg = mpdiv_serve_config(pool_digits, max_batch, max_inflight, max_pending, low_water, max_wait_us, batch_step,
                             flags)
    _check(ctx, lib().mpdiv_serve_start(ctx, ctypes.byref(cfg)))


def mpdiv_serve_submit(ctx, u_host, v_host) -> int:
    """u_host, v_host: contiguous uint32 numpy arrays. Returns the ticket."""
    import numpy as np

    u_host = np.ascontiguousarray(u_host, dtype=np.uint32)
    v_host = np.ascontiguousarray(v_host, dtype=np.uint32)
    t = _U64()
    _check(ctx, lib().mpdiv_serve_submit(ctx, u_host.ctypes.data, len(u_host), v_host.ctypes.data, len(v_host),
                                         ctypes.byref(t)))
    return t.value


def mpdiv_serve_poll(ctx, ticket: int, q_cap: int, r_cap: int, timeout_us: int = 0):
    """(rc, q, r, status): rc is MPDIV_OK or MPDIV_PENDING (q, r None then)."""
    import numpy as np

    q = np.zeros(q_cap, np.uint32)
    r = np.zeros(r_cap, np.uint32)
    st = _I32()
    st.value = -1
    rc = lib().mpdiv_serve_poll(ctx, ticket, q.ctypes.data, q_cap, r.ctypes.data, r_cap, ctypes.byref(st), timeout_us)
    if rc == MPDIV_PENDING or rc == MPDIV_ETIMEDOUT:
        return rc, None, None, None
    try:
        _check(ctx, rc)
    except MpdivError as e:
        e.status = st.value  # a failed request's status (MPDIV_ST_INTERNAL), -1 if none was written
        raise
    return rc, q, r, st.value


def mpdiv_serve_stop(ctx) -> None:
    _check(ctx, lib().mpdiv_serve_stop(ctx))


def mpdiv_serve_stats(ctx, by_class: bool = False):
    """(completed, launches, batched items); with by_class also the launches and
    their requests per footprint class (two lists of MPDIV_SERVE_CLASSES)."""
    c, l, b = _I64(), _I64(), _I64()
    cl, ci = (_I64 * MPDIV_SERVE_CLASSES)(), (_I64 * MPDIV_SERVE_CLASSES)()
    _check(ctx, lib().mpdiv_serve_stats(ctx, ctypes.byref(c), ctypes.byref(l), ctypes.byref(b), cl, ci))
    if by_class:
        return c.value, l.value, b.value, list(cl), list(ci)
    return c.value, l.value, b.value


def mpdiv_debug_serve_fail_launch(ctx, launch_index: int) -> None:
    """Test entry: the server's launch with this index fails on the host (-1: none)."""
    _check(ctx, lib().mpdiv_debug_serve_fail_launch(ctx, launch_index))


def mpdiv_serve_replay(ctx, arrival_ns, u, u_off, u_len, v, v_off, v_len, q, q_off, q_len, r, r_off, r_len,
                       status, latency_ns, phase_ns=None) -> int:
    """Open-loop replay with host numpy arrays (see include/mpdiv.h). Returns EBUSY retries.
    phase_ns, if given, is an int64 array of 3 entries per request (submit delay, queue wait, run)."""
    import numpy as np

    arrs = [arrival_ns, u, u_off, u_len, v, v_off, v_len, q, q_off, q_len, r, r_off, r_len, status, latency_ns]
    for a in arrs + ([] if phase_ns is None else [phase_ns]):
        if not (isinstance(a, np.ndarray) and a.flags.c_contiguous):
            raise ValueError("replay arrays must be contiguous numpy arrays")
    if phase_ns is not None and (phase_ns.dtype != np.int64 or phase_ns.size < 3 * len(arrival_ns)):
        raise ValueError("phase_ns must be an int64 array of 3 entries per request")
    rej = _I64()
    _check(ctx, lib().mpdiv_serve_replay(ctx, len(arrival_ns), *[a.ctypes.data for a in arrs], ctypes.byref(rej),
                                         None if phase_ns is None else phase_ns.ctypes.data))
    return rej.value

"""Test oracle for batched exact division of midsize integers.

This package is test infrastructure. Only the test-suite, the smoke check and
the benchmark's CPU-baseline leg may import it; the product path never does,
and it shares no code with the CUDA path.

* ``knuthd.cpp`` -- the plain definition (q, r) = (floor(u/v), u mod v) by
  Knuth's Algorithm D on 32-bit digits, plus floor(B^h / v) (Definition 1 of
  the paper) and an independent schoolbook checker. Built on demand with g++.
* ``shinv_model.py`` -- the paper's Algorithms 1-3 restated, as printed, with
  Python's unbounded integers: the Refine loop count, the shifted inverse of
  Algorithm 1 and the digit products the algorithms make (Section 2.3's cost).

Digits are little-endian uint32 numpy arrays throughout.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SRC = os.path.join(_HERE, "knuthd.cpp")
_lock = threading.Lock()
_lib = None

U32P = ctypes.POINTER(ctypes.c_uint32)
U16P = ctypes.POINTER(ctypes.c_uint16)
U8P = ctypes.POINTER(ctypes.c_uint8)
I32P = ctypes.POINTER(ctypes.c_int32)
I64P = ctypes.POINTER(ctypes.c_int64)


def build(force: bool = False) -> str:
    """Compile the oracle library with g++ (-O3, no target-specific flags)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["g++", "-O3", "-std=c++17", "-shared", "-fPIC", "-pthread", _SRC, "-o", tmp]
        )
        os.replace(tmp, _SO)
    return _SO


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            L.oracle_divmod_u32.argtypes = [U32P, ctypes.c_int, U32P, ctypes.c_int, U32P, ctypes.c_int, U32P, ctypes.c_int]
            L.oracle_divmod_u16.argtypes = [U16P, ctypes.c_int, U16P, ctypes.c_int, U16P, ctypes.c_int, U16P, ctypes.c_int]
            L.oracle_divmod_u8.argtypes = [U8P, ctypes.c_int, U8P, ctypes.c_int, U8P, ctypes.c_int, U8P, ctypes.c_int]
            for f in (L.oracle_divmod_u32, L.oracle_divmod_u16, L.oracle_divmod_u8):
                f.restype = ctypes.c_int
            L.oracle_addback_count.restype = ctypes.c_longlong
            L.oracle_addback_count.argtypes = []
            L.oracle_addback_reset.restype = None
            L.oracle_addback_reset.argtypes = []
            L.oracle_shinv_u32.argtypes = [U32P, ctypes.c_int, ctypes.c_int, U32P, ctypes.c_int]
            L.oracle_shinv_u32.restype = ctypes.c_int
            L.oracle_check_u32.argtypes = [U32P, ctypes.c_int, U32P, ctypes.c_int, U32P, ctypes.c_int, U32P, ctypes.c_int]
            L.oracle_check_u32.restype = ctypes.c_int
            L.oracle_divmod_batch_u32.argtypes = [
                ctypes.c_longlong, U32P, ctypes.c_int, ctypes.c_longlong, U32P, ctypes.c_int, ctypes.c_longlong,
                U32P, ctypes.c_int, ctypes.c_longlong, U32P, ctypes.c_int, ctypes.c_longlong, I32P, ctypes.c_int,
            ]
            L.oracle_divmod_batch_u32.restype = ctypes.c_int
            L.oracle_divmod_ragged_u32.argtypes = [
                ctypes.c_longlong, U32P, I64P, I32P, U32P, I64P, I32P, U32P, I64P, I32P, U32P, I64P, I32P, I32P,
                ctypes.c_int,
            ]
            L.oracle_divmod_ragged_u32.restype = ctypes.c_int
            _lib = L
    return _lib


def _p(a: np.ndarray, t):
    return a.ctypes.data_as(t)


def _c(a, dtype=np.uint32) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=dtype))


# ---------------------------------------------------------------- conversions
def to_int(d) -> int:
    """Little-endian uint32 digits -> Python int."""
    d = _c(d)
    return int.from_bytes(d.astype("<u4").tobytes(), "little")


def from_int(x: int, n: int) -> np.ndarray:
    """Python int -> n little-endian uint32 digits (x must fit)."""
    if x < 0 or x >= 1 << (32 * n):
        raise ValueError("value does not fit")
    return np.frombuffer(x.to_bytes(4 * n, "little"), dtype="<u4").astype(np.uint32)


def sig_len(d) -> int:
    d = _c(d)
    nz = np.nonzero(d)[0]
    return int(nz[-1]) + 1 if nz.size else 0


# ---------------------------------------------------------------- single items
def divmod_u32(u, v, qn: int | None = None, rn: int | None = None):
    """(q, r, status) for one item: q has qn digits (default: enough for any
    quotient, max(len u - significant digits of v + 1, 1)), r has rn digits
    (default len v). status 0 ok, 1 division by zero."""
    u, v = _c(u), _c(v)
    if qn is None:
        qn = max(len(u) - max(sig_len(v), 1) + 1, 1)
    if rn is None:
        rn = max(len(v), 1)
    q = np.zeros(qn, np.uint32)
    r = np.zeros(rn, np.uint32)
    st = lib().oracle_divmod_u32(_p(u, U32P), len(u), _p(v, U32P), len(v), _p(q, U32P), qn, _p(r, U32P), rn)
    if st == 2:
        raise ValueError("output buffers too short")
    return q, r, st


def divmod_narrow(u, v, bits: int):
    """Algorithm D on 8- or 16-bit digits (to drive the add-back step)."""
    dt, fn, P = {8: (np.uint8, "oracle_divmod_u8", U8P), 16: (np.uint16, "oracle_divmod_u16", U16P)}[bits]
    u, v = _c(u, dt), _c(v, dt)
    qn, rn = max(len(u) - len(v) + 1, 1), max(len(v), 1)
    q = np.zeros(qn, dt)
    r = np.zeros(rn, dt)
    st = getattr(lib(), fn)(_p(u, P), len(u), _p(v, P), len(v), _p(q, P), qn, _p(r, P), rn)
    return q, r, st


def addback_count() -> int:
    return int(lib().oracle_addback_count())


def addback_reset() -> None:
    lib().oracle_addback_reset()


def shinv_u32(v, h: int, outn: int | None = None) -> np.ndarray:
    """floor(B^h / v), B = 2^32 (Definition 1)."""
    v = _c(v)
    if outn is None:
        outn = h + 1
    out = np.zeros(outn, np.uint32)
    st = lib().oracle_shinv_u32(_p(v, U32P), len(v), h, _p(out, U32P), outn)
    if st:
        raise ValueError(f"shinv failed with status {st}")
    return out


def check_u32(u, v, q, r) -> int:
    """0 when u == q v + r and r < v; see knuthd.cpp for the other codes."""
    u, v, q, r = _c(u), _c(v), _c(q), _c(r)
    return int(lib().oracle_check_u32(_p(u, U32P), len(u), _p(v, U32P), len(v), _p(q, U32P), len(q), _p(r, U32P), len(r)))


# ---------------------------------------------------------------- batches
def divmod_batch_u32(U: np.ndarray, V: np.ndarray, qn: int, rn: int, nthreads: int = 0):
    """Uniform batch: U is (items, un), V is (items, vn). Returns (Q, R, status, threads)."""
    U, V = _c(U), _c(V)
    n = U.shape[0]
    Q = np.zeros((n, qn), np.uint32)
    R = np.zeros((n, rn), np.uint32)
    st = np.zeros(n, np.int32)
    used = lib().oracle_divmod_batch_u32(
        n, _p(U, U32P), U.shape[1], U.shape[1], _p(V, U32P), V.shape[1], V.shape[1],
        _p(Q, U32P), qn, qn, _p(R, U32P), rn, rn, _p(st, I32P), nthreads,
    )
    return Q, R, st, used


def divmod_ragged_u32(u_flat, u_off, u_len, v_flat, v_off, v_len, q_off, q_len, r_off, r_len, nthreads: int = 0):
    """Ragged batch over flat digit arrays with per-item offsets and lengths."""
    u_flat, v_flat = _c(u_flat), _c(v_flat)
    u_off, v_off, q_off, r_off = (_c(a, np.int64) for a in (u_off, v_off, q_off, r_off))
    u_len, v_len, q_len, r_len = (_c(a, np.int32) for a in (u_len, v_len, q_len, r_len))
    n = len(u_off)
    q_flat = np.zeros(int((q_off + q_len).max()) if n else 0, np.uint32)
    r_flat = np.zeros(int((r_off + r_len).max()) if n else 0, np.uint32)
    st = np.zeros(n, np.int32)
    used = lib().oracle_divmod_ragged_u32(
        n, _p(u_flat, U32P), _p(u_off, I64P), _p(u_len, I32P), _p(v_flat, U32P), _p(v_off, I64P), _p(v_len, I32P),
        _p(q_flat, U32P), _p(q_off, I64P), _p(q_len, I32P), _p(r_flat, U32P), _p(r_off, I64P), _p(r_len, I32P),
        _p(st, I32P), nthreads,
    )
    return q_flat, r_flat, st, used

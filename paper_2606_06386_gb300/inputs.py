"""Seeded synthetic inputs for batched midsize-integer division.

This module only draws operands: it holds none of the division method's
arithmetic, and both the CUDA path's tests/benchmark and the CPU oracle take
their inputs from here. Every draw comes from SplitMix64 (Steele, Lea and
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014) used as a
counter-based generator: output i of stream s is mix(seed + s*C + (i+1)*gamma),
with the published gamma 0x9E3779B97F4A7C15 and the published finaliser.

The paper draws its operands as random integers (Section 4, Methodology); the
workloads below follow that, at the sizes of the division configurations this
library is measured on. Digits are little-endian uint32; "top digit nonzero"
means the top digit is drawn uniformly from [1, 2^32).
"""

from __future__ import annotations

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
STREAM_STRIDE = np.uint64(0xD1B54A32D192ED03)
SEED_BASE = 0x6D70646976  # b"mpdiv" read as an integer
M64 = (1 << 64) - 1


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def splitmix64(seed: int, stream: int, count: int) -> np.ndarray:
    """count outputs of SplitMix64 for (seed, stream), as uint64."""
    with np.errstate(over="ignore"):
        base = np.uint64((seed + stream * int(STREAM_STRIDE)) & M64)
        ctr = np.arange(1, count + 1, dtype=np.uint64)
        return _mix(base + ctr * GAMMA)


def digits(seed: int, stream: int, count: int) -> np.ndarray:
    """count uniform uint32 digits (two per 64-bit draw)."""
    z = splitmix64(seed, stream, (count + 1) // 2)
    return z.view(np.uint32)[:count].copy()


def uniform01(seed: int, stream: int, count: int) -> np.ndarray:
    """count doubles uniform in [0, 1): top 53 bits of each draw."""
    z = splitmix64(seed, stream, count)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))


def _top_nonzero(top: np.ndarray) -> np.ndarray:
    # uniform in [1, 2^32): 1 + (x mod (2^32 - 1))
    return (1 + (top.astype(np.uint64) % np.uint64(0xFFFFFFFF))).astype(np.uint32)


def uniform_batch(n_items: int, n: int, seed: int, stream: int, top_nonzero: bool = True) -> np.ndarray:
    """(n_items, n) uniform digits; top digit of each row nonzero if asked."""
    a = digits(seed, stream, n_items * n).reshape(n_items, n)
    if top_nonzero and n > 0:
        a[:, -1] = _top_nonzero(a[:, -1])
    return a


# ------------------------------------------------------------------ helpers
def int_to_digits(x: int, n: int) -> np.ndarray:
    return np.frombuffer(int(x).to_bytes(4 * n, "little"), dtype="<u4").astype(np.uint32)


def digits_to_int(d: np.ndarray) -> int:
    return int.from_bytes(np.ascontiguousarray(d, dtype="<u4").tobytes(), "little")


B = 1 << 32


# ------------------------------------------------------------------ workloads
def plain_1024(n_random: int = 256):
    """Plain method at 2^15 bits: n_random uniform (u: 1024 digits, v: 512 digits)
    pairs plus 16 seeded edge cases (v a power of two, v = B^k - 1, u < v,
    u an exact multiple of v), all in full-width buffers.
    Returns (U (items,1024), V (items,512), names)."""
    seed = SEED_BASE + 0
    n, kl = 1024, 512
    U = uniform_batch(n_random, n, seed, 0)
    V = uniform_batch(n_random, kl, seed, 1)
    names = ["uniform"] * n_random
    ru = lambda s, m: digits_to_int(uniform_batch(1, m, seed, s)[0])  # noqa: E731
    edge = []
    # v a power of two
    for j, v in enumerate([1, 1 << 31, B**511, 1 << (32 * 300 + 17)]):
        edge.append((ru(10 + j, n), v, f"v_pow2_{j}"))
    # v = B^k - 1
    for j, k in enumerate([1, 2, 511, 512]):
        edge.append((ru(20 + j, n), B**k - 1, f"v_Bk_minus_1_k{k}"))
    # u < v
    v0 = ru(30, kl)
    edge.append((0, v0, "u_zero"))
    edge.append((v0 - 1, v0, "u_v_minus_1"))
    edge.append((ru(31, kl - 1), ru(32, kl), "u_511_digits"))
    vt = ru(33, kl)
    edge.append((vt - (1 << (32 * (kl - 1))), vt, "u_v_top_digit_minus_1"))
    # u = c v
    v1 = ru(40, kl)
    for j, c in enumerate([1, B**100, ru(41, 400), B**512 - 1]):
        edge.append((c * v1, v1, f"u_c_times_v_{j}"))
    EU = np.stack([int_to_digits(u, n) for u, _, _ in edge])
    EV = np.stack([int_to_digits(v, kl) for _, v, _ in edge])
    names += [nm for _, _, nm in edge]
    return np.concatenate([U, EU]), np.concatenate([V, EV]), names


SWEEP = [(1024, 512, 8192), (2048, 1024, 4096), (4096, 2048, 2048), (8192, 4096, 1024)]


def sweep(n: int, kl: int, n_items: int, stream_base: int = 0):
    """Plain per-size batched sweep: uniform digits, top digits nonzero."""
    seed = SEED_BASE + 1
    U = uniform_batch(n_items, n, seed, stream_base + 2 * n)
    V = uniform_batch(n_items, kl, seed, stream_base + 2 * n + 1)
    return U, V


def mixed_sizes(n_items: int = 8192, seed: int = SEED_BASE + 2):
    """Mixed precisions: dividend bits 2^(15 + 3x), x uniform, rounded to whole
    digits (1024..8192); divisor length round((0.25 + 0.75 y) n) >= 1, y uniform.
    Returns (u_len, v_len) int32 arrays."""
    x = uniform01(seed, 0, n_items)
    y = uniform01(seed, 1, n_items)
    bits = np.exp2(15.0 + 3.0 * x)
    u_len = np.clip(np.rint(bits / 32.0), 1024, 8192).astype(np.int32)
    v_len = np.maximum(1, np.rint((0.25 + 0.75 * y) * u_len)).astype(np.int32)
    v_len = np.minimum(v_len, u_len)
    return u_len, v_len


def ragged_operands(u_len: np.ndarray, v_len: np.ndarray, seed: int, stream: int = 10):
    """Flat digit arrays for a ragged batch (top digit of every item nonzero).
    Returns (u_flat, u_off, v_flat, v_off)."""
    u_len = np.asarray(u_len, np.int64)
    v_len = np.asarray(v_len, np.int64)
    u_off = np.concatenate([[0], np.cumsum(u_len)[:-1]]).astype(np.int64)
    v_off = np.concatenate([[0], np.cumsum(v_len)[:-1]]).astype(np.int64)
    u_flat = digits(seed, stream, int(u_len.sum()))
    v_flat = digits(seed, stream + 1, int(v_len.sum()))
    if len(u_len):
        u_flat[u_off + u_len - 1] = _top_nonzero(u_flat[u_off + u_len - 1])
        v_flat[v_off + v_len - 1] = _top_nonzero(v_flat[v_off + v_len - 1])
    return u_flat, u_off, v_flat, v_off


def poisson_arrivals(n_requests: int, rate_per_s: float, seed: int = SEED_BASE + 3, stream: int = 0) -> np.ndarray:
    """Arrival times (s) of a Poisson stream: cumulative exponential gaps."""
    gaps = -np.log1p(-uniform01(seed, stream, n_requests)) / rate_per_s
    return np.cumsum(gaps)


STRESS_VARIANTS = ("a_short_divisor", "b_just_over_half", "c_all_ones", "d_sparse", "e_v_Bk_minus_1")


def stress(variant: str, n_items: int = 1024, n: int = 8192):
    """Stress cases at 2^18 bits (n = 8192 digits):
    a: u uniform, v of 32 digits;  b: v of 4097 digits (2^17 + 32 bits);
    c: u = B^n - 1, v = B^(n/2) - 1;  d: 1%-nonzero digits for u (n) and v (n/2);
    e: u uniform, v = B^(n/2) - 1.  Returns (U, V)."""
    seed = SEED_BASE + 4
    s = 100 * (STRESS_VARIANTS.index(variant) + 1)
    half = n // 2
    if variant == "a_short_divisor":
        return uniform_batch(n_items, n, seed, s), uniform_batch(n_items, 32, seed, s + 1)
    if variant == "b_just_over_half":
        return uniform_batch(n_items, n, seed, s), uniform_batch(n_items, half + 1, seed, s + 1)
    if variant == "c_all_ones":
        return (np.full((n_items, n), 0xFFFFFFFF, np.uint32), np.full((n_items, half), 0xFFFFFFFF, np.uint32))
    if variant == "d_sparse":
        U = np.where(uniform01(seed, s + 2, n_items * n).reshape(n_items, n) < 0.01,
                     digits(seed, s, n_items * n).reshape(n_items, n), 0).astype(np.uint32)
        V = np.where(uniform01(seed, s + 3, n_items * half).reshape(n_items, half) < 0.01,
                     digits(seed, s + 1, n_items * half).reshape(n_items, half), 0).astype(np.uint32)
        zero = ~V.any(axis=1)
        r = 0
        while zero.any():  # redraw all-zero divisors with a fresh stream
            r += 1
            idx = np.nonzero(zero)[0]
            W = np.where(uniform01(seed, s + 10 + 2 * r, len(idx) * half).reshape(len(idx), half) < 0.01,
                         digits(seed, s + 11 + 2 * r, len(idx) * half).reshape(len(idx), half), 0).astype(np.uint32)
            V[idx] = W
            zero = ~V.any(axis=1)
        return U, V
    if variant == "e_v_Bk_minus_1":
        return uniform_batch(n_items, n, seed, s), np.full((n_items, half), 0xFFFFFFFF, np.uint32)
    raise ValueError(variant)


# The paper's own datasets (Section 4, Datasets and Methodology): precisions of
# 2^13..2^18 bits with 2^32 / bits instances each; u has precision M - 2 and v
# a random precision in [2, M/2], in the paper's 64-bit digits (M = bits / 64).
PAPER_TABLE = [(1 << b, 1 << (32 - b)) for b in (13, 14, 15, 16, 17, 18)]
# One size beyond the paper's table, built the same way: 2^19 bits, 2^13 instances.
BEYOND_TABLE = [(1 << 19, 1 << 13)]


def paper_workload(bits: int, n_items: int, seed: int = SEED_BASE + 6):
    """Operands of one Table 1 dataset in uint32 digits: u has 2(M - 2) digits
    (top digit nonzero); v has 2p digits, p uniform in [2, M/2] per item (top
    digit nonzero), stored zero-padded to M digits (M = bits / 64, so M 32-bit
    digits = M/2 64-bit digits). Returns (U, V, v_len)."""
    m64 = bits // 64
    un = 2 * (m64 - 2)
    vmax = m64
    U = uniform_batch(n_items, un, seed, 2 * bits)
    p = 2 + np.floor(uniform01(seed, 2 * bits + 1, n_items) * (m64 // 2 - 1)).astype(np.int64)
    v_len = (2 * p).astype(np.int32)
    V = digits(seed, 2 * bits + 2, n_items * vmax).reshape(n_items, vmax)
    col = np.arange(vmax)[None, :]
    V = np.where(col < v_len[:, None], V, 0).astype(np.uint32)
    rows = np.arange(n_items)
    V[rows, v_len - 1] = _top_nonzero(V[rows, v_len - 1])
    return U, V, v_len

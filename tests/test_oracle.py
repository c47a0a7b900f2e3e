"""Pins for the CPU oracle (Knuth Algorithm D in oracle/knuthd.cpp).

Each test ties the oracle to something other than itself: CPython's own long
division on operands that fit in 128 bits (brute force), closed forms of the
quotient and remainder, the exact identity u = q v + r checked by an
independent schoolbook product, and planted mistakes that the checker must
reject.
"""

import random

import numpy as np
import pytest

import oracle as O
from paper_2606_06386_gb300 import inputs as I

B = 1 << 32


def _div(u: int, v: int, n: int, k: int):
    q, r, st = O.divmod_u32(O.from_int(u, n), O.from_int(v, k))
    return O.to_int(q), O.to_int(r), st


def test_bruteforce_small_operands_against_python_int():
    # every length combination up to 4 digits (128 bits), random and structured values
    rnd = random.Random(7)
    special = [0, 1, 2, B - 1, B, B + 1, B**2 - 1, B**2, B**3 - 1, B**4 - 1, 1 << 63, (1 << 64) + 1]
    cases = 0
    for n in range(1, 5):
        for k in range(1, 5):
            vals_u = [x for x in special if x < B**n] + [rnd.getrandbits(32 * n) for _ in range(60)]
            vals_v = [x for x in special if 0 < x < B**k] + [rnd.getrandbits(32 * k) or 1 for _ in range(60)]
            for u in vals_u:
                for v in vals_v[:: max(1, len(vals_v) // 12)]:
                    q, r, st = _div(u, v, n, k)
                    assert st == 0
                    assert (q, r) == divmod(u, v), (u, v)
                    cases += 1
    assert cases > 1000


def test_division_by_zero_status():
    q, r, st = O.divmod_u32(O.from_int(12345, 3), np.zeros(2, np.uint32))
    assert st == 1 and not q.any() and not r.any()


@pytest.mark.parametrize("bits", [8, 16])
def test_narrow_digits_drive_addback(bits):
    # With 8/16-bit digits the add-back step of Algorithm D (probability ~2/B per
    # quotient digit) fires often; the same template must still agree with
    # CPython's division, and the counter proves the branch ran.
    rnd = random.Random(bits)
    O.addback_reset()
    base = 1 << bits
    dt = np.uint8 if bits == 8 else np.uint16
    for _ in range(3000):
        n = rnd.randint(2, 12)
        k = rnd.randint(2, n)
        u = rnd.getrandbits(bits * n)
        v = rnd.getrandbits(bits * k) | (1 << (bits * k - 1 - rnd.randint(0, bits - 1)))
        ud = np.array([(u >> (bits * i)) & (base - 1) for i in range(n)], dt)
        vd = np.array([(v >> (bits * i)) & (base - 1) for i in range(k)], dt)
        q, r, st = O.divmod_narrow(ud, vd, bits)
        qi = sum(int(x) << (bits * i) for i, x in enumerate(q))
        ri = sum(int(x) << (bits * i) for i, x in enumerate(r))
        assert (qi, ri) == divmod(u, v)
    if bits == 8:  # ~2/256 per quotient digit: thousands of digits make it certain
        assert O.addback_count() > 0


def test_config_sized_samples_against_python_int():
    U, V, names = I.plain_1024(n_random=8)
    for i in range(len(U)):
        u, v = O.to_int(U[i]), O.to_int(V[i])
        q, r, st = O.divmod_u32(U[i], V[i])
        assert st == 0
        assert (O.to_int(q), O.to_int(r)) == divmod(u, v), names[i]
    U, V = I.sweep(8192, 4096, 2)
    for i in range(2):
        q, r, st = O.divmod_u32(U[i], V[i])
        assert (O.to_int(q), O.to_int(r)) == divmod(O.to_int(U[i]), O.to_int(V[i]))


def test_closed_form_power_of_two_divisor():
    rnd = random.Random(3)
    for j in [0, 1, 31, 32, 33, 95, 32 * 300 + 17, 32 * 511]:
        u = rnd.getrandbits(32 * 1024)
        q, r, _ = _div(u, 1 << j, 1024, 512)
        assert q == u >> j and r == u & ((1 << j) - 1)


def test_closed_form_v_B_pow_k_minus_1():
    # B^k == 1 (mod B^k - 1): r is the sum of the k-digit blocks of u, reduced
    rnd = random.Random(4)
    for k in [1, 2, 5, 511, 512]:
        u = rnd.getrandbits(32 * 1024)
        m = B**k - 1
        s, x = 0, u
        while x:
            s += x & m
            x >>= 32 * k
        while s >= m:
            s = (s & m) + (s >> (32 * k))
        if s == m:
            s = 0
        q, r, _ = _div(u, m, 1024, 512)
        assert r == s
        assert q * m + r == u


def test_closed_form_all_ones():
    # (B^n - 1) / (B^k - 1) with k | n is sum_{i < n/k} B^(i k), remainder 0
    for n, k in [(8, 4), (1024, 512), (8192, 4096), (12, 3)]:
        q, r, _ = _div(B**n - 1, B**k - 1, n, k)
        assert r == 0 and q == sum(B ** (i * k) for i in range(n // k))


def test_closed_form_multiples_and_small_dividend():
    rnd = random.Random(5)
    for _ in range(20):
        v = rnd.getrandbits(32 * 300) | 1
        c = rnd.getrandbits(32 * rnd.randint(1, 600))
        q, r, _ = _div(c * v, v, 1024, 512)
        assert (q, r) == (c, 0)
        u = rnd.randrange(0, v)
        q, r, _ = _div(u, v, 1024, 512)
        assert (q, r) == (0, u)


def test_shinv_definition_and_closed_forms():
    rnd = random.Random(6)
    for _ in range(30):
        k = rnd.randint(1, 40)
        v = rnd.getrandbits(32 * k) | 1
        h = rnd.randint(k, 80)
        s = O.to_int(O.shinv_u32(O.from_int(v, k), h))
        assert s == B**h // v
    # shinv_h(B^k) = B^(h-k); shinv_h(2) = 2^(32h - 1)
    assert O.to_int(O.shinv_u32(O.from_int(B**3, 4), 10)) == B**7
    assert O.to_int(O.shinv_u32(O.from_int(2, 1), 10)) == 1 << (32 * 10 - 1)


def test_checker_accepts_truth_and_rejects_planted_mistakes():
    U, V = I.sweep(1024, 512, 3)
    for i in range(3):
        q, r, _ = O.divmod_u32(U[i], V[i])
        assert O.check_u32(U[i], V[i], q, r) == 0
        q2 = q.copy()
        q2[0] ^= 1  # wrong quotient digit
        assert O.check_u32(U[i], V[i], q2, r) != 0
        r2 = r.copy()
        r2[5] ^= 1 << 7  # wrong remainder digit
        assert O.check_u32(U[i], V[i], q, r2) != 0
        # r + v with q - 1 keeps the identity but breaks r < v
        qi, ri, vi = O.to_int(q), O.to_int(r), O.to_int(V[i])
        assert O.check_u32(U[i], V[i], O.from_int(qi - 1, len(q)), O.from_int(ri + vi, len(r) + 1)) == 2


def test_batch_entry_matches_single_and_uses_threads():
    U, V = I.sweep(1024, 512, 16)
    Q, R, st, used = O.divmod_batch_u32(U, V, 513, 512, nthreads=4)
    assert used == 4 and not st.any()
    for i in range(0, 16, 5):
        q, r, _ = O.divmod_u32(U[i], V[i])
        assert (Q[i] == q).all() and (R[i] == r).all()


def test_ragged_entry_matches_single():
    u_len, v_len = I.mixed_sizes(12)
    u_flat, u_off, v_flat, v_off = I.ragged_operands(u_len, v_len, seed=99)
    q_len = np.maximum(u_len - v_len + 1, 1).astype(np.int32)
    q_off = np.concatenate([[0], np.cumsum(q_len)[:-1]]).astype(np.int64)
    r_off = np.concatenate([[0], np.cumsum(v_len)[:-1]]).astype(np.int64)
    qf, rf, st, _ = O.divmod_ragged_u32(u_flat, u_off, u_len, v_flat, v_off, v_len, q_off, q_len, r_off, v_len, 3)
    assert not st.any()
    for i in range(12):
        u = O.to_int(u_flat[u_off[i] : u_off[i] + u_len[i]])
        v = O.to_int(v_flat[v_off[i] : v_off[i] + v_len[i]])
        assert O.to_int(qf[q_off[i] : q_off[i] + q_len[i]]) == u // v
        assert O.to_int(rf[r_off[i] : r_off[i] + v_len[i]]) == u % v

"""Pins for the exact-integer model of Algorithms 1-3 (oracle/shinv_model.py).

* The whole-shifted Newton step of Eq. (3) must reproduce the iterates and
  quotients printed in the paper's worked examples (tests/golden).
* Algorithm 1 must return floor(B^h / v) + lambda with lambda in {0, 1}
  (Theorem 2), checked against the Knuth-D oracle's floor(B^h / v).
* Algorithm 3 must return exactly (u quo v, u rem v), with delta in {-1, 0, 1}.
* The Refine loop runs ceil(max(log2(h-k-1), 0)) + 2 times.
* Planted mistakes (sign of PowDiff, one Refine iteration short) must be caught.
"""

import os
import random

import pytest

import oracle as O
import oracle.shinv_model as M

B32 = 1 << 32
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "worked_examples.txt")


def _golden():
    vals = {}
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *rest = line.split()
            vals[key] = [int(x) for x in rest]
    return vals


def test_worked_examples_eq3_iterates_and_quotients():
    g = _golden()
    B, h, v = g["base"][0], g["h"][0], g["v"][0]
    its = g["iterates"]
    w = its[0]
    for expect in its[1:]:
        w = M.newton_shift_step(w, v, h, B)
        assert w == expect
    # Example 1: q = shift_{-h}(u * shinv_h(v)), no correction
    u1 = g["example1_u"][0]
    assert M.shift(-h, u1 * w, B) == g["example1_q"][0] == u1 // v
    # Example 2: q0 is one short; the remainder u - q0 v exceeds v; delta = +1
    u2 = g["example2_u"][0]
    q0 = M.shift(-h, u2 * w, B)
    assert q0 == g["example2_q0"][0]
    assert u2 - q0 * v == g["example2_rem0"][0] >= v
    assert q0 + 1 == g["example2_q"][0] == u2 // v
    # the converged iterate is the shifted inverse of Definition 1
    assert w == B**h // v


def _rand_pair(rnd, nmax):
    n = rnd.randint(1, nmax)
    kl = rnd.randint(1, n)
    u = rnd.getrandbits(32 * n)
    v = rnd.getrandbits(32 * kl) or 1
    r = rnd.random()
    if r < 0.1:
        v = B32 ** rnd.randint(1, kl) - 1
    elif r < 0.15:
        v = B32 ** rnd.randint(0, kl - 1)
    elif r < 0.2:
        v = 1 << rnd.randint(0, 32 * kl - 1)
    return u, v


def test_shinv_within_theorem2_against_knuth_oracle():
    rnd = random.Random(21)
    for _ in range(400):
        u, v = _rand_pair(rnd, 24)
        h = max(M.prec(u, B32), 1)
        kl = M.prec(v, B32)
        exact = O.to_int(O.shinv_u32(O.from_int(v, kl), h))
        s = M.shinv(v, h, B32)
        assert s - exact in (0, 1), (u, v)


def test_div_matches_knuth_oracle_with_bounded_delta():
    rnd = random.Random(22)
    deltas = set()
    for _ in range(400):
        u, v = _rand_pair(rnd, 24)
        n, kl = max(M.prec(u, B32), 1), M.prec(v, B32)
        q, r, d = M.div(u, v, B32)
        qo, ro, st = O.divmod_u32(O.from_int(u, n), O.from_int(v, kl))
        assert st == 0 and (q, r) == (O.to_int(qo), O.to_int(ro))
        assert d in (-1, 0, 1)
        deltas.add(d)
    assert 1 in deltas  # the delta = +1 correction is common (Example 2)


def test_overestimated_shinv_and_negative_delta_at_base_16():
    # Theorem 2: the revised Shinv may return floor(B^h/v) + 1. These base-16
    # divisors reach lambda = 1, and some dividends then need delta = -1.
    B = 16
    for v, h in [(32638565307, 11), (13408681392, 11)]:
        assert M.shinv(v, h, B) == B**h // v + 1
    rnd = random.Random(23)
    v, h = 13408681392, 11
    seen = set()
    for _ in range(20000):
        u = rnd.randrange(B ** (h - 1), B**h)
        q, r, d = M.div(u, v, B)
        assert (q, r) == divmod(u, v)
        seen.add(d)
    assert -1 in seen


def test_refine_iteration_count_formula():
    assert M.refine_iterations(5, 4) == 2  # h-k-1 = 0: log undefined, read as 2
    assert M.refine_iterations(6, 4) == 2  # h-k-1 = 1
    assert M.refine_iterations(7, 4) == 3  # h-k-1 = 2
    assert M.refine_iterations(1024, 511) == 11
    assert M.refine_iterations(8192, 4095) == 14
    assert M.refine_iterations(8192, 31) == 15
    tr = M.Trace()
    rnd = random.Random(24)
    v = rnd.getrandbits(32 * 512) | (1 << (32 * 512 - 1))
    M.shinv(v, 1024, B32, tr)
    assert tr.iterations == 11


def test_special_cases_of_algorithm1():
    B = B32
    assert M.shinv(7, 5, B) == B**5 // 7  # v < B
    assert M.shinv(B**6, 5, B) == 0  # v > B^h
    assert M.shinv(B**5 // 2 + 1, 5, B) == 1  # 2v > B^h
    assert M.shinv(B**3, 7, B) == B**4  # v = B^k


def _first_bad(mutant):
    rnd = random.Random(25)
    for _ in range(300):
        u, v = _rand_pair(rnd, 20)
        h = max(M.prec(u, B32), 1)
        s = mutant(v, h)
        if s - B32**h // v not in (0, 1):
            return True
    return False


def test_planted_mistakes_are_caught(monkeypatch):
    orig_pd = M.powdiff

    def flipped(v, w, h, ell, B, tr, lo=0):
        s, x = orig_pd(v, w, h, ell, B, tr, lo)
        return (1 - s if x else s), x

    monkeypatch.setattr(M, "powdiff", flipped)
    assert _first_bad(lambda v, h: M.shinv(v, h, B32))
    monkeypatch.setattr(M, "powdiff", orig_pd)
    orig_it = M.refine_iterations
    monkeypatch.setattr(M, "refine_iterations", lambda h, k: max(2, orig_it(h, k) - 1))
    assert _first_bad(lambda v, h: M.shinv(v, h, B32))


@pytest.mark.parametrize("n,kl", [(1024, 512), (64, 32), (300, 37)])
def test_product_sizes_stay_near_cost_model(n, kl):
    # Section 2.3: the division costs a handful of full multiplications; at
    # half-length divisors the exact trace stays below 7 units of n(n+1)/2.
    rnd = random.Random(n)
    u = rnd.getrandbits(32 * n) | (1 << (32 * n - 1))
    v = rnd.getrandbits(32 * kl) | (1 << (32 * kl - 1))
    tr = M.Trace()
    q, r, _ = M.div(u, v, B32, tr)
    assert (q, r) == divmod(u, v)
    total = tr.digit_products()
    assert total <= 7 * n * (n + 1) / 2


def test_clipped_division_is_exact_and_cheaper():
    # Section 5's clipped products: the quotient from the top columns only and
    # the remainder modulo B^(k+2); the corrections restore the exact result
    rnd = random.Random(26)
    for _ in range(300):
        u, v = _rand_pair(rnd, 24)
        tr = M.Trace()
        assert M.div_clipped(u, v, B32, tr) == divmod(u, v)
    n, kl = 512, 256
    u = rnd.getrandbits(32 * n) | (1 << (32 * n - 1))
    v = rnd.getrandbits(32 * kl) | (1 << (32 * kl - 1))
    tf, tc = M.Trace(), M.Trace()
    M.div(u, v, B32, tf)
    M.div_clipped(u, v, B32, tc)
    assert tc.digit_products() < 0.7 * tf.digit_products()


def test_clipped_quotient_is_at_most_one_short():
    rnd = random.Random(27)
    for _ in range(200):
        n = rnd.randint(3, 30)
        kl = rnd.randint(2, n)
        u = rnd.getrandbits(32 * n) | (1 << (32 * n - 1))
        v = rnd.getrandbits(32 * kl) | (1 << (32 * kl - 1))
        h = M.prec(u, B32)
        w = M.shinv(v, h, B32)
        lo = h - 2
        low = sum(((w >> (32 * j)) & (B32 - 1)) * (u % B32 ** (lo - j)) * B32**j for j in range(M.prec(w, B32)) if lo - j > 0)
        q_full = (u * w) // B32**h
        q_clip = (u * w - low) // B32**h
        assert q_full - q_clip in (0, 1)


def test_clipped_newton_step_is_at_most_one_unit_off():
    # Step with w*x clipped below e - 2 (e = digits Step drops): each Step result
    # is Algorithm 1's or one unit away (down on the + branch, up on the -
    # branch); at base 16 the clip changes some steps
    seen = {"steps": 0, "changed": 0}
    orig = M.step

    def checking_step(h, v, w, m, ell, g, B, tr, clip=False, guard=2):
        a = orig(h, v, w, m, ell, g, B, M.Trace())
        b = orig(h, v, w, m, ell, g, B, M.Trace(), True, guard)
        seen["steps"] += 1
        seen["changed"] += a != b
        assert b - a in (-1, 0, 1)
        return orig(h, v, w, m, ell, g, B, tr, clip, guard)

    rnd = random.Random(33)
    M.step = checking_step
    try:
        for _ in range(1500):
            n = rnd.randint(3, 14)
            kl = rnd.randint(2, n)
            u = rnd.randrange(16 ** (n - 1), 16**n)
            v = rnd.randrange(16 ** (kl - 1), 16**kl)
            M.shinv(v, M.prec(u, 16), 16, None, True)
    finally:
        M.step = orig
    assert seen["changed"] > 0 and seen["steps"] > 1000


@pytest.mark.parametrize("B", [16, 256, 1 << 16, B32])
def test_clipped_newton_steps_keep_division_exact(B):
    # the shifted inverse with clipped Newton steps stays within -1..+2 of
    # floor(B^h / v) (the Knuth oracle at base 2^32, integer floor otherwise),
    # and the clipped division (Section 5) returns the exact quotient and remainder
    rnd = random.Random(B % 1000 + 7)
    for _ in range(300):
        n = rnd.randint(3, 40 if B == B32 else 14)
        kl = rnd.randint(2, n)
        u = rnd.randrange(B ** (n - 1), B**n)
        v = rnd.randrange(B ** (kl - 1), B**kl)
        h = M.prec(u, B)
        w = M.shinv(v, h, B, None, True)
        exact = O.to_int(O.shinv_u32(O.from_int(v, kl), h)) if B == B32 else B**h // v
        assert w - exact in (-1, 0, 1, 2)
        assert M.div_clipped(u, v, B, None, 2, True) == divmod(u, v)


def test_clipped_newton_steps_save_a_fifth_of_the_products():
    # half-length divisor at 2^15 bits: clipping Step's w*x as well removes
    # about three quarters of the Newton steps' digit products
    rnd = random.Random(34)
    n, kl = 1024, 512
    u = rnd.getrandbits(32 * n) | (1 << (32 * n - 1))
    v = rnd.getrandbits(32 * kl) | (1 << (32 * kl - 1))
    t0, t1 = M.Trace(), M.Trace()
    assert M.div_clipped(u, v, B32, t0) == M.div_clipped(u, v, B32, t1, clip_step=True) == divmod(u, v)
    assert t1.digit_products() < 0.8 * t0.digit_products()
    assert t1.digit_products() < 0.9 * n * (n + 1) / 2


@pytest.mark.parametrize("B", [16, 256, 1 << 16])
def test_clipped_powdiff_error_is_the_dropped_sum(B, monkeypatch):
    # PowDiff's close product summed from column lo up drops the digit products
    # below lo. At every call the clipped Newton iteration makes, the signed
    # result B^h - v w comes out larger by exactly the dropped sum (no wrap
    # modulo B^L), which is below min(prec v, prec w) (B - 1)^2 B^(lo-1) times
    # B/(B-1) < min(prec v, prec w) B^(lo+1); the exact value from Python
    # integers.
    orig = M.powdiff
    seen = {"calls": 0, "moved": 0}

    def checking(v, w, h, ell, B_, tr, lo=0):
        s, x = orig(v, w, h, ell, B_, tr, lo)
        if lo > 0:
            s0, x0 = orig(v, w, h, ell, B_, M.Trace(), 0)
            assert (s0, x0) == ((1, B_**h - v * w) if B_**h >= v * w else (0, v * w - B_**h))
            d = (x if s else -x) - (x0 if s0 else -x0)
            assert 0 <= d < min(M.prec(v, B_), M.prec(w, B_)) * B_ ** (lo + 1), (v, w, h, ell, lo)
            seen["calls"] += 1
            seen["moved"] += d > 0
        return s, x

    monkeypatch.setattr(M, "powdiff", checking)
    rnd = random.Random(B + 3)
    for _ in range(300):
        n = rnd.randint(6, 30)
        kl = rnd.randint(2, n - 1)
        v = rnd.randrange(B ** (kl - 1), B**kl)
        M.shinv(v, n, B, None, True)
    assert seen["calls"] > 100 and seen["moved"] > 20


def test_clipped_powdiff_saves_a_third_of_its_products():
    # at 2^16 bits (2048 / 1024 digits): PowDiff's close products lose about a
    # third of their digit pairs, and the division stays exact
    rnd = random.Random(35)
    n, kl = 2048, 1024
    u = rnd.getrandbits(32 * n) | (1 << (32 * n - 1))
    v = rnd.getrandbits(32 * kl) | (1 << (32 * kl - 1))
    tr = M.Trace()
    assert M.div_clipped(u, v, B32, tr, clip_step=True) == divmod(u, v)
    mod = [p for p in tr.products if p[0] == "powdiff_mod"]
    kept = sum(max(0, min(k, keep - i) - max(0, lo - i)) for _, m, k, keep, lo in mod for i in range(m))
    full = sum(max(0, min(k, keep - i)) for _, m, k, keep, lo in mod for i in range(m))
    assert any(lo > 0 for *_, lo in mod)
    assert 0.6 * full < kept < 0.72 * full


def test_clipped_iteration_bound_at_realistic_sizes():
    # readings 14-15 at base 2^32 and hundreds of digits, where every Newton
    # step and PowDiff of the clipped iteration drops columns: the shifted
    # inverse stays within -1..+2 of floor(B^h / v) (the Knuth oracle) and
    # the clipped division is exact
    rnd = random.Random(36)
    clipped = 0
    for _ in range(24):
        n = rnd.randint(100, 600)
        kl = rnd.randint(2, n - 1)
        u = rnd.getrandbits(32 * n) | (1 << (32 * n - 1))
        v = rnd.getrandbits(32 * kl) | (1 << (32 * kl - 1 - rnd.randint(0, 31)))
        tr = M.Trace()
        w = M.shinv(v, n, B32, tr, True)
        exact = O.to_int(O.shinv_u32(O.from_int(v, kl), n))
        assert w - exact in (-1, 0, 1, 2)
        clipped += any(p[0] == "powdiff_mod" and p[4] > 0 for p in tr.products)
        assert M.div_clipped(u, v, B32, None, 2, True) == divmod(u, v)
    assert clipped >= 16  # the PowDiff clip acts unless the divisor is nearly as long as the dividend

"""Tests of the model of the kernel's clipped-product design (tests/kernel_model.py).

The model is not the oracle: it restates the design choices the division
kernels make beyond the paper (clipped Newton step, PowDiff, quotient and
remainder products), so that the kernels' intermediate values and work counts
can be checked against it. Here it is pinned to the oracle and to brute force:

* with every clip off it equals Algorithms 1-3 as printed (the oracle's model),
  iterate for iterate and product for product;
* its digit-product count equals a brute-force count of the pairs
  lo <= i + j < keep;
* the clipped division returns the Knuth oracle's (q, r), and each clipped
  step stays within the bounds the design claims.
"""

import random

import pytest

import oracle as O
import oracle.shinv_model as M
import kernel_model as K

from test_shinv_model import counted_schoolbook

B32 = 1 << 32


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


@pytest.mark.parametrize("B", [16, 256, B32])
def test_unclipped_model_is_algorithm1_as_printed(B):
    rnd = random.Random(51 + B % 97)
    for _ in range(150):
        n = rnd.randint(2, 30)
        kl = rnd.randint(1, n)
        v = rnd.randrange(B ** (kl - 1), B**kl)
        t0, t1 = M.Trace(), K.KTrace()
        assert K.shinv(v, n, B, t1, False) == M.shinv(v, n, B, t0)
        assert t1.iterates == t0.iterates and t1.iterations == t0.iterations
        assert [p[:4] for p in t1.products] == t0.products
        assert t1.digit_products() == t0.digit_products()


def test_clipped_count_equals_brute_force():
    rnd = random.Random(52)
    for _ in range(200):
        m, n = rnd.randint(1, 12), rnd.randint(1, 12)
        keep = rnd.choice([None, rnd.randint(1, m + n)])
        lo = rnd.randint(0, m + n)
        a = rnd.randrange(16 ** (m - 1), 16**m)
        b = rnd.randrange(16 ** (n - 1), 16**n)
        s_hi, c = counted_schoolbook(a, b, 16, keep, lo)
        s_lo, _ = counted_schoolbook(a, b, 16, min(lo, m + n if keep is None else keep))
        mod = 16 ** (m + n if keep is None else keep)
        assert (s_hi + s_lo) % mod == (a * b) % mod
        assert K.pairs_between(m, n, keep, lo) == c, (m, n, keep, lo)
        assert K.low_pairs(a, b, lo, 16) == counted_schoolbook(a, b, 16, lo)[0]
    # a planted off-by-one at the lower bound is caught
    bad = lambda m, n, keep, lo: K.pairs_between(m, n, keep, max(0, lo - 1))  # noqa: E731
    assert any(bad(m, n, None, lo) != counted_schoolbook(16 ** (m - 1), 16 ** (n - 1), 16, None, lo)[1]
               for m, n, lo in ((3, 3, 2), (5, 2, 4), (4, 4, 1)))


def test_clipped_division_is_exact_and_cheaper():
    # Section 5's clipped products: the quotient from the top columns only and
    # the remainder modulo B^(k+2); the corrections restore the exact result
    rnd = random.Random(26)
    for _ in range(300):
        u, v = _rand_pair(rnd, 24)
        tr = K.KTrace()
        assert K.div_clipped(u, v, B32, tr) == divmod(u, v)
    n, kl = 512, 256
    u = rnd.getrandbits(32 * n) | (1 << (32 * n - 1))
    v = rnd.getrandbits(32 * kl) | (1 << (32 * kl - 1))
    tf, tc = K.KTrace(), K.KTrace()
    M.div(u, v, B32, tf)
    K.div_clipped(u, v, B32, tc)
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
    orig = K.step

    def checking_step(h, v, w, m, ell, g, B, tr, clip=False, guard=2):
        a = orig(h, v, w, m, ell, g, B, K.KTrace())
        b = orig(h, v, w, m, ell, g, B, K.KTrace(), True, guard)
        seen["steps"] += 1
        seen["changed"] += a != b
        assert b - a in (-1, 0, 1)
        return orig(h, v, w, m, ell, g, B, tr, clip, guard)

    rnd = random.Random(33)
    K.step = checking_step
    try:
        for _ in range(1500):
            n = rnd.randint(3, 14)
            kl = rnd.randint(2, n)
            u = rnd.randrange(16 ** (n - 1), 16**n)
            v = rnd.randrange(16 ** (kl - 1), 16**kl)
            K.shinv(v, M.prec(u, 16), 16, None, True)
    finally:
        K.step = orig
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
        w = K.shinv(v, h, B, None, True)
        exact = O.to_int(O.shinv_u32(O.from_int(v, kl), h)) if B == B32 else B**h // v
        assert w - exact in (-1, 0, 1, 2)
        assert K.div_clipped(u, v, B, None, 2, True) == divmod(u, v)


def test_clipped_newton_steps_save_a_fifth_of_the_products():
    # half-length divisor at 2^15 bits: clipping Step's w*x as well removes
    # about three quarters of the Newton steps' digit products
    rnd = random.Random(34)
    n, kl = 1024, 512
    u = rnd.getrandbits(32 * n) | (1 << (32 * n - 1))
    v = rnd.getrandbits(32 * kl) | (1 << (32 * kl - 1))
    t0, t1 = K.KTrace(), K.KTrace()
    assert K.div_clipped(u, v, B32, t0) == K.div_clipped(u, v, B32, t1, clip_step=True) == divmod(u, v)
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
    orig = K.powdiff
    seen = {"calls": 0, "moved": 0}

    def checking(v, w, h, ell, B_, tr, lo=0):
        s, x = orig(v, w, h, ell, B_, tr, lo)
        if lo > 0:
            s0, x0 = orig(v, w, h, ell, B_, K.KTrace(), 0)
            assert (s0, x0) == ((1, B_**h - v * w) if B_**h >= v * w else (0, v * w - B_**h))
            d = (x if s else -x) - (x0 if s0 else -x0)
            assert 0 <= d < min(M.prec(v, B_), M.prec(w, B_)) * B_ ** (lo + 1), (v, w, h, ell, lo)
            seen["calls"] += 1
            seen["moved"] += d > 0
        return s, x

    monkeypatch.setattr(K, "powdiff", checking)
    rnd = random.Random(B + 3)
    for _ in range(300):
        n = rnd.randint(6, 30)
        kl = rnd.randint(2, n - 1)
        v = rnd.randrange(B ** (kl - 1), B**kl)
        K.shinv(v, n, B, None, True)
    assert seen["calls"] > 100 and seen["moved"] > 20


def test_clipped_powdiff_saves_a_third_of_its_products():
    # at 2^16 bits (2048 / 1024 digits): PowDiff's close products lose about a
    # third of their digit pairs, and the division stays exact
    rnd = random.Random(35)
    n, kl = 2048, 1024
    u = rnd.getrandbits(32 * n) | (1 << (32 * n - 1))
    v = rnd.getrandbits(32 * kl) | (1 << (32 * kl - 1))
    tr = K.KTrace()
    assert K.div_clipped(u, v, B32, tr, clip_step=True) == divmod(u, v)
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
        tr = K.KTrace()
        w = K.shinv(v, n, B32, tr, True)
        exact = O.to_int(O.shinv_u32(O.from_int(v, kl), n))
        assert w - exact in (-1, 0, 1, 2)
        clipped += any(p[0] == "powdiff_mod" and p[4] > 0 for p in tr.products)
        assert K.div_clipped(u, v, B32, None, 2, True) == divmod(u, v)
    assert clipped >= 16  # the PowDiff clip acts unless the divisor is nearly as long as the dividend

"""Pins for the exact-integer model of Algorithms 1-3 (oracle/shinv_model.py).

Every pin checks the model against something other than itself: the paper's
printed worked examples, the Knuth-D oracle, closed forms, or brute force.

* The whole-shifted Newton step of Eq. (3) must reproduce the iterates and
  quotients printed in the paper's worked examples (tests/golden).
* Algorithm 1 must return floor(B^h / v) + lambda with lambda in {0, 1}
  (Theorem 2), checked against the Knuth-D oracle's floor(B^h / v).
* Algorithm 3 must return exactly (u quo v, u rem v), with delta in {-1, 0, 1}.
* The Refine loop runs ceil(max(log2(h-k-1), 0)) + 2 times.
* Planted mistakes (sign of PowDiff, one Refine iteration short) must be caught.
* The digit-product count of a trace (Section 2.3's cost, Fig. 3's n-digit
  product kept to n digits) equals a brute-force count taken by an
  instrumented schoolbook multiplication whose value is checked against
  Python's product; closed forms pin the quotient and remainder products; and
  planted off-by-one counts are caught.
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

    def flipped(v, w, h, ell, B, tr):
        s, x = orig_pd(v, w, h, ell, B, tr)
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


# ---------------------------------------------------------------- the digit-product count
def counted_schoolbook(a: int, b: int, B: int, keep=None, lo: int = 0):
    """Schoolbook multiplication digit by digit over the pairs (i, j) with
    lo <= i + j < keep, counting each digit product it makes: (sum, count)."""
    A = [(a // B**i) % B for i in range(M.prec(a, B))]
    C = [(b // B**j) % B for j in range(M.prec(b, B))]
    hi = len(A) + len(C) if keep is None else keep
    s = count = 0
    for i, ai in enumerate(A):
        for j, cj in enumerate(C):
            if lo <= i + j < hi:
                s += ai * cj * B ** (i + j)
                count += 1
    return s, count


def _count_pin_failures(count):
    """Shapes where count(m, n, keep) disagrees with the brute-force count of
    an instrumented schoolbook product whose value is checked against Python's
    product modulo B^keep. Operands have nonzero top digits and arbitrary
    (also zero) inner digits."""
    rnd = random.Random(41)
    B = 16
    bad = []
    shapes = [(1, 1, None), (1, 5, None), (5, 1, 3), (3, 3, 1), (4, 7, 4), (7, 4, 4), (6, 6, 11), (6, 6, 12),
              (9, 2, 10), (2, 9, 2)]
    shapes += [(rnd.randint(1, 12), rnd.randint(1, 12), None) for _ in range(20)]
    shapes += [(m, n, rnd.randint(1, m + n)) for m, n in ((rnd.randint(1, 12), rnd.randint(1, 12)) for _ in range(60))]
    for m, n, keep in shapes:
        a = rnd.randrange(B ** (m - 1), B**m)
        b = rnd.randrange(B ** (n - 1), B**n)
        s, c = counted_schoolbook(a, b, B, keep)
        mod = B ** (m + n if keep is None else keep)
        assert s % mod == (a * b) % mod  # the enumerated pairs are exactly those of the product mod B^keep
        if count(m, n, keep) != c:
            bad.append((m, n, keep))
    return bad


def test_digit_product_count_equals_brute_force():
    assert _count_pin_failures(M.pairs_below) == []
    # through a trace: one record per product, summed
    tr = M.Trace()
    rnd = random.Random(42)
    expect = 0
    for _ in range(30):
        m, n = rnd.randint(1, 10), rnd.randint(1, 10)
        keep = rnd.choice([None, rnd.randint(1, m + n)])
        a = rnd.randrange(16 ** (m - 1), 16**m)
        b = rnd.randrange(16 ** (n - 1), 16**n)
        tr.mult("x", a, b, 16, keep)
        expect += counted_schoolbook(a, b, 16, keep)[1]
    assert tr.digit_products() == expect


def test_planted_off_by_one_counts_are_caught():
    mutants = [
        lambda m, n, keep: m * n if keep is None else sum(max(0, min(n, keep - i + 1)) for i in range(m)),
        lambda m, n, keep: m * n if keep is None else sum(max(0, min(n, keep - i - 1)) for i in range(m)),
        lambda m, n, keep: m * n if keep is None else sum(max(0, min(n, keep - i)) for i in range(m - 1)),
        lambda m, n, keep: m * n if keep is None else sum(max(0, min(n + 1, keep - i)) for i in range(m)),
        lambda m, n, keep: m * n,  # the close product counted as a full one
        lambda m, n, keep: (m + 1) * n if keep is None else M.pairs_below(m, n, keep),
    ]
    for f in mutants:
        assert _count_pin_failures(f), f


def test_full_trace_at_2e15_bits_matches_closed_forms_and_the_cost_model():
    # Algorithms 1-3 as printed at n = 1024, k_l = 512 (2^15-bit dividend,
    # half-length divisor). The quotient product u * shinv_h(v) costs
    # prec(u) prec(floor(B^h / v)) (+ one digit when Theorem 2's lambda = 1),
    # the remainder product v q costs prec(v) prec(q) with q from the Knuth
    # oracle, and the whole division about 2.10 units of n(n+1)/2 (1.10 M
    # products: 0.316 M in Shinv, 0.525 M in the quotient, 0.263 M in the
    # remainder), Section 2.3's 5-7 full multiplications read with Fig. 3's
    # n-digit unit.
    rnd = random.Random(43)
    n, kl = 1024, 512
    u = rnd.getrandbits(32 * n) | (1 << (32 * n - 1))
    v = rnd.getrandbits(32 * kl) | (1 << (32 * kl - 1))
    tr = M.Trace()
    q, r, delta = M.div(u, v, B32, tr)
    qo, ro, st = O.divmod_u32(O.from_int(u, n), O.from_int(v, kl))
    assert st == 0 and (q, r) == (O.to_int(qo), O.to_int(ro))
    by_tag = {}
    for tag, m, k, keep in tr.products:
        by_tag[tag] = by_tag.get(tag, 0) + M.pairs_below(m, k, keep)
    shinv_exact = O.to_int(O.shinv_u32(O.from_int(v, kl), n))
    assert by_tag["quotient"] == n * M.prec(shinv_exact, B32) == 1024 * 513
    q0 = q - delta
    assert by_tag["remainder"] == kl * M.prec(q0, B32)
    newton = by_tag["powdiff_full"] + by_tag.get("powdiff_mod", 0) + by_tag["step"]
    assert abs(newton - 0.316e6) < 0.01 * 0.316e6
    total = tr.digit_products()
    assert total == newton + by_tag["quotient"] + by_tag["remainder"]
    assert abs(total - 1.10e6) < 0.01 * 1.10e6
    assert abs(total / (n * (n + 1) / 2) - 2.10) < 0.01

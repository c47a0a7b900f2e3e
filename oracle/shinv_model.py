"""Exact-integer model of the whole-shifted-inverse division (test infrastructure).

This module is part of the test oracle. Only the test-suite, the smoke check and
the benchmark's CPU-baseline leg may import it; the product path never does.

It restates, with Python's unbounded integers and in the paper's order and
notation, the three algorithms of the paper (arXiv 2606.06386):

* ``shinv``   -- Algorithm 1, Shinv(v, h, B): special cases, the two-digit
  initial approximation w = B^3 quo V, then Refine.
* ``refine`` / ``step`` -- Algorithm 1, functions Refine and Step.
* ``powdiff`` -- Algorithm 2, PowDiff(v, w, h, l, B) with explicit sign.
* ``div``     -- Algorithm 3, Div(u, v): q = shift_{-h}(u * shinv_h(v)) then
  the two one-step corrections of Theorem 2 (delta in {-1, 0, 1}).
* ``div_clipped`` -- Algorithm 3 with the clipped products of Section 5
  (quotient, remainder and, optionally, Newton step), as the GPU computes it.

Nothing here is blocked, fused or reordered: each line is one step of the
algorithm as printed, with the readings below where the text is ambiguous.

Readings of the paper taken here (Section 2.2, Algorithms 1-3):

* shift_n(x) = floor(x * B^n) (Definition 1); for n < 0 this is floor
  division by B^-n, also for the negative intermediate of Step.
* The Refine loop bound ceil(max(log2(h-k-1), 0)) + 2 is taken as 2 whenever
  h - k - 1 <= 1 (the logarithm is undefined or zero there).
* The final shift of Refine is h-k-4 digits when h - k < 2, else -2 (read
  literally; the variable the paper calls q there is not the quotient).
* The initial approximation uses the two top digits, V = v_{k-1} + v_k B, and
  w = B^3 quo V, which can equal B^2 (three digits) when V = B.
* Step's negative branch subtracts one when any of the (h - 2m) dropped low
  digits of tmp is nonzero, which makes the shift a floor (Definition 1).
* The B < 16 digit-grouping branch of Algorithm 1 is not modelled: every base
  used here is at least 16.

The model also records, per call, the sizes of every operand it multiplies
(``trace``), which the tests use to check operation counts.
"""

from __future__ import annotations

from dataclasses import dataclass, field


def prec(x: int, B: int) -> int:
    """Number of base-B digits of x >= 0 (0 for x = 0)."""
    if x < 0:
        raise ValueError("prec of a negative integer")
    n = 0
    while x:
        x //= B
        n += 1
    return n


def shift(n: int, x: int, B: int) -> int:
    """Whole shift, Definition 1: floor(x * B^n)."""
    if n >= 0:
        return x * B**n
    return x // B ** (-n)  # Python // is floor division, also for x < 0


@dataclass
class Trace:
    """Per-call record of the multiplications made and of the Refine loop."""

    iterations: int = 0
    products: list = field(default_factory=list)  # (tag, prec a, prec b)
    iterates: list = field(default_factory=list)  # w after each Refine step

    def mult(self, tag: str, a: int, b: int, B: int, keep: int | None = None, lo: int = 0) -> int:
        """Record a product of prec(a) x prec(b) digits; ``keep`` is the number of
        low digits a close product (MultMod) keeps, ``lo`` the lowest column a
        clipped product computes."""
        self.products.append((tag, prec(a, B), prec(b, B), keep, lo))
        return a * b

    def digit_products(self) -> int:
        """Digit products of the multiplications made: the digit pairs (i, j) of
        an m x n product with lo <= i + j < keep (keep = m + n for a full product,
        L for one kept modulo B^L; lo = 0 unless the product is clipped)."""
        total = 0
        for _, m, n, keep, lo in self.products:
            hi = m + n if keep is None else keep
            total += sum(max(0, min(n, hi - i) - max(0, lo - i)) for i in range(m))
        return total


def powdiff(v: int, w: int, h: int, ell: int, B: int, tr: Trace, lo: int = 0) -> tuple[int, int]:
    """Algorithm 2: (sign, |B^h - v*w|), sign 1 when B^h - v*w >= 0.

    With ``lo`` > 0 the close product (MultMod) sums only the digit products
    at columns lo and up (the clipped PowDiff of ``step``): P is then
    (v w - D) mod B^L with D the dropped sum, 0 <= D < min(prec v, prec w)
    B^(lo+1), and the signed result B^h - v w comes out larger by D.
    """
    L = prec(v, B) + prec(w, B) - ell + 1
    if v == 0 or w == 0 or L >= h:
        P = tr.mult("powdiff_full", v, w, B)
        if B**h > P:
            return 1, B**h - P
        return 0, P - B**h
    # MultMod: the product kept modulo B^L (the close product)
    P = tr.mult("powdiff_mod", v, w, B, keep=L, lo=min(lo, L))
    if lo > 0:
        P -= low_pairs(v, w, lo, B)
    P %= B**L
    if P == 0:
        return 1, 0
    if (P // B ** (L - 1)) % B == 0:
        return 0, P
    return 1, B**L - P


def low_pairs(a: int, b: int, lo: int, B: int) -> int:
    """Sum of the digit products a_i b_j B^(i+j) with i + j < lo."""
    total = 0
    for j in range(prec(b, B)):
        if lo - j <= 0:
            break
        total += ((b // B**j) % B) * (a % B ** (lo - j)) * B**j
    return total


def step(h: int, v: int, w: int, m: int, ell: int, g: int, B: int, tr: Trace,
         clip: bool = False, guard: int = 2) -> int:
    """Algorithm 1, Step: one Newton iteration on the shifted inverse.

    With ``clip``, w * x is clipped the way Section 5 proposes for the
    quotient: Step keeps only the digits of w * x at and above position
    e = h - 2m, so the digit products below e - guard are skipped and the
    columns from e - guard up are summed exactly. The shifted product is then
    at most one short (the skipped sum is below B^(e-1) times the shorter
    operand's digit count), and the floor's sticky digit is read from the
    summed columns only. PowDiff's close product is clipped too, below column
    lo = e - prec(w) - 1 - guard: its dropped sum D < B^(lo+2) makes w x
    larger by w D < B^(prec(w) + lo + 2) = B^(e - 1), so the shifted product
    is at most one larger. Each Step result is then within -1..+2 units of
    Algorithm 1's.
    """
    lo = max(0, h - 2 * m - prec(w, B) - 1 - guard) if clip else 0
    sign, x = powdiff(v, w, h - m, ell - g, B, tr, lo)
    if not clip:
        tmp = tr.mult("step", w, x, B)
    else:
        plo = max(0, h - 2 * m - guard)
        tmp = tr.mult("step", w, x, B, lo=plo)
        if plo > 0:
            if prec(w, B) + prec(x, B) <= plo:
                tmp = 0  # every column lies below the clip: nothing is summed
            else:
                tmp -= low_pairs(w, x, plo, B)
    if sign:
        return shift(m, w, B) + shift(2 * m - h, tmp, B)
    res = shift(m, w, B) - (tmp // B ** (h - 2 * m))
    if tmp % B ** (h - 2 * m) != 0:
        res -= 1
    return res


def refine_iterations(h: int, k: int) -> int:
    """Loop count of Refine: ceil(max(log2(h-k-1), 0)) + 2, read as 2 when h-k-1 <= 1."""
    t = h - k - 1
    if t <= 1:
        return 2
    c = 0
    while (1 << c) < t:  # ceil(log2 t) for t >= 2, exact in integers
        c += 1
    return c + 2


def refine(v: int, h: int, k: int, w: int, ell: int, B: int, tr: Trace, clip: bool = False) -> int:
    """Algorithm 1, Refine: shorter iterates with divisor prefixes (``clip``:
    Step's clipped product, see ``step``)."""
    g = 2
    w = shift(g, w, B)
    n_it = refine_iterations(h, k)
    for i in range(n_it):
        m = min(h - k + 1 - ell, ell)
        s = max(0, k - 2 * ell + 1 - g)
        w = step(k + ell + m - s + g, shift(-s, v, B), w, m, ell, g, B, tr, clip)
        if i < 2:
            w = shift(-m, w, B)
        else:
            w = shift(-1, w, B)
            ell = ell + m - 1
        tr.iterates.append(w)
    tr.iterations = n_it
    q = h - k - 4 if h - k < 2 else -2
    return shift(q, w, B)


def shinv(v: int, h: int, B: int, tr: Trace | None = None, clip: bool = False) -> int:
    """Algorithm 1, Shinv(v, h, B) for B >= 16 and v > 0 (``clip``: Step's
    clipped product, see ``step``; False: the paper's algorithm)."""
    if tr is None:
        tr = Trace()
    if v <= 0:
        raise ZeroDivisionError("shinv of a non-positive integer")
    if B < 16:
        raise ValueError("the digit-grouping branch for B < 16 is not modelled")
    k = prec(v, B) - 1  # B^k <= v < B^(k+1)
    if v < B:
        return B**h // v
    if v > B**h:
        return 0
    if 2 * v > B**h:
        return 1
    if v == B**k:
        return B ** (h - k)
    V = (v // B ** (k - 1)) % B + ((v // B**k) % B) * B
    w = B**3 // V
    return refine(v, h, k, w, 2, B, tr, clip)


def div(u: int, v: int, B: int, tr: Trace | None = None) -> tuple[int, int, int]:
    """Algorithm 3 with Theorem 2's corrections: returns (q, r, delta)."""
    if tr is None:
        tr = Trace()
    if v <= 0:
        raise ZeroDivisionError("division by zero")
    h = prec(u, B)
    w = shinv(v, h, B, tr)
    q = shift(-h, tr.mult("quotient", u, w, B), B)
    m = tr.mult("remainder", v, q, B)
    delta = 0
    if u < m:
        q -= 1
        m -= v
        delta = -1
    r = u - m
    if r >= v:
        q += 1
        r -= v
        delta += 1
    return q, r, delta


def newton_shift_step(w: int, v: int, h: int, B: int) -> int:
    """The whole-shifted Newton step of Eq. (3): w + shift_{-h}(shift_h(w) - v w^2)."""
    return w + shift(-h, shift(h, w, B) - v * w * w, B)


def div_clipped(u: int, v: int, B: int, tr: Trace | None = None, guard: int = 2,
                clip_step: bool = False) -> tuple[int, int]:
    """Algorithm 3 with clipped products (the refinement Section 5 proposes):

    * w = shinv_h(v) by Algorithm 1, with Step's product clipped when
      ``clip_step`` is set (see ``step``): w may then differ from Algorithm 1's
      by one unit;
    * q0 is formed from the digit products of u * w at columns h - guard and
      above only (the carries of the lower columns are dropped), which leaves
      q0 at most one short of shift_{-h}(u * w);
    * u - v q0 then lies in [-2v, 4v), so it is taken from v q0 modulo B^(k+2)
      (k + 1 = prec(v)) and read as a two's-complement number;
    * the corrections of Theorem 2 finish the division.
    """
    if tr is None:
        tr = Trace()
    if v <= 0:
        raise ZeroDivisionError("division by zero")
    h = prec(u, B)
    w = shinv(v, h, B, tr, clip_step)
    lo = max(0, h - guard)
    full = tr.mult("quotient_clipped", u, w, B, lo=lo)
    q = (full - low_pairs(u, w, lo, B)) // B**h
    K1 = prec(v, B) + 1
    t = (u - tr.mult("remainder_low", v, q, B, keep=K1)) % B**K1
    if t >= B**K1 // 2:
        t -= B**K1
    while t < 0:
        q -= 1
        t += v
    while t >= v:
        q += 1
        t -= v
    return q, t

"""Exact-integer model of the whole-shifted-inverse division (test infrastructure).

This module is part of the test oracle. Only the test-suite, the smoke check and
the benchmark's CPU-baseline leg may import it; the product path never does.

It restates, with Python's unbounded integers and in the paper's order and
notation, the three algorithms of the paper (arXiv 2606.06386) exactly as
printed, with the paper's full and close (MultMod) products:

* ``shinv``   -- Algorithm 1, Shinv(v, h, B): special cases, the two-digit
  initial approximation w = B^3 quo V, then Refine.
* ``refine`` / ``step`` -- Algorithm 1, functions Refine and Step.
* ``powdiff`` -- Algorithm 2, PowDiff(v, w, h, l, B) with explicit sign.
* ``div``     -- Algorithm 3, Div(u, v): q = shift_{-h}(u * shinv_h(v)) then
  the two one-step corrections of Theorem 2 (delta in {-1, 0, 1}).

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
* Cost (Section 2.3, Fig. 3): a product of an m-digit by an n-digit number
  costs its m n digit products; a close product kept modulo B^L costs the
  digit pairs (i, j) with i + j < L only.

The model also records, per call, the sizes of every operand it multiplies
(``Trace``), from which ``Trace.digit_products`` counts the digit products the
algorithms make.
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


def pairs_below(m: int, n: int, keep: int | None) -> int:
    """Digit pairs (i, j), i < m, j < n, with i + j < keep (all m n of them
    when keep is None): the digit products of an m x n product kept modulo
    B^keep. Row i contributes min(n, keep - i) pairs when that is positive."""
    if keep is None:
        return m * n
    return sum(max(0, min(n, keep - i)) for i in range(m))


@dataclass
class Trace:
    """Per-call record of the multiplications made and of the Refine loop."""

    iterations: int = 0
    products: list = field(default_factory=list)  # (tag, prec a, prec b, keep)
    iterates: list = field(default_factory=list)  # w after each Refine step

    def mult(self, tag: str, a: int, b: int, B: int, keep: int | None = None) -> int:
        """Record a product of prec(a) x prec(b) digits; ``keep`` is the number of
        low digits a close product (MultMod) keeps. Returns a * b."""
        self.products.append((tag, prec(a, B), prec(b, B), keep))
        return a * b

    def digit_products(self) -> int:
        """Digit products of the multiplications made (Section 2.3's cost): m n
        for a full m x n product, the pairs below L for one kept modulo B^L."""
        return sum(pairs_below(m, n, keep) for _, m, n, keep in self.products)


def powdiff(v: int, w: int, h: int, ell: int, B: int, tr: Trace) -> tuple[int, int]:
    """Algorithm 2: (sign, |B^h - v*w|), sign 1 when B^h - v*w >= 0."""
    L = prec(v, B) + prec(w, B) - ell + 1
    if v == 0 or w == 0 or L >= h:
        P = tr.mult("powdiff_full", v, w, B)
        if B**h > P:
            return 1, B**h - P
        return 0, P - B**h
    # MultMod: the product kept modulo B^L (the close product)
    P = tr.mult("powdiff_mod", v, w, B, keep=L) % B**L
    if P == 0:
        return 1, 0
    if (P // B ** (L - 1)) % B == 0:
        return 0, P
    return 1, B**L - P


def step(h: int, v: int, w: int, m: int, ell: int, g: int, B: int, tr: Trace) -> int:
    """Algorithm 1, Step: one Newton iteration on the shifted inverse."""
    sign, x = powdiff(v, w, h - m, ell - g, B, tr)
    tmp = tr.mult("step", w, x, B)
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


def refine(v: int, h: int, k: int, w: int, ell: int, B: int, tr: Trace) -> int:
    """Algorithm 1, Refine: shorter iterates with divisor prefixes."""
    g = 2
    w = shift(g, w, B)
    n_it = refine_iterations(h, k)
    for i in range(n_it):
        m = min(h - k + 1 - ell, ell)
        s = max(0, k - 2 * ell + 1 - g)
        w = step(k + ell + m - s + g, shift(-s, v, B), w, m, ell, g, B, tr)
        if i < 2:
            w = shift(-m, w, B)
        else:
            w = shift(-1, w, B)
            ell = ell + m - 1
        tr.iterates.append(w)
    tr.iterations = n_it
    q = h - k - 4 if h - k < 2 else -2
    return shift(q, w, B)


def shinv(v: int, h: int, B: int, tr: Trace | None = None) -> int:
    """Algorithm 1, Shinv(v, h, B) for B >= 16 and v > 0."""
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
    return refine(v, h, k, w, 2, B, tr)


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

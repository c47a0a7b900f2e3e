"""Model of the CUDA kernel's clipped-product design (test infrastructure).

This is NOT the oracle. The oracle (``oracle/``) computes what the paper
defines: Knuth's Algorithm D for (q, r), and Algorithms 1-3 exactly as printed
(``oracle/shinv_model.py``). This module models the design choices the
division kernels make beyond the paper, so that tests can check the kernels'
intermediate values and work counts against a readable restatement:

* Step's product w x summed only from column e - guard up (e = h - 2m, the
  digits Step drops): the shifted product may be one short, and the floor's
  sticky digit is read from the summed columns;
* PowDiff's close product (MultMod) summed only from column
  lo = e - prec(w) - 1 - guard up: the signed result B^h - v w comes out larger
  by the dropped sum D < min(prec v, prec w) B^(lo+1);
* the quotient q0 from the digit products of u w at columns h - guard and up;
* u - v q0 from v q0 modulo B^(prec(v)+1), read as a two's-complement number,
  then the corrections of Theorem 2 (as many as needed).

Section 5 of the paper proposes clipped products for the quotient; the clipped
Newton step and PowDiff extend the idea. The parity that matters -- (q, r)
against the Knuth oracle -- never goes through this module. With every clip
off it reproduces Algorithms 1-3 as printed, which a test checks against the
oracle's model.

``KTrace.digit_products`` counts the digit products the kernel computes: the
pairs (i, j) of an m x n product with lo <= i + j < keep.
"""

from __future__ import annotations

from dataclasses import dataclass, field

from oracle.shinv_model import prec, refine_iterations, shift


def pairs_between(m: int, n: int, keep: int | None, lo: int) -> int:
    """Digit pairs (i, j), i < m, j < n, with lo <= i + j < keep (keep None:
    no upper bound). Row i contributes the j in [max(0, lo - i), min(n, keep - i))."""
    hi = m + n if keep is None else keep
    return sum(max(0, min(n, hi - i) - max(0, lo - i)) for i in range(m))


@dataclass
class KTrace:
    """Per-call record of the products the kernel design computes."""

    iterations: int = 0
    products: list = field(default_factory=list)  # (tag, prec a, prec b, keep, lo)
    iterates: list = field(default_factory=list)

    def mult(self, tag: str, a: int, b: int, B: int, keep: int | None = None, lo: int = 0) -> int:
        self.products.append((tag, prec(a, B), prec(b, B), keep, lo))
        return a * b

    def digit_products(self) -> int:
        return sum(pairs_between(m, n, keep, lo) for _, m, n, keep, lo in self.products)


def low_pairs(a: int, b: int, lo: int, B: int) -> int:
    """Sum of the digit products a_i b_j B^(i+j) with i + j < lo."""
    total = 0
    for j in range(prec(b, B)):
        if lo - j <= 0:
            break
        total += ((b // B**j) % B) * (a % B ** (lo - j)) * B**j
    return total


def powdiff(v: int, w: int, h: int, ell: int, B: int, tr: KTrace, lo: int = 0) -> tuple[int, int]:
    """Algorithm 2 with the close product summed from column lo up."""
    L = prec(v, B) + prec(w, B) - ell + 1
    if v == 0 or w == 0 or L >= h:
        P = tr.mult("powdiff_full", v, w, B)
        if B**h > P:
            return 1, B**h - P
        return 0, P - B**h
    P = tr.mult("powdiff_mod", v, w, B, keep=L, lo=min(lo, L))
    if lo > 0:
        P -= low_pairs(v, w, lo, B)
    P %= B**L
    if P == 0:
        return 1, 0
    if (P // B ** (L - 1)) % B == 0:
        return 0, P
    return 1, B**L - P


def step(h: int, v: int, w: int, m: int, ell: int, g: int, B: int, tr: KTrace,
         clip: bool = False, guard: int = 2) -> int:
    """Step with w x summed from column e - guard up and PowDiff's close
    product from e - prec(w) - 1 - guard up (``clip``); each result is then
    within -1..+2 units of Algorithm 1's."""
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


def refine(v: int, h: int, k: int, w: int, ell: int, B: int, tr: KTrace, clip: bool = False) -> int:
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


def shinv(v: int, h: int, B: int, tr: KTrace | None = None, clip: bool = False) -> int:
    """The shifted inverse as the kernel computes it (``clip``: clipped Newton
    steps and PowDiff, the kernels' default; False: Algorithm 1 as printed)."""
    if tr is None:
        tr = KTrace()
    if v <= 0:
        raise ZeroDivisionError("shinv of a non-positive integer")
    k = prec(v, B) - 1
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


def div_clipped(u: int, v: int, B: int, tr: KTrace | None = None, guard: int = 2,
                clip_step: bool = False) -> tuple[int, int]:
    """The kernel's default division: shifted inverse (clipped Newton steps
    when ``clip_step``), q0 from the columns of u w at h - guard and up,
    u - v q0 from v q0 modulo B^(prec(v)+1), then the corrections."""
    if tr is None:
        tr = KTrace()
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

"""Unit tests of the block-group primitives of the division path (through the
test entry mpdiv_debug_primitive), against Python integers, at several block
sizes: carries and borrows that run across every warp, the power-of-B steps,
the reductions, negation, and the clipped and full strip products."""

import numpy as np
import pytest

import oracle
from paper_2606_06386_gb300 import inputs as I

from gpu_util import ctx, dev, host_u32

pytestmark = pytest.mark.gpu
B = 1 << 32
FULL = 0xFFFFFFFF


def _run(op, X, Y, arg, cap, warps, cols=0):
    import torch
    import paper_2606_06386_gb300 as mp

    X = np.ascontiguousarray(X, np.uint32)
    Y = np.ascontiguousarray(Y, np.uint32)
    out = torch.full((X.shape[0], cap), -1, dtype=torch.int32, device="cuda:0")
    res = torch.full((X.shape[0],), -7, dtype=torch.int32, device="cuda:0")
    mp.mpdiv_debug_primitive(ctx(cols=cols), op, dev(X), dev(Y), arg, out, res, warps)
    torch.cuda.synchronize()
    return host_u32(out), res.cpu().numpy()


def _operands(n, m, k=12, seed=0):
    """k rows of structured and random operands of n and m digits."""
    X = I.uniform_batch(k, n, seed=300 + seed, stream=n, top_nonzero=False)
    Y = I.uniform_batch(k, m, seed=400 + seed, stream=m, top_nonzero=False)
    X[0] = FULL          # all ones: carries run through every digit
    Y[0] = 0
    Y[0, 0] = 1
    X[1] = 0             # zero: borrows run through every digit
    Y[1] = 0
    Y[1, 0] = 1
    X[2] = FULL
    Y[2] = FULL
    X[3] = 0
    Y[3] = 0
    X[4] = 0
    X[4, -1] = 1         # a single top digit
    Y[4] = 0
    Y[4, 0] = FULL
    return X, Y


@pytest.mark.parametrize("warps", [1, 4, 32])
@pytest.mark.parametrize("n,m", [(1, 1), (37, 5), (700, 700), (2500, 1300)])
def test_add_sub_cmp_prec(warps, n, m):
    X, Y = _operands(n, m, seed=warps)
    cap = max(n, m)
    for op in (0, 1):
        O, R = _run(op, X, Y, 0, cap, warps)
        for i in range(len(X)):
            x, y = oracle.to_int(X[i]), oracle.to_int(Y[i])
            s = x + y if op == 0 else x - y
            assert oracle.to_int(O[i]) == s % B**cap, (op, i)
            assert R[i] == (1 if (s >= B**cap if op == 0 else s < 0) else 0), (op, i)
    _, R = _run(2, X, Y, 0, 3, warps)
    for i in range(len(X)):
        x, y = oracle.to_int(X[i]), oracle.to_int(Y[i])
        assert R[i] == (x > y) - (x < y)
    _, R = _run(3, X, Y, 0, 3, warps)
    for i in range(len(X)):
        assert R[i] == oracle.sig_len(X[i])


@pytest.mark.parametrize("warps", [1, 2, 8, 16])
@pytest.mark.parametrize("n,e", [(5, 0), (5, 4), (300, 0), (300, 17), (2000, 1999), (2000, 700)])
def test_powers_of_b(warps, n, e):
    X, Y = _operands(n, 1, seed=e)
    cap = n
    O, R = _run(4, X, Y, e, cap, warps)
    for i in range(len(X)):
        x = oracle.to_int(X[i])
        if x >= B**e and x % B**cap >= B**e:
            assert R[i] == 1 and oracle.to_int(O[i]) == x - B**e
        else:
            assert R[i] == 0
    O, R = _run(5, X, Y, e, cap, warps)
    for i in range(len(X)):
        x = oracle.to_int(X[i])
        assert R[i] == (0 if x + B**e >= B**cap else 1)
        if R[i]:
            assert oracle.to_int(O[i]) == x + B**e


@pytest.mark.parametrize("warps", [1, 4, 32])
@pytest.mark.parametrize("n", [1, 33, 640, 3000])
def test_scan_and_negate(warps, n):
    X, Y = _operands(n, 1, seed=n)
    X[5] = FULL
    X[5, 0] = 7          # all ones above a low digit
    O, _ = _run(7, X, Y, 0, 3, warps)
    for i in range(len(X)):
        d = [int(t) for t in X[i]]
        nz = [j for j, t in enumerate(d) if t != 0]
        nf = [j for j, t in enumerate(d) if t != FULL]
        want = [nz[0] if nz else -1, nz[-1] if nz else -1, nf[-1] if nf else -1]
        assert [int(np.int32(np.uint32(t))) for t in O[i][:3]] == want, i
    cap = n + 2
    O, _ = _run(8, X, Y, 0, cap, warps)
    for i in range(len(X)):
        x = oracle.to_int(X[i])
        if x:
            assert oracle.to_int(O[i]) == B**cap - x


@pytest.mark.parametrize("cols", [3, 5, 7])
@pytest.mark.parametrize("warps", [1, 4, 16])
@pytest.mark.parametrize("n,m,plo", [(1, 1, 0), (50, 3, 0), (300, 300, 0), (1200, 700, 0), (1200, 700, 1000),
                                     (900, 900, 1799), (2100, 37, 400)])
def test_full_and_clipped_products(cols, warps, n, m, plo):
    X, Y = _operands(n, m, k=6, seed=cols)
    cap = n + m
    O, R = _run(6, X, Y, plo, cap, warps, cols)
    for i in range(len(X)):
        x, y = oracle.to_int(X[i]), oracle.to_int(Y[i])
        low = sum(int(X[i][a]) * (y % B ** (plo - a)) * B**a for a in range(min(n, plo)))  # pairs below plo
        want = ((x * y - low) // B**plo) % B ** (cap - plo)
        assert oracle.to_int(O[i][plo:]) == want, i
        assert not O[i][:plo].any()
        assert R[i] == plo

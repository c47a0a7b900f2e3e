"""The number-theoretic-transform product (MPDIV_FLAG_NTT_PRODUCTS) on the GPU:
the product itself against Python integers at every transform length up to
8192 points (with maximal coefficients, truncated and clipped outputs), and
the division with full products by the transform, bit-exact against the
oracle, with the shifted inverse and the product count equal to the exact
model of Algorithms 1-3."""

import random

import numpy as np
import pytest

import oracle
import oracle.shinv_model as M
from paper_2606_06386_gb300 import inputs as I

from gpu_util import assert_same, ctx, dev, host_u32, oracle_uniform, run_uniform

pytestmark = pytest.mark.gpu
B = 1 << 32
FULL = 0xFFFFFFFF
NTT = 4 | 2  # MPDIV_FLAG_NTT_PRODUCTS (implies full products)


def _prim(X, Y, plo, cap, warps):
    import torch
    import paper_2606_06386_gb300 as mp

    X = np.ascontiguousarray(X, np.uint32)
    Y = np.ascontiguousarray(Y, np.uint32)
    out = torch.full((X.shape[0], cap), -1, dtype=torch.int32, device="cuda:0")
    res = torch.full((X.shape[0],), -7, dtype=torch.int32, device="cuda:0")
    mp.mpdiv_debug_primitive(ctx(), 9, dev(X), dev(Y), plo, out, res, warps)
    torch.cuda.synchronize()
    return host_u32(out), res.cpu().numpy()


def _operands(n, m, seed):
    X = I.uniform_batch(6, n, seed=500 + seed, stream=n, top_nonzero=False)
    Y = I.uniform_batch(6, m, seed=600 + seed, stream=m, top_nonzero=False)
    X[0] = FULL  # every coefficient at its maximum, min(n, m) (B - 1)^2
    Y[0] = FULL
    X[1] = 0
    Y[1] = FULL
    X[2] = FULL
    Y[2] = 0
    Y[2, 0] = 1
    X[3, :] = 0
    X[3, -1] = 1  # a single top digit
    return X, Y


@pytest.mark.parametrize("warps", [1, 4, 16, 32])
@pytest.mark.parametrize(
    "n,m,plo,cap",
    [(1, 1, 0, 2), (3, 2, 0, 5), (50, 3, 0, 53), (300, 300, 0, 600), (1200, 700, 0, 1900), (1200, 700, 1000, 1900),
     (2000, 2000, 0, 2500), (4096, 4096, 0, 8192), (8191, 1, 0, 8192), (5000, 3192, 6000, 8192), (1025, 1024, 0, 2049)],
)
def test_transform_product(warps, n, m, plo, cap):
    X, Y = _operands(n, m, seed=warps)
    O, R = _prim(X, Y, plo, cap, warps)
    for i in range(len(X)):
        want = (oracle.to_int(X[i]) * oracle.to_int(Y[i])) % B**cap
        assert oracle.to_int(O[i][plo:]) == want >> (32 * plo), i
        assert not O[i][:plo].any()
        assert R[i] == plo


@pytest.mark.parametrize("tcut", [0, 2])
@pytest.mark.parametrize("n,kl", [(1024, 512), (2048, 1024), (4096, 2048), (8192, 4096), (4096, 32), (300, 37),
                                  (97, 96), (500, 2), (2, 2)])
def test_transform_division_exact(n, kl, tcut):
    # tcut 2: every product of at least two digits by the transform where it fits
    k = 8 if n >= 4096 else 24
    U, V = I.sweep(n, kl, k)
    Q, R, S, _ = run_uniform(U, V, flags=NTT, tcut=tcut)
    Qo, Ro, So = oracle_uniform(U, V)
    assert_same(Q, R, S, Qo, Ro, So)


def test_transform_division_edge_cases():
    U, V, names = I.plain_1024(n_random=32)
    for tcut in (0, 2):
        Q, R, S, _ = run_uniform(U, V, flags=NTT, tcut=tcut)
        Qo, Ro, So = oracle_uniform(U, V)
        assert_same(Q, R, S, Qo, Ro, So, names)


def test_transform_shinv_equals_full_model():
    # every Newton-step, PowDiff, quotient-sized product by the transform: the
    # shifted inverse is exactly Algorithm 1's with full products
    import torch
    import paper_2606_06386_gb300 as mp

    rnd = random.Random(41)
    vs, hs = [], []
    for _ in range(24):
        kl = rnd.choice([2, 3, 40, 300, 1500])
        v = rnd.getrandbits(32 * kl) | (1 << (32 * kl - 1 - rnd.randint(0, 31)))
        h = rnd.randint(kl, min(3 * kl + 10, 3000))
        vs.append(v)
        hs.append(h)
    V = np.stack([oracle.from_int(v, 1500) for v in vs])
    out = torch.zeros((len(vs), 3002), dtype=torch.int32, device="cuda:0")
    it = torch.zeros(len(vs), dtype=torch.int32, device="cuda:0")
    st = torch.full((len(vs),), -1, dtype=torch.int32, device="cuda:0")
    mp.mpdiv_debug_shinv(ctx(flags=NTT, cols=3, tcut=2), dev(V), torch.tensor(hs, dtype=torch.int32, device="cuda:0"),
                         out, it, st)
    torch.cuda.synchronize()
    O, S, IT = host_u32(out), st.cpu().numpy(), it.cpu().numpy()
    for i, (v, h) in enumerate(zip(vs, hs)):
        assert S[i] == 0, i
        tr = M.Trace()
        assert oracle.to_int(O[i]) == M.shinv(v, h, B, tr), (i, h)
        assert IT[i] == tr.iterations


@pytest.mark.parametrize("n,kl", [(64, 32), (1024, 512), (97, 96), (500, 2)])
def test_transform_product_counter(n, kl):
    # the count of algorithmic digit products does not depend on how the
    # products are computed: the full model's count
    U = I.uniform_batch(4, n, seed=79, stream=n)
    V = I.uniform_batch(4, kl, seed=80, stream=kl)
    _, _, S, _, P = run_uniform(U, V, flags=NTT, tcut=2, products=True)
    for i in range(4):
        tr = M.Trace()
        M.div(oracle.to_int(U[i]), oracle.to_int(V[i]), B, tr)
        assert S[i] == 0 and P[i] == tr.digit_products()


@pytest.mark.parametrize("n", [512, 1024, 4096, 8192])
def test_transform_cost_unit(n):
    # (u v) mod B^n by the transform (n <= 4096) and by the strip product above
    import torch
    import paper_2606_06386_gb300 as mp

    U = I.uniform_batch(6, n, seed=92, stream=n)
    V = I.uniform_batch(6, n, seed=93, stream=n)
    U[0] = FULL
    V[0] = FULL
    out = torch.zeros((6, n), dtype=torch.int32, device="cuda:0")
    mp.mpdiv_mul_batch(ctx(flags=NTT, tcut=2), dev(U), dev(V), out)
    torch.cuda.synchronize()
    O = host_u32(out)
    for i in range(6):
        assert oracle.to_int(O[i]) == (oracle.to_int(U[i]) * oracle.to_int(V[i])) % (B**n)


def test_transform_ragged_queue():
    # the mixed-precision launch with the transform (one block per item from the
    # size-sorted queue): every item exact
    import torch
    import paper_2606_06386_gb300 as mp

    rnd = np.random.default_rng(7)
    u_len = rnd.integers(1024, 4097, 48).astype(np.int32)
    v_len = np.maximum(1, (u_len * rnd.uniform(0.25, 1.0, 48)).astype(np.int32))
    u_flat, u_off, v_flat, v_off = I.ragged_operands(u_len, v_len, seed=71)
    q_len, r_len = u_len.copy(), v_len.copy()
    q_off = np.concatenate([[0], np.cumsum(q_len)[:-1]]).astype(np.int64)
    r_off = np.concatenate([[0], np.cumsum(r_len)[:-1]]).astype(np.int64)
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")  # noqa: E731
    q = torch.full((int(q_len.sum()),), -1, dtype=torch.int32, device="cuda:0")
    r = torch.full((int(r_len.sum()),), -1, dtype=torch.int32, device="cuda:0")
    st = torch.full((len(u_len),), -7, dtype=torch.int32, device="cuda:0")
    mp.mpdiv_batch_ragged(ctx(flags=NTT), dev(u_flat), T(u_off), T(u_len), dev(v_flat), T(v_off), T(v_len), q,
                          T(q_off), T(q_len), r, T(r_off), T(r_len), st, None)
    torch.cuda.synchronize()
    Q, R, S = host_u32(q), host_u32(r), st.cpu().numpy()
    qo, ro, so, _ = oracle.divmod_ragged_u32(u_flat, u_off, u_len, v_flat, v_off, v_len, q_off, q_len, r_off, r_len)
    assert (S == so).all() and (Q == qo).all() and (R == ro).all()


def test_transform_with_karatsuba_steps():
    # products below the transform cutoff that are Newton-step products go
    # through one Karatsuba level, the longer ones through the transform
    for n, kl in [(4096, 2048), (2048, 1024), (4096, 100)]:
        U, V = I.sweep(n, kl, 12)
        Q, R, S, _ = run_uniform(U, V, flags=NTT, kcut=512, tcut=3000)
        Qo, Ro, So = oracle_uniform(U, V)
        assert_same(Q, R, S, Qo, Ro, So)


def test_transform_serving():
    # the serving loop on a context with the transform: one queue launch per
    # batch; every result equals the oracle's
    import paper_2606_06386_gb300 as mp

    rnd = np.random.default_rng(11)
    u_len = rnd.integers(1500, 4097, 24).astype(np.int32)
    v_len = np.maximum(1, (u_len * rnd.uniform(0.2, 1.0, 24)).astype(np.int32))
    u_flat, u_off, v_flat, v_off = I.ragged_operands(u_len, v_len, seed=72)
    items = [(u_flat[u_off[i]:u_off[i] + u_len[i]].copy(), v_flat[v_off[i]:v_off[i] + v_len[i]].copy())
             for i in range(len(u_len))]
    c = mp.mpdiv_init(0, flags=NTT, transform_cutoff=1024)
    try:
        mp.mpdiv_serve_start(c, pool_digits=1 << 22, max_batch=8, max_inflight=2)
        tickets = [mp.mpdiv_serve_submit(c, u, v) for u, v in items]
        got = []
        for t, (u, v) in zip(tickets, items):
            rc, q, r, st = mp.mpdiv_serve_poll(c, t, len(u), len(v), timeout_us=60_000_000)
            assert rc == mp.MPDIV_OK and st == 0
            got.append((q, r))
        mp.mpdiv_serve_stop(c)
    finally:
        mp.mpdiv_destroy(c)
    for (u, v), (q, r) in zip(items, got):
        qo, ro, _ = oracle.divmod_u32(u, v, len(u), len(v))
        assert (q == qo).all() and (r == ro).all()

"""Mixed-precision batches (persistent launch over a size-sorted queue, CUDA
graph replay), stress shapes at 2^18 bits, Theorem 2's delta = -1 path and the
block-size tuner, all bit-exact against the CPU oracle."""

import random

import numpy as np
import pytest

import oracle
import oracle.shinv_model as M
from paper_2606_06386_gb300 import inputs as I

from gpu_util import assert_same, ctx, dev, host_u32, oracle_uniform, run_uniform

pytestmark = pytest.mark.gpu


def _ragged(u_len, v_len, seed, c=None, edge=False):
    import torch
    import paper_2606_06386_gb300 as mp

    c = c or ctx()
    u_len = np.asarray(u_len, np.int32)
    v_len = np.asarray(v_len, np.int32)
    u_flat, u_off, v_flat, v_off = I.ragged_operands(u_len, v_len, seed=seed)
    if edge:  # some items with a dividend smaller than the divisor, zero digits, v = 1
        u_flat[u_off[0] : u_off[0] + u_len[0]] = 0
        v_flat[v_off[1] : v_off[1] + v_len[1]] = 0
        v_flat[v_off[1]] = 1
    q_len = u_len.copy()
    q_off = np.concatenate([[0], np.cumsum(q_len)[:-1]]).astype(np.int64)
    r_len = v_len.copy()
    r_off = np.concatenate([[0], np.cumsum(r_len)[:-1]]).astype(np.int64)
    n = len(u_len)
    T = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")  # noqa: E731
    q = torch.full((int(q_len.sum()),), -1, dtype=torch.int32, device="cuda:0")
    r = torch.full((int(r_len.sum()),), -1, dtype=torch.int32, device="cuda:0")
    st = torch.full((n,), -7, dtype=torch.int32, device="cuda:0")
    it = torch.full((n,), -1, dtype=torch.int32, device="cuda:0")
    args = (dev(u_flat), T(u_off, None), T(u_len, None), dev(v_flat), T(v_off, None), T(v_len, None), q,
            T(q_off, None), T(q_len, None), r, T(r_off, None), T(r_len, None), st, it)
    mp.mpdiv_batch_ragged(c, *args)
    torch.cuda.synchronize()
    Q, R, S, IT = host_u32(q), host_u32(r), st.cpu().numpy(), it.cpu().numpy()
    # replay with the same shapes (captured graph) must give the same digits
    q.fill_(-1)
    r.fill_(-1)
    mp.mpdiv_batch_ragged(c, *args)
    torch.cuda.synchronize()
    assert (host_u32(q) == Q).all() and (host_u32(r) == R).all()
    qo, ro, so, _ = oracle.divmod_ragged_u32(u_flat, u_off, u_len, v_flat, v_off, v_len, q_off, q_len, r_off, r_len)
    bad = [i for i in range(n) if S[i] != so[i]
           or not (Q[q_off[i]:q_off[i] + q_len[i]] == qo[q_off[i]:q_off[i] + q_len[i]]).all()
           or not (R[r_off[i]:r_off[i] + r_len[i]] == ro[r_off[i]:r_off[i] + r_len[i]]).all()]
    assert not bad, f"{len(bad)} of {n} items differ, first {bad[0]} (u {u_len[bad[0]]}, v {v_len[bad[0]]} digits)"
    return IT


PERSIST = 8  # MPDIV_FLAG_PERSISTENT_QUEUE


@pytest.mark.parametrize("warps", [0, 2, 4, 16])
def test_mixed_precision_persistent_launch(warps):
    # block shapes of the self-splitting kernel: untuned defaults (16-warp
    # blocks splitting to 8 and 4), and configured block sizes 2 and 4 (8-warp
    # blocks splitting to 4 and 2 warps) and 16 (16-warp blocks, no split)
    u_len, v_len = I.mixed_sizes(192, seed=I.SEED_BASE + 20)
    _ragged(u_len, v_len, seed=5, c=ctx(warps=warps, flags=PERSIST))


@pytest.mark.parametrize("warps", [0, 1, 4, 8])
def test_mixed_precision_by_size_class(warps):
    # the default ragged form: one plain launch per size class over its item
    # list, the launches forked as branches of one graph (configured block
    # sizes, or the untuned defaults per class)
    u_len, v_len = I.mixed_sizes(192, seed=I.SEED_BASE + 21)
    _ragged(u_len, v_len, seed=7, c=ctx(warps=warps))


@pytest.mark.parametrize("flags", [0, PERSIST])
@pytest.mark.parametrize("warps", [0, 2])
def test_mixed_small_shapes_and_edges(warps, flags):
    rnd = np.random.default_rng(3)
    u_len = rnd.integers(1, 300, size=200).astype(np.int32)
    v_len = np.maximum(1, (u_len * rnd.uniform(0.05, 1.3, size=200)).astype(np.int32))
    _ragged(u_len, v_len, seed=6, edge=True, c=ctx(warps=warps, flags=flags))


@pytest.mark.parametrize("flags", [0, PERSIST])
def test_mixed_with_2e19_bit_items(flags):
    # dividends up to 2^19 bits in the batch (five size classes)
    u_len = np.array([16384, 9000, 4096, 2048, 1000, 16384, 300, 8192], np.int32)
    v_len = np.array([8192, 100, 4000, 1024, 999, 16000, 150, 8192], np.int32)
    _ragged(u_len, v_len, seed=8, c=ctx(flags=flags))


def test_one_class_and_single_item_batches():
    # a batch of one size class (one launch, no fork) and a batch of one item
    u_len = np.full(40, 3000, np.int32)
    v_len = np.arange(1, 41, dtype=np.int32) * 70
    _ragged(u_len, v_len, seed=9)
    _ragged(np.array([5000], np.int32), np.array([77], np.int32), seed=10)


@pytest.mark.parametrize("variant", I.STRESS_VARIANTS)
def test_stress_2e18_bits(variant):
    U, V = I.stress(variant, n_items=24)
    Q, R, S, it = run_uniform(U, V)
    Qo, Ro, So = oracle_uniform(U, V)
    assert_same(Q, R, S, Qo, Ro, So)
    for i in range(len(U)):
        h = oracle.sig_len(U[i])
        kl = oracle.sig_len(V[i])
        if kl > 1 and h > kl:  # the Newton iteration runs: its count is the formula's
            vi = oracle.to_int(V[i])
            special = vi == (1 << (32 * (kl - 1))) or (h == kl and 2 * vi > (1 << (32 * h)))
            if not special:
                assert it[i] == M.refine_iterations(h, kl - 1)


def test_inject_lambda_keeps_results_exact():
    # shinv + 1 (Theorem 2's lambda = 1) must be absorbed by the delta = -1 correction
    import paper_2606_06386_gb300 as mp

    U, V, names = I.plain_1024(n_random=64)
    Q, R, S, _ = run_uniform(U, V, flags=mp.MPDIV_FLAG_INJECT_LAMBDA)
    Qo, Ro, So = oracle_uniform(U, V)
    assert_same(Q, R, S, Qo, Ro, So, names)


@pytest.mark.parametrize("cols", [3, 5, 7])
@pytest.mark.parametrize("warps", [1, 2, 4, 8, 16, 32])
def test_every_launch_shape_is_exact(warps, cols):
    U, V = I.sweep(2048, 1024, 16)
    Q, R, S, _ = run_uniform(U, V, warps=warps, cols=cols)
    Qo, Ro, So = oracle_uniform(U, V)
    assert_same(Q, R, S, Qo, Ro, So)
    # ragged small shapes with several strips and tails, at every strip width
    U = I.uniform_batch(16, 333, seed=5, stream=cols)
    V = I.uniform_batch(16, 131, seed=6, stream=cols)
    Q, R, S, _ = run_uniform(U, V, warps=warps, cols=cols)
    Qo, Ro, So = oracle_uniform(U, V)
    assert_same(Q, R, S, Qo, Ro, So)


@pytest.mark.parametrize(
    "n,kl,full,applies",
    [(2048, 1024, True, False),  # the last step's scratch does not fit: strip products
     (4096, 2048, True, True), (8192, 4096, True, True),  # 2:1 steps: square chunks
     (3000, 1000, True, True),  # near-square last step
     (5000, 2600, True, True), (6000, 3100, True, True), (2500, 2400, True, False),
     (8192, 4096, False, False)])  # clipped Newton steps have no full product to split
def test_karatsuba_products_are_exact(n, kl, full, applies):
    # one Karatsuba level on the Newton step's full product, forced on from 512
    # digits: the same digits as the oracle, and fewer digit products than the
    # strip products wherever it applies
    import paper_2606_06386_gb300 as mp

    U = I.uniform_batch(8, n, seed=n, stream=kl)
    V = I.uniform_batch(8, kl, seed=n + 1, stream=kl)
    flags = mp.MPDIV_FLAG_FULL_PRODUCTS if full else 0
    Q, R, S, _, Pk = run_uniform(U, V, flags=flags, kcut=512, products=True)
    Qo, Ro, So = oracle_uniform(U, V)
    assert_same(Q, R, S, Qo, Ro, So)
    _, _, _, _, Ps = run_uniform(U, V, flags=flags, kcut=-1, products=True)
    if applies:
        assert (Pk < Ps).all()
    else:
        assert (Pk == Ps).all()


def test_karatsuba_keeps_the_shifted_inverse_of_the_model():
    import torch
    import paper_2606_06386_gb300 as mp

    rnd = random.Random(41)
    vs = [rnd.getrandbits(32 * 1500) | (1 << (32 * 1500 - 1)) for _ in range(4)]
    V = np.stack([oracle.from_int(v, 1500) for v in vs])
    out = torch.zeros((4, 1600), dtype=torch.int32, device="cuda:0")
    it = torch.zeros(4, dtype=torch.int32, device="cuda:0")
    st = torch.full((4,), -1, dtype=torch.int32, device="cuda:0")
    h_t = torch.full((4,), 3000, dtype=torch.int32, device="cuda:0")
    mp.mpdiv_debug_shinv(ctx(flags=mp.MPDIV_FLAG_FULL_PRODUCTS, kcut=512), dev(V), h_t, out, it, st)
    torch.cuda.synchronize()
    O = host_u32(out)
    for i, v in enumerate(vs):
        assert st[i].item() == 0
        assert oracle.to_int(O[i]) == M.shinv(v, 3000, 1 << 32)


def test_autotune_picks_a_launch_shape():
    import paper_2606_06386_gb300 as mp

    c = mp.mpdiv_init(0)
    try:
        w = mp.mpdiv_autotune(c, 1024, 512, 1024)
        assert w in (1, 2, 4, 8, 16, 32)
        tw, tc, kc, _ = mp.mpdiv_tuning(c, 1000)
        assert tw == w and tc in (3, 5, 7) and kc in (0, 512, 1024, 2048)
    finally:
        mp.mpdiv_destroy(c)


@pytest.mark.parametrize("warps", [3, 6, 12, 40])
def test_configured_block_size_rounds_to_a_built_kernel(warps):
    # the kernels are built for 1, 2, 4, 8, 16 and 32 warps; another configured
    # block size runs the next one up (32 at most), with the same digits
    import paper_2606_06386_gb300 as mp

    U = I.uniform_batch(8, 700, seed=60, stream=warps)
    V = I.uniform_batch(8, 300, seed=61, stream=warps)
    Q, R, S, _ = run_uniform(U, V, warps=warps)
    Qo, Ro, So = oracle_uniform(U, V)
    assert_same(Q, R, S, Qo, Ro, So)
    assert mp.mpdiv_tuning(ctx(warps=warps), 700)[0] == min(32, 1 << (warps - 1).bit_length())


@pytest.mark.parametrize("flags", [0, PERSIST])
def test_bench_mixed_configuration_every_item(flags):
    # the mixed workload exactly as the benchmark runs it: 8192 divisions,
    # 2^15..2^18-bit dividends, shapes tuned per size class first, one call
    # (replayed as a graph) in either ragged form; every item against the oracle
    import paper_2606_06386_gb300 as mp

    c = mp.mpdiv_init(0, flags=flags)
    try:
        for n in (1024, 2048, 4096, 8192):
            mp.mpdiv_autotune(c, n, n // 2, 1024)
        u_len, v_len = I.mixed_sizes()
        _ragged(u_len, v_len, seed=I.SEED_BASE + 2, c=c)
    finally:
        mp.mpdiv_destroy(c)


def test_order_cache_follows_the_shape_list_exactly():
    # the cached size-sorted order is reused only for a shape list equal entry
    # for entry: shape lists with the same item count, the same lengths in
    # another order, and one divisor length changed, each in turn on one
    # context, every item against the oracle (and each replayed as a graph)
    import paper_2606_06386_gb300 as mp

    c = mp.mpdiv_init(0)
    try:
        rnd = np.random.default_rng(11)
        u_a = rnd.integers(200, 3000, size=96).astype(np.int32)
        v_a = np.maximum(1, (u_a * rnd.uniform(0.2, 1.0, size=96)).astype(np.int32)).astype(np.int32)
        u_b, v_b = u_a[::-1].copy(), v_a[::-1].copy()
        u_c, v_c = u_a.copy(), v_a.copy()
        v_c[50] = max(1, v_c[50] // 3)
        for k, (u_len, v_len) in enumerate([(u_a, v_a), (u_b, v_b), (u_a, v_a), (u_c, v_c), (u_a, v_a)]):
            _ragged(u_len, v_len, seed=30 + k, c=c)
    finally:
        mp.mpdiv_destroy(c)


def test_ragged_calls_on_two_streams_of_one_context():
    # two calls of one context on two streams, without a host wait between
    # them, with different shape lists: the context orders them on the GPU
    import torch
    import paper_2606_06386_gb300 as mp

    c = mp.mpdiv_init(0)
    try:
        sets = []
        for seed, n in ((61, 120), (62, 80)):
            rnd = np.random.default_rng(seed)
            u_len = rnd.integers(100, 2500, size=n).astype(np.int32)
            v_len = np.maximum(1, (u_len * rnd.uniform(0.2, 1.0, size=n)).astype(np.int32)).astype(np.int32)
            u_flat, u_off, v_flat, v_off = I.ragged_operands(u_len, v_len, seed=seed)
            q_len, r_len = u_len.copy(), v_len.copy()
            q_off = np.concatenate([[0], np.cumsum(q_len)[:-1]]).astype(np.int64)
            r_off = np.concatenate([[0], np.cumsum(r_len)[:-1]]).astype(np.int64)
            T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")  # noqa: E731
            q = torch.full((int(q_len.sum()),), -1, dtype=torch.int32, device="cuda:0")
            r = torch.full((int(r_len.sum()),), -1, dtype=torch.int32, device="cuda:0")
            st = torch.full((n,), -7, dtype=torch.int32, device="cuda:0")
            args = (dev(u_flat), T(u_off), T(u_len), dev(v_flat), T(v_off), T(v_len), q, T(q_off), T(q_len), r,
                    T(r_off), T(r_len), st)
            host = (u_flat, u_off, u_len, v_flat, v_off, v_len, q_off, q_len, r_off, r_len)
            sets.append((args, host, q, r, st))
        torch.cuda.synchronize()
        streams = [torch.cuda.Stream(), torch.cuda.Stream()]
        for _ in range(3):
            for (args, *_), s in zip(sets, streams):
                mp.mpdiv_batch_ragged(c, *args, stream=s)
        torch.cuda.synchronize()
        for args, host, q, r, st in sets:
            qo, ro, so, _ = oracle.divmod_ragged_u32(*host)
            assert (st.cpu().numpy() == so).all()
            Q, R = host_u32(q), host_u32(r)
            u_flat, u_off, u_len, v_flat, v_off, v_len, q_off, q_len, r_off, r_len = host
            for i in range(len(u_len)):
                assert (Q[q_off[i]:q_off[i] + q_len[i]] == qo[q_off[i]:q_off[i] + q_len[i]]).all(), i
                assert (R[r_off[i]:r_off[i] + r_len[i]] == ro[r_off[i]:r_off[i] + r_len[i]]).all(), i
    finally:
        mp.mpdiv_destroy(c)

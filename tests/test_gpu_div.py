"""Parity of the CUDA division path with the CPU oracle (bit-exact), through the C ABI."""

import random

import numpy as np
import pytest

import oracle
import oracle.shinv_model as M
import kernel_model as K
from paper_2606_06386_gb300 import inputs as I

from gpu_util import assert_same, dev, host_u32, oracle_uniform, run_uniform, ctx

pytestmark = pytest.mark.gpu
B = 1 << 32


def test_plain_1024_with_edge_cases():
    # 256 uniform (u: 1024 digits, v: 512 digits) + 16 seeded edge cases
    U, V, names = I.plain_1024()
    Q, R, S, it = run_uniform(U, V)
    Qo, Ro, So = oracle_uniform(U, V)
    assert_same(Q, R, S, Qo, Ro, So, names)
    # Newton iteration count = ceil(log2(h-k-1)) + 2 on the uniform items (h = 1024, k = 511)
    assert (it[:256] == M.refine_iterations(1024, 511)).all()


@pytest.mark.parametrize(
    "n,kl",
    [(1, 1), (2, 1), (2, 2), (3, 2), (5, 3), (8, 3), (40, 17), (97, 96), (230, 100), (300, 150), (333, 1),
     (512, 511), (700, 2), (1000, 999), (1500, 3)],
)
def test_small_and_ragged_shapes(n, kl):
    U = I.uniform_batch(24, n, seed=1000 + n, stream=kl)
    V = I.uniform_batch(24, kl, seed=2000 + n, stream=kl)
    Q, R, S, _ = run_uniform(U, V)
    Qo, Ro, So = oracle_uniform(U, V)
    assert_same(Q, R, S, Qo, Ro, So)


def test_full_size_2e18_bits():
    # 2^18-bit dividends, 2^17-bit divisors: every item against the oracle
    U, V = I.sweep(8192, 4096, 48)
    Q, R, S, it = run_uniform(U, V, qn=4097, rn=4096)
    Qo, Ro, So = oracle_uniform(U, V, 4097, 4096)
    assert_same(Q, R, S, Qo, Ro, So)
    assert (it == M.refine_iterations(8192, 4095)).all()


def test_special_values():
    n, kl = 64, 32
    rnd = random.Random(9)
    cases = []
    for u, v in [
        (0, 5), (0, 1), (7, 0), (123, 456), (rnd.getrandbits(32 * n), 1), (rnd.getrandbits(32 * n), 2),
        (rnd.getrandbits(32 * n), B - 1), (rnd.getrandbits(32 * n), B**31), (rnd.getrandbits(32 * n), B**31 + 1),
        (B**n - 1, B**kl - 1), (B**(n - 1), B**(kl - 1)), (B**kl - 1, B**kl - 1), (B**kl - 2, B**kl - 1),
        ((B**kl - 1) * (B**kl - 1), B**kl - 1), (B**32 * 3, (B**32) // 2 + 1), (B**32 - 1, B**31 * 2**31),
        (rnd.getrandbits(32 * n), 1 << (32 * kl - 1)), (rnd.getrandbits(32 * n), (1 << (32 * kl - 1)) + 1),
    ]:
        cases.append((u, v))
    U = np.stack([oracle.from_int(u, n) for u, _ in cases])
    V = np.stack([oracle.from_int(v, kl) for _, v in cases])
    Q, R, S, _ = run_uniform(U, V)
    Qo, Ro, So = oracle_uniform(U, V)
    assert_same(Q, R, S, Qo, Ro, So)
    assert S[2] == 1  # v == 0


def test_shinv_within_theorem2_and_equal_to_the_models():
    # parity: the GPU's shifted inverse against the Knuth oracle's
    # floor(B^h / v), within Theorem 2's lambda in {0, 1} with the paper's full
    # products and within -1..+2 with the clipped Newton steps (readings 14-15).
    # Beside it, digit for digit: with full products Algorithm 1 as printed
    # (the oracle's model); by default the model of the kernel's clipped design
    # (tests/kernel_model.py), a check of the design, not of parity.
    import torch
    import paper_2606_06386_gb300 as mp

    rnd = random.Random(31)
    vs, hs = [], []
    for _ in range(60):
        kl = rnd.randint(2, 40)
        v = rnd.getrandbits(32 * kl) | (1 << (32 * kl - 1 - rnd.randint(0, 31)))
        h = rnd.randint(kl, 90)
        vs.append(v)
        hs.append(h)
    V = np.stack([oracle.from_int(v, 40) for v in vs])
    out = torch.zeros((len(vs), 100), dtype=torch.int32, device="cuda:0")
    it = torch.zeros(len(vs), dtype=torch.int32, device="cuda:0")
    st = torch.full((len(vs),), -1, dtype=torch.int32, device="cuda:0")
    h_t = torch.tensor(hs, dtype=torch.int32, device="cuda:0")
    exact = [oracle.to_int(oracle.shinv_u32(oracle.from_int(v, 40), h)) for v, h in zip(vs, hs)]
    for flags, clip in ((0, True), (mp.MPDIV_FLAG_FULL_PRODUCTS, False)):
        out.zero_()
        st.fill_(-1)
        mp.mpdiv_debug_shinv(ctx(flags=flags, cols=3), dev(V), h_t, out, it, st)
        torch.cuda.synchronize()
        O = host_u32(out)
        S = st.cpu().numpy()
        I_ = it.cpu().numpy()
        for i, (v, h) in enumerate(zip(vs, hs)):
            assert S[i] == 0
            s_gpu = oracle.to_int(O[i])
            assert s_gpu - exact[i] in ((-1, 0, 1, 2) if clip else (0, 1)), (i, v, h, flags)
            if clip:
                tr = K.KTrace()
                assert s_gpu == K.shinv(v, h, B, tr, True), (i, v, h)
            else:
                tr = M.Trace()
                assert s_gpu == M.shinv(v, h, B, tr), (i, v, h)
            assert I_[i] == tr.iterations


@pytest.mark.parametrize("full", [False, True])
@pytest.mark.parametrize("n,kl", [(64, 32), (300, 37), (1024, 512), (97, 96), (500, 2)])
def test_product_counter_equals_model(n, kl, full):
    # the kernel's count of algorithmic digit products equals Algorithms 1-3
    # as printed (the oracle's model) with the paper's full products, and the
    # model of the kernel's clipped design (tests/kernel_model.py) by default;
    # both counts are pinned to brute force on the CPU
    import torch
    import paper_2606_06386_gb300 as mp

    U = I.uniform_batch(4, n, seed=77, stream=n)
    V = I.uniform_batch(4, kl, seed=78, stream=kl)
    q = torch.zeros((4, n), dtype=torch.int32, device="cuda:0")
    r = torch.zeros((4, kl), dtype=torch.int32, device="cuda:0")
    st = torch.zeros(4, dtype=torch.int32, device="cuda:0")
    pr = torch.zeros(4, dtype=torch.int64, device="cuda:0")
    mp.mpdiv_batch(ctx(flags=mp.MPDIV_FLAG_FULL_PRODUCTS if full else 0, cols=3), dev(U), dev(V), q, r, st, None, pr)
    torch.cuda.synchronize()
    P = pr.cpu().numpy()
    for i in range(4):
        u, v = oracle.to_int(U[i]), oracle.to_int(V[i])
        if full:
            tr = M.Trace()
            M.div(u, v, B, tr)
        else:
            tr = K.KTrace()
            assert K.div_clipped(u, v, B, tr, clip_step=True) == divmod(u, v)
        assert P[i] == tr.digit_products()


def test_full_products_mode_is_exact():
    import paper_2606_06386_gb300 as mp

    U, V, names = I.plain_1024(n_random=64)
    Q, R, S, _ = run_uniform(U, V, flags=mp.MPDIV_FLAG_FULL_PRODUCTS)
    Qo, Ro, So = oracle_uniform(U, V)
    assert_same(Q, R, S, Qo, Ro, So, names)
    U, V = I.sweep(8192, 4096, 8)
    Q, R, S, _ = run_uniform(U, V, flags=mp.MPDIV_FLAG_FULL_PRODUCTS)
    Qo, Ro, So = oracle_uniform(U, V)
    assert_same(Q, R, S, Qo, Ro, So)


@pytest.mark.parametrize("n", [1, 7, 100, 1024, 3000, 8192, 16384])
def test_multiplication_cost_unit(n):
    # (u v) mod B^n, the product of Fig. 3 that the cost model counts in
    import torch
    import paper_2606_06386_gb300 as mp

    U = I.uniform_batch(6, n, seed=90, stream=n)
    V = I.uniform_batch(6, n, seed=91, stream=n)
    out = torch.zeros((6, n), dtype=torch.int32, device="cuda:0")
    mp.mpdiv_mul_batch(ctx(), dev(U), dev(V), out)
    torch.cuda.synchronize()
    O = host_u32(out)
    for i in range(6):
        assert oracle.to_int(O[i]) == (oracle.to_int(U[i]) * oracle.to_int(V[i])) % (B**n)


@pytest.mark.parametrize("bits", [b for b, _ in I.PAPER_TABLE])
def test_paper_table1_datasets(bits):
    # the paper's datasets (u of M-2 64-bit digits, v of random precision in
    # [2, M/2] 64-bit digits, zero-padded), 2^13..2^18 bits: every item exact,
    # and the Refine count of Algorithm 1 at each item's own precisions
    n_items = 64 if bits <= 1 << 16 else 32
    U, V, v_len = I.paper_workload(bits, n_items)
    Q, R, S, it = run_uniform(U, V)
    Qo, Ro, So = oracle_uniform(U, V)
    assert_same(Q, R, S, Qo, Ro, So)
    h = U.shape[1]
    assert all(it[i] == M.refine_iterations(h, int(v_len[i]) - 1) for i in range(n_items))


@pytest.mark.parametrize("kind", ["half", "paper", "short"])
def test_2e19_bits_beyond_the_paper(kind):
    # 2^19-bit dividends (16384 digits), which the paper's A100 could not hold
    # in shared memory: half-length divisors, the paper's random precisions,
    # and a 64-digit divisor; every item exact
    import paper_2606_06386_gb300 as mp

    if kind == "half":
        U, V = I.sweep(16384, 8192, 6)
    elif kind == "paper":
        U, V, _ = I.paper_workload(1 << 19, 6)
    else:
        U = I.uniform_batch(6, 16384, seed=19, stream=1)
        V = I.uniform_batch(6, 64, seed=19, stream=2)
    Q, R, S, it = run_uniform(U, V)
    Qo, Ro, So = oracle_uniform(U, V)
    assert_same(Q, R, S, Qo, Ro, So)
    # the paper's full products do not fit a block's shared memory at this size
    import torch

    q = torch.zeros((1, U.shape[1]), dtype=torch.int32, device="cuda:0")
    r = torch.zeros((1, V.shape[1]), dtype=torch.int32, device="cuda:0")
    st = torch.zeros(1, dtype=torch.int32, device="cuda:0")
    with pytest.raises(mp.MpdivError) as e:
        mp.mpdiv_batch(ctx(flags=mp.MPDIV_FLAG_FULL_PRODUCTS), dev(U[:1]), dev(V[:1]), q, r, st)
    assert e.value.code == mp.MPDIV_EUNSUPPORTED


@pytest.mark.parametrize("cols", [3, 5, 7])
def test_strip_fold_carry_ripple(cols):
    # operands built so that every strip's two overflow digits, added to the
    # next strip's first two columns, carry out of them: u is all ones except
    # digits 1, 1 at each strip start (strips of 32 * cols columns), v = B - 1.
    # Each strip's low two digits are then B^2 - 1 and the previous strip's
    # overflow is B - 2, so the rare ripple path runs at every boundary.
    import torch
    import paper_2606_06386_gb300 as mp

    n = 1000
    w = 32 * cols
    u = np.full(n, 0xFFFFFFFF, np.uint32)
    for s in range(1, n // w + 1):
        if s * w + 1 < n:
            u[s * w] = u[s * w + 1] = 1
    v = np.zeros(n, np.uint32)
    v[0] = 0xFFFFFFFF
    out = torch.zeros((2, n), dtype=torch.int32, device="cuda:0")
    U = np.stack([u, v])
    V = np.stack([v, u])  # both operand roles
    mp.mpdiv_mul_batch(ctx(cols=cols), dev(U), dev(V), out)
    torch.cuda.synchronize()
    O = host_u32(out)
    want = (oracle.to_int(u) * oracle.to_int(v)) % (B**n)
    assert oracle.to_int(O[0]) == want and oracle.to_int(O[1]) == want


def test_multiply_pipe_microbenchmark():
    # the roofline's measured ceiling: digit products of the strip multiply's
    # idiom and plain 32-bit multiply-adds on every SM; each digit product
    # takes two multiply results (low and high word)
    import paper_2606_06386_gb300 as mp

    c = ctx()
    prod, ms0 = mp.mpdiv_measure_peak(c, 0, 1024)
    imad, ms1 = mp.mpdiv_measure_peak(c, 1, 1024)
    strip, ms2 = mp.mpdiv_measure_peak(c, 2, 2)
    assert ms0 > 0 and ms1 > 0 and ms2 > 0
    assert 0 < prod < imad
    # the inner loop also loads its digits and rotates its window: below the idiom
    assert 0 < strip < 1.05 * prod
    assert imad < 2 * 64 * 152 * 2.1e9  # far below nonsense: 64 multiply results/clk/SM at most twice over


@pytest.mark.parametrize("offset,n,kl", [(1, 1024, 512), (2, 2048, 1024), (3, 4096, 2048), (4, 1027, 515), (1, 8192, 4096)])
def test_operand_and_result_alignment(offset, n, kl):
    # operand and result rows that start off a 16-byte boundary (a base
    # pointer offset by 1..3 digits, or an odd row length): the 16-byte
    # staging must fall back to digit-by-digit copies or peel the unaligned
    # head and tail, with the same digits
    import torch
    import paper_2606_06386_gb300 as mp

    k = 8
    U, V = I.sweep(n, kl, k)
    qn, rn = n - kl + 1, kl

    def slab(rows, cols, src=None):
        t = torch.full((offset + rows * cols + 3,), -1, dtype=torch.int32, device="cuda:0")
        v = t[offset : offset + rows * cols].view(rows, cols)
        if src is not None:
            v.copy_(dev(src))
        return t, v

    _, u = slab(k, n, U)
    _, v = slab(k, kl, V)
    qb, q = slab(k, qn)
    rb, r = slab(k, rn)
    st = torch.full((k,), -7, dtype=torch.int32, device="cuda:0")
    mp.mpdiv_batch(ctx(), u, v, q, r, st)
    torch.cuda.synchronize()
    Qo, Ro, So = oracle_uniform(U, V, qn, rn)
    assert_same(host_u32(q), host_u32(r), st.cpu().numpy(), Qo, Ro, So)
    # nothing written outside the result rows
    assert (qb[:offset] == -1).all() and (qb[offset + k * qn :] == -1).all()
    assert (rb[:offset] == -1).all() and (rb[offset + k * rn :] == -1).all()


def test_bench_sweep_configuration_sampled():
    # the benchmark's own workload and launch configuration: the four sweep
    # sizes at their full batch sizes (8192/4096/2048/1024 divisions), shapes
    # picked by the tuner as bench.py does, one plain launch per size; 64
    # sampled items per size against the oracle, every status zero
    import torch
    import paper_2606_06386_gb300 as mp

    c = mp.mpdiv_init(0)
    try:
        rnd = np.random.default_rng(2024)
        for n, kl, b in I.SWEEP:
            U, V = I.sweep(n, kl, b)
            mp.mpdiv_autotune(c, n, kl, b)
            q = torch.empty((b, n - kl + 1), dtype=torch.int32, device="cuda:0")
            r = torch.empty((b, kl), dtype=torch.int32, device="cuda:0")
            st = torch.full((b,), -7, dtype=torch.int32, device="cuda:0")
            mp.mpdiv_batch(c, dev(U), dev(V), q, r, st)
            torch.cuda.synchronize()
            assert (st == 0).all()
            idx = np.sort(rnd.choice(b, 64, replace=False))
            Qo, Ro, So = oracle_uniform(U[idx], V[idx], n - kl + 1, kl)
            assert_same(host_u32(q)[idx], host_u32(r)[idx], st.cpu().numpy()[idx], Qo, Ro, So)
    finally:
        mp.mpdiv_destroy(c)


@pytest.mark.parametrize("regs", [64, 128])
@pytest.mark.parametrize("n,warps,cols", [(2048, 4, 3), (4096, 4, 5), (8192, 8, 5), (8192, 16, 7)])
def test_register_budgets_of_the_plain_kernel(tmp_path, monkeypatch, n, warps, cols, regs):
    # the plain kernel's 64- and 128-register builds (the latter for 4, 8 and
    # 16 warps), chosen through a tuning file, give the oracle's digits
    import paper_2606_06386_gb300 as mp

    f = tmp_path / "tune.txt"
    f.write_text(f"{n} {warps} {cols} 0 {regs}\n")
    monkeypatch.setenv("MPDIV_TUNE_FILE", str(f))
    c = mp.mpdiv_init(0)
    monkeypatch.delenv("MPDIV_TUNE_FILE")
    try:
        assert mp.mpdiv_tuning(c, n) == (warps, cols, 0, regs)
        import torch

        U, V = I.sweep(n, n // 2, 24)
        q = torch.zeros((24, n // 2 + 1), dtype=torch.int32, device="cuda:0")
        r = torch.zeros((24, n // 2), dtype=torch.int32, device="cuda:0")
        st = torch.full((24,), -1, dtype=torch.int32, device="cuda:0")
        mp.mpdiv_batch(c, dev(U), dev(V), q, r, st)
        torch.cuda.synchronize()
        Qo, Ro, So = oracle_uniform(U, V, n // 2 + 1, n // 2)
        assert_same(host_u32(q), host_u32(r), st.cpu().numpy(), Qo, Ro, So)
    finally:
        mp.mpdiv_destroy(c)


@pytest.mark.parametrize("n,kl", [(1024, 512), (2048, 1024), (4096, 2048), (3000, 1100)])
def test_fit_pass_and_retry_pass(n, kl):
    # the plain launch sizes its shared memory for the batch's digit counts
    # (more blocks per SM); items whose effective divisor (or dividend) is
    # shorter than its buffer need a larger plan and are divided by the retry
    # pass: here a quarter of the divisors and some dividends have leading
    # zero digits. Every status is 0 (no item is left behind) and every digit
    # the oracle's, with the default shapes and with every strip width.
    U = I.uniform_batch(64, n, seed=90 + n, stream=kl)
    V = I.uniform_batch(64, kl, seed=91 + n, stream=kl)
    rnd = np.random.default_rng(n + kl)
    for i in range(0, 64, 4):
        V[i, rnd.integers(1, kl):] = 0  # prec(v) < kl
        if V[i].max() == 0:
            V[i, 0] = 3
    for i in range(1, 64, 8):
        U[i, rnd.integers(kl, n):] = 0  # prec(u) < n
    Qo, Ro, So = oracle_uniform(U, V)
    for cols in (0, 3, 5, 7):
        Q, R, S, _ = run_uniform(U, V, cols=cols)
        assert (S == 0).all()
        assert_same(Q, R, S, Qo, Ro, So)


@pytest.mark.parametrize("n,kl,warps,cols,items", [(1024, 512, 2, 3, 4096), (1024, 512, 1, 3, 4096),
                                                    (4096, 2048, 4, 5, 1024)])
def test_retry_pass_on_a_batch_of_several_waves(n, kl, warps, cols, items):
    # a batch of several waves, where the plain launch runs as a fit pass and
    # a retry pass (checked through mpdiv_batch_launches): the divisors have
    # random lengths below their buffers, as in the paper's datasets, so most
    # items need the larger plan and the retry pass divides them, one block
    # per item; every status 0 and every digit the oracle's
    import paper_2606_06386_gb300 as mp

    c = ctx(warps=warps, cols=cols)  # shapes whose fit pass holds more blocks per SM
    assert mp.mpdiv_batch_launches(c, items, n, kl) == 2
    U = I.uniform_batch(items, n, seed=95 + n, stream=kl)
    V = I.uniform_batch(items, kl, seed=96 + n, stream=kl)
    rnd = np.random.default_rng(n * 7 + kl)
    for i in range(items):
        if i % 8:  # one item in eight keeps its full length (the fit pass divides it)
            V[i, rnd.integers(1, kl):] = 0
            if V[i].max() == 0:
                V[i, 0] = 5
    Q, R, S, _ = run_uniform(U, V, warps=warps, cols=cols)
    assert (S == 0).all()
    Qo, Ro, So = oracle_uniform(U, V)
    assert_same(Q, R, S, Qo, Ro, So)

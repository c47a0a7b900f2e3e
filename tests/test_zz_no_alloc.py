"""The allocation-free entry point, mpdiv_batch_ragged_noalloc.

It serves callers that cannot allocate device memory at the point they divide
(a pool that owns the whole device, an allocator closed after start-up). Its
queue lives in a fixed scratch array inside the library, shared by every call;
this test checks, on two calls in a row with different batches, that its
results equal those of the context-based entry point mpdiv_batch_ragged digit
for digit (the tolerance of every division test here is zero), which also
shows the second call starts from a clean queue. The first items of each batch
(among them a dividend shorter than its divisor and a power-of-two divisor)
are also checked against the Knuth oracle directly, since both entry points
run the same division code. The file name makes pytest collect it last.
"""

import numpy as np
import pytest

import oracle
from paper_2606_06386_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _batch(n, seed):
    import torch

    rnd = np.random.default_rng(seed)
    u_len = rnd.integers(1, 1500, size=n).astype(np.int32)
    v_len = np.clip((u_len * rnd.uniform(0.1, 1.2, size=n)).astype(np.int32), 1, 1500).astype(np.int32)
    u_len[0], v_len[0] = 40, 90  # u < v: q = 0, r = u
    u_flat, u_off, v_flat, v_off = I.ragged_operands(u_len, v_len, seed=seed)
    v_flat[v_off[1] : v_off[1] + v_len[1]] = 0  # item 1: v = 2^(32 (v_len - 1) + 13)
    v_flat[v_off[1] + v_len[1] - 1] = 1 << 13
    q_len, r_len = u_len.copy(), v_len.copy()
    q_off = np.concatenate([[0], np.cumsum(q_len)[:-1]]).astype(np.int64)
    r_off = np.concatenate([[0], np.cumsum(r_len)[:-1]]).astype(np.int64)
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")  # noqa: E731
    ins = dict(u=d(u_flat.view(np.int32)), u_off=d(u_off), u_len=d(u_len), v=d(v_flat.view(np.int32)),
               v_off=d(v_off), v_len=d(v_len), q_off=d(q_off), q_len=d(q_len), r_off=d(r_off), r_len=d(r_len))
    host = dict(u_flat=u_flat, u_off=u_off, u_len=u_len, v_flat=v_flat, v_off=v_off, v_len=v_len, q_off=q_off,
                q_len=q_len, r_off=r_off, r_len=r_len)
    return ins, int(q_len.sum()), int(r_len.sum()), n, torch.from_numpy(u_len), host


def _outs(nq, nr, n):
    import torch

    return (torch.full((nq,), -1, dtype=torch.int32, device="cuda:0"),
            torch.full((nr,), -1, dtype=torch.int32, device="cuda:0"),
            torch.full((n,), -7, dtype=torch.int32, device="cuda:0"))


def test_noalloc_matches_context_entry_point_on_two_calls():
    import torch
    import paper_2606_06386_gb300 as mp

    ctx = mp.mpdiv_init(0)
    try:
        for seed, n in ((41, 150), (42, 97)):  # two calls in a row, different batches
            ins, nq, nr, n, u_len_host, host = _batch(n, seed)
            q0, r0, s0 = _outs(nq, nr, n)
            mp.mpdiv_batch_ragged(ctx, ins["u"], ins["u_off"], ins["u_len"], ins["v"], ins["v_off"], ins["v_len"],
                                  q0, ins["q_off"], ins["q_len"], r0, ins["r_off"], ins["r_len"], s0)
            q1, r1, s1 = _outs(nq, nr, n)
            rc = mp.mpdiv_batch_ragged_noalloc(ins["u"], ins["u_off"], ins["u_len"], ins["v"], ins["v_off"],
                                               ins["v_len"], q1, ins["q_off"], ins["q_len"], r1, ins["r_off"],
                                               ins["r_len"], s1, u_len_host)
            assert rc == mp.MPDIV_OK
            torch.cuda.synchronize()
            assert (s0 == 0).all()
            assert torch.equal(s1, s0)
            assert torch.equal(q1, q0)
            assert torch.equal(r1, r0)
            # the first 20 items against the Knuth oracle
            k = 20
            qo, ro, so, _ = oracle.divmod_ragged_u32(
                host["u_flat"], host["u_off"][:k], host["u_len"][:k], host["v_flat"], host["v_off"][:k],
                host["v_len"][:k], host["q_off"][:k], host["q_len"][:k], host["r_off"][:k], host["r_len"][:k])
            Q1 = q1.cpu().numpy().view(np.uint32)
            R1 = r1.cpu().numpy().view(np.uint32)
            S1 = s1.cpu().numpy()
            for i in range(k):
                qa, ql = host["q_off"][i], host["q_len"][i]
                ra, rl = host["r_off"][i], host["r_len"][i]
                assert S1[i] == so[i] == 0
                assert (Q1[qa : qa + ql] == qo[qa : qa + ql]).all(), i
                assert (R1[ra : ra + rl] == ro[ra : ra + rl]).all(), i
            assert not Q1[host["q_off"][0] : host["q_off"][0] + host["q_len"][0]].any()  # u < v: q = 0
    finally:
        mp.mpdiv_destroy(ctx)


def test_noalloc_rejects_more_items_than_its_scratch_holds():
    import torch
    import paper_2606_06386_gb300 as mp

    n = mp.MPDIV_NOALLOC_MAX_ITEMS + 1
    z64 = torch.zeros(n, dtype=torch.int64, device="cuda:0")
    o32 = torch.ones(n, dtype=torch.int32, device="cuda:0")
    digits = torch.ones(n, dtype=torch.int32, device="cuda:0")
    st = torch.zeros(n, dtype=torch.int32, device="cuda:0")
    rc = mp.mpdiv_batch_ragged_noalloc(digits, z64, o32, digits, z64, o32, digits, z64, o32, digits, z64, o32, st,
                                       torch.ones(n, dtype=torch.int32))
    assert rc == mp.MPDIV_EUNSUPPORTED

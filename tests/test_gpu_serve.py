"""The continuous-batching server: every result is the same alone and in a
mix with others, and equals the oracle's."""

import numpy as np
import pytest

import oracle
from paper_2606_06386_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _mix(n, seed):
    u_len, v_len = I.mixed_sizes(n, seed=seed)
    u_len = np.minimum(u_len, 2048)
    v_len = np.minimum(v_len, u_len)
    u_flat, u_off, v_flat, v_off = I.ragged_operands(u_len, v_len, seed=seed)
    items = [(u_flat[u_off[i]:u_off[i] + u_len[i]].copy(), v_flat[v_off[i]:v_off[i] + v_len[i]].copy())
             for i in range(n)]
    return items


def test_results_alone_equal_results_in_the_mix():
    import paper_2606_06386_gb300 as mp

    items = _mix(48, seed=I.SEED_BASE + 30)
    c = mp.mpdiv_init(0)
    try:
        mp.mpdiv_serve_start(c, pool_digits=1 << 22, max_batch=16, max_inflight=3)
        alone = []
        for u, v in items[:8]:  # one at a time: each request is a batch of its own
            t = mp.mpdiv_serve_submit(c, u, v)
            rc, q, r, st = mp.mpdiv_serve_poll(c, t, len(u), len(v), timeout_us=30_000_000)
            assert rc == mp.MPDIV_OK and st == 0
            alone.append((q, r))
        tickets = [mp.mpdiv_serve_submit(c, u, v) for u, v in items]  # all at once: mixed batches
        mixed = []
        for t, (u, v) in zip(tickets, items):
            rc, q, r, st = mp.mpdiv_serve_poll(c, t, len(u), len(v), timeout_us=30_000_000)
            assert rc == mp.MPDIV_OK and st == 0
            mixed.append((q, r))
        completed, launches, batched = mp.mpdiv_serve_stats(c)
        assert completed == 56 and launches >= 8 + 3
        mp.mpdiv_serve_stop(c)
    finally:
        mp.mpdiv_destroy(c)
    for i in range(8):
        assert (alone[i][0] == mixed[i][0]).all() and (alone[i][1] == mixed[i][1]).all()
    for (u, v), (q, r) in zip(items, mixed):
        qo, ro, _ = oracle.divmod_u32(u, v, len(u), len(v))
        assert (q == qo).all() and (r == ro).all()


def test_replay_of_a_poisson_stream():
    import paper_2606_06386_gb300 as mp

    n = 300
    u_len, v_len = I.mixed_sizes(n, seed=I.SEED_BASE + 31)
    u_len = np.minimum(u_len, 2048).astype(np.int32)
    v_len = np.minimum(v_len, u_len).astype(np.int32)
    u_flat, u_off, v_flat, v_off = I.ragged_operands(u_len, v_len, seed=31)
    arr = (I.poisson_arrivals(n, 20000.0, seed=31) * 1e9).astype(np.int64)
    q_len, r_len = u_len.copy(), v_len.copy()
    q_off = np.concatenate([[0], np.cumsum(q_len)[:-1]]).astype(np.int64)
    r_off = np.concatenate([[0], np.cumsum(r_len)[:-1]]).astype(np.int64)
    q = np.zeros(int(q_len.sum()), np.uint32)
    r = np.zeros(int(r_len.sum()), np.uint32)
    st = np.full(n, -9, np.int32)
    lat = np.zeros(n, np.int64)
    c = mp.mpdiv_init(0)
    try:
        mp.mpdiv_serve_start(c, pool_digits=1 << 22, max_batch=64, max_inflight=3)
        mp.mpdiv_serve_replay(c, arr, u_flat, u_off, u_len, v_flat, v_off, v_len, q, q_off, q_len, r, r_off, r_len,
                              st, lat)
        mp.mpdiv_serve_stop(c)
    finally:
        mp.mpdiv_destroy(c)
    assert (st == 0).all() and (lat > 0).all()
    qo, ro, so, _ = oracle.divmod_ragged_u32(u_flat, u_off, u_len, v_flat, v_off, v_len, q_off, q_len, r_off, r_len)
    assert (q == qo).all() and (r == ro).all()

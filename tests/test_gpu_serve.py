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


@pytest.mark.parametrize("device_pools", [False, True], ids=["mapped_rings", "device_pools"])
def test_replay_of_a_poisson_stream(device_pools):
    # both places for operands and results: the pinned host rings the kernels
    # use directly (the default) and device-resident pools (copies per batch)
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
    ph = np.full(3 * n, -5, np.int64)
    c = mp.mpdiv_init(0)
    try:
        mp.mpdiv_serve_start(c, pool_digits=1 << 22, max_batch=64, max_inflight=3,
                             flags=mp.MPDIV_SERVE_DEVICE_POOLS if device_pools else 0)
        mp.mpdiv_serve_replay(c, arr, u_flat, u_off, u_len, v_flat, v_off, v_len, q, q_off, q_len, r, r_off, r_len,
                              st, lat, ph)
        mp.mpdiv_serve_stop(c)
    finally:
        mp.mpdiv_destroy(c)
    assert (st == 0).all() and (lat > 0).all()
    # the phases (submit delay, queue wait, run) are ordered and add up to the latency
    ph = ph.reshape(n, 3)
    assert (ph >= 0).all() and (ph.sum(axis=1) == lat).all()
    qo, ro, so, _ = oracle.divmod_ragged_u32(u_flat, u_off, u_len, v_flat, v_off, v_len, q_off, q_len, r_off, r_len)
    assert (q == qo).all() and (r == ro).all()


def _submit_retry(mp, c, u, v, tries=20000):
    import time

    for _ in range(tries):
        try:
            return mp.mpdiv_serve_submit(c, u, v)
        except mp.MpdivError as e:
            if e.code != mp.MPDIV_EBUSY:
                raise
            time.sleep(0.0005)
    raise AssertionError("the server never admitted the request")


def _wait_completed(mp, c, n, seconds=30.0):
    import time

    t0 = time.time()
    while mp.mpdiv_serve_stats(c)[0] < n:
        assert time.time() - t0 < seconds, "requests did not complete"
        time.sleep(0.001)


def test_ticket_table_and_admission_limits():
    # a finished ticket is collected once; at most 1024 finished tickets (here,
    # with max_pending 4) wait unpolled, after which submit is refused until
    # the oldest of them is collected; stop keeps results pollable, refuses
    # new work, and a stopped server can be started again
    import paper_2606_06386_gb300 as mp

    u = np.array([7, 1], np.uint32)  # 2^32 + 7
    v = np.array([3], np.uint32)
    q_want, r_want = divmod((1 << 32) + 7, 3)
    c = mp.mpdiv_init(0)
    try:
        mp.mpdiv_serve_start(c, pool_digits=1 << 20, max_batch=64, max_inflight=4, max_pending=4)
        t = _submit_retry(mp, c, u, v)
        rc, q, r, st = mp.mpdiv_serve_poll(c, t, 2, 1, timeout_us=30_000_000)
        assert rc == mp.MPDIV_OK and st == 0 and oracle.to_int(q) == q_want and r[0] == r_want
        with pytest.raises(mp.MpdivError) as e:
            mp.mpdiv_serve_poll(c, t, 2, 1)
        assert e.value.code == mp.MPDIV_EINVAL
        tickets = [_submit_retry(mp, c, u, v) for _ in range(1024)]
        _wait_completed(mp, c, 1 + 1024)
        with pytest.raises(mp.MpdivError) as e:
            mp.mpdiv_serve_submit(c, u, v)  # its slot still holds an unpolled result
        assert e.value.code == mp.MPDIV_EBUSY
        rc, q, r, st = mp.mpdiv_serve_poll(c, tickets[0], 2, 1)
        assert rc == mp.MPDIV_OK and oracle.to_int(q) == q_want
        tickets.append(mp.mpdiv_serve_submit(c, u, v))
        mp.mpdiv_serve_stop(c)
        with pytest.raises(mp.MpdivError) as e:
            mp.mpdiv_serve_submit(c, u, v)
        assert e.value.code == mp.MPDIV_ESTATE
        for tk in tickets[1:]:
            rc, q, r, st = mp.mpdiv_serve_poll(c, tk, 2, 1, timeout_us=30_000_000)
            assert rc == mp.MPDIV_OK and st == 0 and oracle.to_int(q) == q_want and r[0] == r_want
        mp.mpdiv_serve_start(c, pool_digits=1 << 20)
        t = _submit_retry(mp, c, u, v)
        rc, q, r, st = mp.mpdiv_serve_poll(c, t, 2, 1, timeout_us=30_000_000)
        assert rc == mp.MPDIV_OK and oracle.to_int(q) == q_want
        mp.mpdiv_serve_stop(c)
    finally:
        mp.mpdiv_destroy(c)


def test_concurrent_polls_of_one_ticket():
    # pollers race for a finished ticket without the server lock: exactly one
    # collects it, the others find it gone
    import threading

    import paper_2606_06386_gb300 as mp

    items = _mix(16, seed=I.SEED_BASE + 32)
    c = mp.mpdiv_init(0)
    try:
        mp.mpdiv_serve_start(c, pool_digits=1 << 22)
        for u, v in items:
            n0 = mp.mpdiv_serve_stats(c)[0]
            t = _submit_retry(mp, c, u, v)
            _wait_completed(mp, c, n0 + 1)
            got, gone = [], []

            def poll():
                try:
                    rc, q, r, st = mp.mpdiv_serve_poll(c, t, len(u), len(v))
                    if rc == mp.MPDIV_OK:
                        got.append((q, r, st))
                except mp.MpdivError as e:
                    gone.append(e.code)

            ths = [threading.Thread(target=poll) for _ in range(8)]
            for th in ths:
                th.start()
            for th in ths:
                th.join()
            assert len(got) == 1 and len(gone) == 7 and set(gone) == {mp.MPDIV_EINVAL}
            qo, ro, _ = oracle.divmod_u32(u, v, len(u), len(v))
            assert (got[0][0] == qo).all() and (got[0][1] == ro).all() and got[0][2] == 0
        mp.mpdiv_serve_stop(c)
    finally:
        mp.mpdiv_destroy(c)


@pytest.mark.parametrize("flags", [0, 8])
def test_serving_full_size_mix(flags):
    # the full size range of the serving workload (2^15..2^18-bit dividends,
    # divisors of 0.25..1.0 of their length) plus a few 2^19-bit requests and
    # degenerate ones (u < v, v = 1), in both launch forms of a batch (plain
    # launch with the class's shape; flag 8, MPDIV_FLAG_PERSISTENT_QUEUE: the
    # self-splitting persistent kernel): every result equals the oracle's
    import paper_2606_06386_gb300 as mp

    n = 96
    u_len, v_len = I.mixed_sizes(n, seed=I.SEED_BASE + 32)
    u_len = u_len.astype(np.int32)
    v_len = v_len.astype(np.int32)
    u_len[:3] = 16384
    v_len[:3] = [8192, 64, 16384]
    u_len[3], v_len[3] = 100, 200  # u shorter than v: q = 0, r = u
    u_flat, u_off, v_flat, v_off = I.ragged_operands(u_len, v_len, seed=32)
    v_flat[v_off[4] : v_off[4] + v_len[4]] = 0
    v_flat[v_off[4]] = 1  # v = 1
    items = [(u_flat[u_off[i] : u_off[i] + u_len[i]].copy(), v_flat[v_off[i] : v_off[i] + v_len[i]].copy())
             for i in range(n)]
    c = mp.mpdiv_init(0, flags=flags)
    try:
        mp.mpdiv_serve_start(c, pool_digits=1 << 23, max_batch=32, max_inflight=3)
        tickets = [_submit_retry(mp, c, u, v) for u, v in items]
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


def test_admission_by_footprint_keeps_classes_apart():
    # requests of every footprint class (dividends of at most 1024, 2048, 4096,
    # 8192 digits and a 2^19-bit one) submitted at once: every launch holds
    # requests of one class, so the requests counted per launch class (the
    # class of the launch's largest dividend) equal the requests per class, a
    # 2^19-bit request never shares the launch of smaller ones, and every
    # result equals the oracle's
    import paper_2606_06386_gb300 as mp

    rnd = np.random.default_rng(77)
    u_len = np.concatenate([rnd.integers(64, 1025, 24), rnd.integers(1025, 2049, 24), rnd.integers(2049, 4097, 12),
                            rnd.integers(4097, 8193, 6), [16384]]).astype(np.int32)
    rnd.shuffle(u_len)
    v_len = np.maximum(1, (u_len * rnd.uniform(0.25, 1.0, len(u_len))).astype(np.int32)).astype(np.int32)
    u_flat, u_off, v_flat, v_off = I.ragged_operands(u_len, v_len, seed=77)
    items = [(u_flat[u_off[i]:u_off[i] + u_len[i]].copy(), v_flat[v_off[i]:v_off[i] + v_len[i]].copy())
             for i in range(len(u_len))]
    cls = [0 if n <= 1024 else 1 if n <= 2048 else 2 if n <= 4096 else 3 if n <= 8192 else 4 for n in u_len]
    c = mp.mpdiv_init(0)
    try:
        mp.mpdiv_serve_start(c, pool_digits=1 << 24, max_batch=64, max_inflight=4, max_wait_us=20000)
        tickets = [_submit_retry(mp, c, u, v) for u, v in items]
        got = []
        for t, (u, v) in zip(tickets, items):
            rc, q, r, st = mp.mpdiv_serve_poll(c, t, len(u), len(v), timeout_us=60_000_000)
            assert rc == mp.MPDIV_OK and st == 0
            got.append((q, r))
        completed, launches, batched, cl, ci = mp.mpdiv_serve_stats(c, by_class=True)
        mp.mpdiv_serve_stop(c)
    finally:
        mp.mpdiv_destroy(c)
    assert completed == len(items) and sum(cl) == launches and sum(ci) == batched == len(items)
    assert ci == [cls.count(k) for k in range(mp.MPDIV_SERVE_CLASSES)]
    assert cl[4] == 1 and all(cl[k] >= 1 for k in range(4))
    for (u, v), (q, r) in zip(items, got):
        qo, ro, _ = oracle.divmod_u32(u, v, len(u), len(v))
        assert (q == qo).all() and (r == ro).all()


@pytest.mark.parametrize("device_pools", [False, True], ids=["mapped_rings", "device_pools"])
def test_a_failed_launch_fails_its_requests_and_the_server_refuses_work(device_pools):
    # the host-side hook fails the server's second launch before any of its
    # work reaches the GPU: the first request's result is exact; the failed
    # batch's requests and those still queued finish with status 4 and poll
    # returns MPDIV_ECUDA for them; submit then returns MPDIV_ECUDA, stop
    # reports the failure, and a new server on the same context works
    import paper_2606_06386_gb300 as mp

    items = _mix(24, seed=I.SEED_BASE + 33)
    c = mp.mpdiv_init(0)
    try:
        flags = mp.MPDIV_SERVE_DEVICE_POOLS if device_pools else 0
        mp.mpdiv_serve_start(c, pool_digits=1 << 22, max_batch=4, max_inflight=2, flags=flags)
        mp.mpdiv_debug_serve_fail_launch(c, 1)
        u, v = items[0]
        t0 = _submit_retry(mp, c, u, v)
        rc, q, r, st = mp.mpdiv_serve_poll(c, t0, len(u), len(v), timeout_us=30_000_000)
        qo, ro, _ = oracle.divmod_u32(u, v, len(u), len(v))
        assert rc == mp.MPDIV_OK and st == 0 and (q == qo).all() and (r == ro).all()
        tickets = []
        for u, v in items[1:]:
            try:
                tickets.append(mp.mpdiv_serve_submit(c, u, v))
            except mp.MpdivError as e:  # the failure may come before every request is in
                assert e.code == mp.MPDIV_ECUDA
                break
        assert tickets
        for t, (u, v) in zip(tickets, items[1:]):
            with pytest.raises(mp.MpdivError) as e:
                mp.mpdiv_serve_poll(c, t, len(u), len(v), timeout_us=30_000_000)
            assert e.value.code == mp.MPDIV_ECUDA and e.value.status == mp.MPDIV_ST_INTERNAL
        with pytest.raises(mp.MpdivError) as e:
            mp.mpdiv_serve_submit(c, *items[1])
        assert e.value.code == mp.MPDIV_ECUDA
        completed, launches, batched = mp.mpdiv_serve_stats(c)
        assert completed == 1 and launches == 2
        with pytest.raises(mp.MpdivError) as e:
            mp.mpdiv_serve_stop(c)
        assert e.value.code == mp.MPDIV_ECUDA
        mp.mpdiv_serve_start(c, pool_digits=1 << 22, flags=flags)  # a new server starts clean
        u, v = items[2]
        t = _submit_retry(mp, c, u, v)
        rc, q, r, st = mp.mpdiv_serve_poll(c, t, len(u), len(v), timeout_us=30_000_000)
        qo, ro, _ = oracle.divmod_u32(u, v, len(u), len(v))
        assert rc == mp.MPDIV_OK and st == 0 and (q == qo).all() and (r == ro).all()
        mp.mpdiv_serve_stop(c)
    finally:
        mp.mpdiv_destroy(c)

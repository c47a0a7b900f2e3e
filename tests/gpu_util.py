"""Helpers for the GPU tests: device staging and batched calls through the C ABI."""

import numpy as np

import oracle
import paper_2606_06386_gb300 as mp


def dev(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).to("cuda:0")


def host_u32(t):
    return t.cpu().numpy().view(np.uint32)


_ctx = {}


def ctx(flags=0, warps=0, cols=0, kcut=0, tcut=0):
    key = (flags, warps, cols, kcut, tcut)
    if key not in _ctx:
        _ctx[key] = mp.mpdiv_init(0, warps_per_block=warps, flags=flags, mul_columns=cols, karatsuba_cutoff=kcut,
                                  transform_cutoff=tcut)
    return _ctx[key]


def run_uniform(U, V, qn=None, rn=None, flags=0, warps=0, cols=0, kcut=0, products=False, tcut=0):
    """Divide row i of U by row i of V on the GPU. Returns (Q, R, status, iters)."""
    import torch

    U = np.ascontiguousarray(U, np.uint32)
    V = np.ascontiguousarray(V, np.uint32)
    n = U.shape[0]
    qn = qn or U.shape[1]
    rn = rn or V.shape[1]
    q = torch.full((n, qn), -1, dtype=torch.int32, device="cuda:0")
    r = torch.full((n, rn), -1, dtype=torch.int32, device="cuda:0")
    st = torch.full((n,), -7, dtype=torch.int32, device="cuda:0")
    it = torch.full((n,), -1, dtype=torch.int32, device="cuda:0")
    pr = torch.zeros((n,), dtype=torch.int64, device="cuda:0") if products else None
    mp.mpdiv_batch(ctx(flags, warps, cols, kcut, tcut), dev(U), dev(V), q, r, st, it, pr)
    torch.cuda.synchronize()
    if products:
        return host_u32(q), host_u32(r), st.cpu().numpy(), it.cpu().numpy(), pr.cpu().numpy()
    return host_u32(q), host_u32(r), st.cpu().numpy(), it.cpu().numpy()


def oracle_uniform(U, V, qn=None, rn=None):
    qn = qn or U.shape[1]
    rn = rn or V.shape[1]
    Q, R, S, _ = oracle.divmod_batch_u32(U, V, qn, rn)
    return Q, R, S


def assert_same(Q, R, S, Qo, Ro, So, names=None):
    n = len(S)
    bad = [i for i in range(n) if S[i] != So[i] or not (Q[i] == Qo[i]).all() or not (R[i] == Ro[i]).all()]
    if bad:
        i = bad[0]
        qd = np.nonzero(Q[i] != Qo[i])[0]
        rd = np.nonzero(R[i] != Ro[i])[0]
        nm = names[i] if names else i
        raise AssertionError(
            f"{len(bad)}/{n} items differ; first item {nm}: status {S[i]} vs {So[i]}, "
            f"q digits differ at {qd[:8]} (of {len(qd)}), r digits differ at {rd[:8]} (of {len(rd)})"
        )

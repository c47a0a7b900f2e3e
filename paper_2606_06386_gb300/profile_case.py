"""Run a few plain division launches of one size, for profilers.

    python -m paper_2606_06386_gb300.profile_case --digits 8192 --vdigits 4096 --items 152 --launches 2 \
        [--warps W] [--cols T] [--regs 64|128] [--products clipped|full|ntt] [--tcut D] [--mul]

The operands are the seeded uniform sweep inputs; the launches go through the
C ABI (mpdiv_batch, or mpdiv_mul_batch for the multiplication cost unit of
--digits digits with --mul) on the current stream. Used to capture the
division kernel with ncu on a small case (one or two waves of blocks).
"""

import argparse
import os
import sys

import numpy as np


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--digits", type=int, default=8192)
    ap.add_argument("--vdigits", type=int, default=0, help="divisor digits (default: half)")
    ap.add_argument("--items", type=int, default=152)
    ap.add_argument("--launches", type=int, default=2)
    ap.add_argument("--warps", type=int, default=0)
    ap.add_argument("--cols", type=int, default=0, help="strip width (columns per lane): 3, 5 or 7")
    ap.add_argument("--regs", type=int, default=0, help="registers per thread of the plain kernel: 64 or 128")
    ap.add_argument("--products", default="clipped", choices=["clipped", "full", "ntt"])
    ap.add_argument("--tcut", type=int, default=0, help="transform cutoff in digits (0: the library's)")
    ap.add_argument("--mul", action="store_true", help="the multiplication cost unit instead of the division")
    a = ap.parse_args()
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch

    import paper_2606_06386_gb300 as mp
    from paper_2606_06386_gb300 import inputs as I

    mp.build()
    kl = a.vdigits or a.digits // 2
    U, V = I.sweep(a.digits, kl, a.items)
    d = lambda x: torch.from_numpy(np.ascontiguousarray(x).view(np.int32)).cuda()  # noqa: E731
    u, v = d(U), d(V)
    q = torch.zeros((a.items, a.digits - kl + 1), dtype=torch.int32, device="cuda")
    r = torch.zeros((a.items, kl), dtype=torch.int32, device="cuda")
    st = torch.zeros(a.items, dtype=torch.int32, device="cuda")
    flags = {"clipped": 0, "full": mp.MPDIV_FLAG_FULL_PRODUCTS, "ntt": mp.MPDIV_FLAG_NTT_PRODUCTS}[a.products]
    ctx = mp.mpdiv_init(0, warps_per_block=a.warps, mul_columns=a.cols, flags=flags, transform_cutoff=a.tcut,
                        registers=a.regs)
    if a.mul:
        v = d(I.uniform_batch(a.items, a.digits, seed=6, stream=a.digits))
        out = torch.zeros_like(u)
        for _ in range(a.launches):
            mp.mpdiv_mul_batch(ctx, u, v, out)
        torch.cuda.synchronize()
        mp.mpdiv_destroy(ctx)
        print(f"{a.launches} launches of {a.items} products ({a.digits} digits)")
        return
    for _ in range(a.launches):
        mp.mpdiv_batch(ctx, u, v, q, r, st)
    torch.cuda.synchronize()
    bad = int((st != 0).sum().item())
    mp.mpdiv_destroy(ctx)
    print(f"{a.launches} launches of {a.items} divisions ({a.digits}/{kl} digits), nonzero status: {bad}")
    sys.exit(1 if bad else 0)


if __name__ == "__main__":
    main()

"""Profiling driver: back-to-back batched hopping-term launches of one
lattice with n right-hand sides, for an external profiler to capture
(python -m paper_1401_2039_gb300.profile_batch --dims 24 24 24 48 --nrhs 12
--prec f32 --recon 18 --launches N).

It builds the batch, loads Gaussian right-hand sides through
wd_batch_dslash once and then launches the hopping term N times on the
batch's resident fields, alternating the output parity.  Prints the mean
launch time (CUDA events on the current stream after a synchronisation) and
the algorithmic bandwidth: per site, the n right-hand sides' spinors in and
out plus the eight links read once for all of them.
"""
from __future__ import annotations

import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    import numpy as np
    import torch

    import synthetic as syn
    from paper_1401_2039_gb300 import WilsonBatch, WilsonDirac

    ap = argparse.ArgumentParser()
    ap.add_argument("--dims", type=int, nargs=4, default=[24, 24, 24, 48])
    ap.add_argument("--nrhs", type=int, default=12)
    ap.add_argument("--prec", default="f32")
    ap.add_argument("--recon", type=int, default=18)
    ap.add_argument("--launches", type=int, default=20)
    args = ap.parse_args()
    dims = tuple(args.dims)
    ph = syn.workloads.APBC_T
    op = WilsonDirac(dims, 0.12, ph, prec=args.prec, recon=args.recon)
    op.set_gauge(torch.from_numpy(syn.su3_links(dims)).cuda())
    vh = syn.volume(dims) // 2
    ins = torch.from_numpy(np.stack([syn.gaussian_spinor(vh, 5 + r)
                                     for r in range(args.nrhs)])).cuda()
    bt = WilsonBatch([op], [args.nrhs])
    print("autotuner, plain hop:", bt.tuning(), "; norm-fused xpay hop:", bt.tuning(norm=True))
    bt.dslash([ins], 1)
    for i in range(3):
        bt.dslash_resident(i & 1)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for i in range(args.launches):
        bt.dslash_resident(i & 1)
    e1.record()
    torch.cuda.synchronize()
    us = e0.elapsed_time(e1) * 1e3 / max(1, args.launches)
    sz = {"f64": 8, "f32": 4, "f16": 2, "bf16": 2}[args.prec]
    byts = vh * (args.nrhs * 48 + 8 * args.recon) * sz
    print(f"batched hop {dims} x {args.nrhs} rhs {args.prec}/{args.recon}: {us:.1f} us per launch, "
          f"{byts / (us * 1e-6) / 1e9:.0f} GB/s algorithmic ({byts / 1e6:.0f} MB)")
    bt.close()
    op.close()


if __name__ == "__main__":
    main()

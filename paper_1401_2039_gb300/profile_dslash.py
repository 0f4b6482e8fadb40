"""Profiling driver: back-to-back resident hopping-term launches of one
workload, for an external profiler to capture (python -m
paper_1401_2039_gb300.profile_dslash --workload NAME --launches N).

It builds the workload's operator, loads one Gaussian half spinor into both
resident slots and launches the storage-precision hopping term N times,
ping-ponging between the slots and alternating the output parity, as the
Schur operator does.  Prints the mean launch time measured with CUDA events
on the operator's work stream.  With --residual it applies the Schur operator
in the residual arithmetic of the reliable updates instead (two hopping-term
launches in double-float or FP64 per application, plus layout conversion).
"""
from __future__ import annotations

import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    import torch

    import synthetic as syn
    from paper_1401_2039_gb300 import WilsonDirac

    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="wilson_32x32x32x64_f16r12", choices=sorted(syn.WORKLOADS))
    ap.add_argument("--prec", default=None, help="override the workload's storage precision")
    ap.add_argument("--recon", type=int, default=None)
    ap.add_argument("--launches", type=int, default=5)
    ap.add_argument("--dagger", action="store_true")
    ap.add_argument("--residual", choices=["df64", "f64", "early"], default=None,
                    help="apply Mhat in this residual arithmetic instead (early: FP32 "
                         "arithmetic on the double-float fields)")
    args = ap.parse_args()
    w = syn.WORKLOADS[args.workload]
    prec = args.prec or w.prec
    recon = args.recon or w.recon
    U = torch.from_numpy(syn.su3_links(w.dims, eps=w.eps, seed=w.gauge_seed)).cuda()
    half = torch.from_numpy(syn.gaussian_spinor(w.vh, w.source_seed)).cuda()
    op = WilsonDirac(w.dims, w.kappa, w.phase, prec=prec, recon=recon)
    op.set_gauge(U)
    if args.residual:
        op.set_residual_precision("df64" if args.residual == "early" else args.residual)
        out = torch.empty_like(half)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.launches):
            op.apply_eo(half, 1, args.dagger, out=out,
                        residual="early" if args.residual == "early" else True)
        e1.record()
        torch.cuda.synchronize()
        us = e0.elapsed_time(e1) * 1e3 / max(1, args.launches)
        print(f"{w.name} Mhat in {args.residual} arithmetic: {args.launches} applications, "
              f"{us:.1f} us each")
        print("launch configuration:", op.dslash_tuning(hi=True))
        op.close()
        return
    op.field_load(0, half)
    op.field_load(1, half)
    ws = torch.cuda.ExternalStream(op.work_stream)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(ws)
    for i in range(args.launches):
        op.dslash_resident(i & 1, 1 - (i & 1), args.dagger)
    e1.record(ws)
    torch.cuda.synchronize()
    us = e0.elapsed_time(e1) * 1e3 / max(1, args.launches)
    print(f"{w.name} prec={prec} recon={recon}: {args.launches} launches, {us:.1f} us each, "
          f"{op.dslash_bytes / (us * 1e-6) / 1e9:.0f} GB/s algorithmic")
    print("launch configuration:", op.dslash_tuning())
    print("xpay + norm variant:", op.dslash_tuning(norm=True))
    op.close()


if __name__ == "__main__":
    main()

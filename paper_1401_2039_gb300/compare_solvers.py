"""The solver comparison of Sec. 5 (Fig. "algosxp") on a synthetic workload:
CGNR, CRNE, MCR1 and MCR2 on the Schur system in FP64, host-driven with the
same vector kernels, each to the workload's FP64 true residual.  Reports the
iterations, the operator applications per iteration, the time per iteration
and the total time (median of --reps timed solves after one warm-up).  For
context it also times the graph-captured FP64 CGNR of wd_solve_cg on the
same system.

    python -m paper_1401_2039_gb300.compare_solvers --workload wilson_24x24x24x48_f32
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# Schur-operator applications per iteration of each method
APPLICATIONS = {"cgnr": 2, "crne": 2, "mcr1": 2, "mcr2": 1}
# flops of one Schur application per half-lattice site (two hopping terms of
# 1320 and the 48 of the final subtraction, as counted for Alg. "schur")
SCHUR_FLOPS_PER_SITE = 2 * 1320 + 48
# GB300's nominal FP64 rate (FP64 FMA pipe); the FP64 hopping term is bound
# by it, not by HBM
FP64_PEAK_TFLOPS = 1.25


def compare(workload: str = "wilson_24x24x24x48_f32", reps: int = 3,
            methods=("cgnr", "crne", "mcr1", "mcr2"), maxiter: int = 20000) -> dict:
    import torch

    import synthetic as syn
    from paper_1401_2039_gb300 import Krylov, WilsonDirac

    w = syn.WORKLOADS[workload]
    U = torch.from_numpy(syn.su3_links(w.dims, eps=w.eps, seed=w.gauge_seed)).cuda()
    b = torch.from_numpy(syn.gaussian_spinor(w.volume, w.source_seed)).cuda()
    op = WilsonDirac(w.dims, w.kappa, w.phase, prec="f64")
    op.set_gauge(U)

    def timed(fn):
        fn()
        times, res = [], None
        for _ in range(max(1, reps)):
            torch.cuda.synchronize()
            t = time.perf_counter()
            res = fn()
            torch.cuda.synchronize()
            times.append((time.perf_counter() - t) * 1e3)
        return res, statistics.median(times)

    # the dominant kernel work: one FP64 Schur application (two FP64 hopping
    # terms and the layout conversions of the canonical boundary), timed alone
    half = b[: w.vh].clone()
    out = torch.empty_like(half)
    for _ in range(3):
        op.apply_eo(half, 1, False, out=out)
    n_apply = 20
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(n_apply):
        op.apply_eo(half, 1, False, out=out)
    e1.record()
    torch.cuda.synchronize()
    apply_ms = e0.elapsed_time(e1) / n_apply
    tflops = SCHUR_FLOPS_PER_SITE * w.vh / (apply_ms * 1e-3) / 1e12
    schur = {"ms": round(apply_ms, 4), "flops_per_site": SCHUR_FLOPS_PER_SITE,
             "roofline": {"bound": "alu (FP64)", "achieved": round(tflops, 4),
                          "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                          "frac": round(tflops / FP64_PEAK_TFLOPS, 4),
                          "peak_kind": "nominal FP64"}}

    rows = []
    for m in methods:
        kr = Krylov(op, m)
        res, ms = timed(lambda: kr.solve(b, tol=w.tol, maxiter=maxiter, check=False))
        it = res.info["iters"]
        rows.append({"method": m, "status": res.status, "iterations": it,
                     "applications_per_iteration": APPLICATIONS[m],
                     "hopping_terms": res.info["dslash_hi"], "ms": round(ms, 3),
                     "ms_per_iteration": round(ms / max(1, it), 4),
                     "true_rel_resid": res.info["true_rel_resid"],
                     "true_residual_checks": res.info["reliable_updates"]})
        kr.close()
    res, ms = timed(lambda: op.solve(b, tol=w.tol, check=False))
    context = {"method": "cgnr, graph-captured fused kernels (wd_solve_cg, WD_F64)",
               "iterations": res.info["iters"], "ms": round(ms, 3),
               "ms_per_iteration": round(ms / max(1, res.info["iters"]), 4),
               "true_rel_resid": res.info["true_rel_resid"]}
    op.close()
    return {"workload": w.name, "dims": list(w.dims), "kappa": w.kappa, "tol": w.tol,
            "arithmetic": "f64", "reps": reps, "methods": rows, "context": context,
            "schur_application_f64": schur}


def main():
    import synthetic as syn
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="wilson_24x24x24x48_f32", choices=sorted(syn.WORKLOADS))
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--methods", default="cgnr,crne,mcr1,mcr2")
    args = ap.parse_args()
    out = compare(args.workload, args.reps, tuple(args.methods.split(",")))
    print(json.dumps(out))


if __name__ == "__main__":
    main()

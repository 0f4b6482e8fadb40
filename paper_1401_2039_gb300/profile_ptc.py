"""Profiling driver: repeated forward applications of the learned
preconditioner network (python -m paper_1401_2039_gb300.profile_ptc
[--dims 16 16 16 32] [--applies N]), for an external profiler to capture the
transport gathers and the tensor-core GEMMs.  Prints the mean time per
application measured with CUDA events."""
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
    from paper_1401_2039_gb300 import PtcNet
    from paper_1401_2039_gb300.train_preconditioner import neumann_weights

    ap = argparse.ArgumentParser()
    ap.add_argument("--dims", type=int, nargs=4, default=[16, 16, 16, 32])
    ap.add_argument("--applies", type=int, default=3)
    args = ap.parse_args()
    dims = tuple(args.dims)
    ch = (1, 16, 16, 16, 1)
    net = PtcNet(dims, syn.workloads.APBC_T, ch)
    net.set_gauge(torch.from_numpy(syn.su3_links(dims, eps=0.3, seed=1)).cuda())
    net.set_weights(torch.from_numpy(neumann_weights(ch, 0.124, 7)).cuda())
    r = torch.from_numpy(syn.gaussian_spinor(syn.volume(dims), 2)).cuda()
    y = torch.empty_like(r)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.applies):
        net.apply(r, out=y)
    e1.record()
    torch.cuda.synchronize()
    print(f"{'x'.join(map(str, dims))}: {args.applies} applications, "
          f"{e0.elapsed_time(e1) / args.applies:.2f} ms each")
    net.close()


if __name__ == "__main__":
    main()

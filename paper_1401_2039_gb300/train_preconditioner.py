"""Train the learned preconditioner and measure what it gains.

    python -m paper_1401_2039_gb300.train_preconditioner [--pairs 2000] [--epochs 3]
        [--out DIR] [--eval-large]

1. Training data: pairs (r, e = D^-1 r) on a 16^3 x 32 lattice (kappa 0.124,
   eps = 0.3 links, gauge seed 1).  With --data residual (default) they are
   CG residuals: for a complex Gaussian b (seeds 1000 + i), x = D^-1 b from the
   mixed-precision even-odd CGNR solve to a 1e-11 FP64 true residual and x_n
   after n = 8, 16 or 32 CGNR iterations give e = x - x_n and r = b - D x_n
   (= D e, low-mode rich, the part of D^-1 that slows a solver down); with
   --data gaussian r is the Gaussian itself and e = D^-1 r; --data mixed
   alternates the two kinds so that both ends of the spectrum are fitted.
2. Training: the 1 -> 16 -> 16 -> 16 -> 1 parallel-transport network, weights
   starting at the degree-4 Neumann polynomial of D^-1 (or the identity map)
   plus small noise, Adam on the loss sum ||N(r) - e||^2 / ||e||^2 over
   minibatches, every step on the GPU.  After every epoch the weights are
   scored by the directions flexible GCR needs with them on a held-out gauge
   field (seed 21); the best scoring weights, the initial ones included, are
   kept (a lower loss on the pairs does not by itself make a better
   preconditioner).
3. Evaluation on gauge fields the network never saw (16^3 x 32 with gauge seed
   11, and 32^3 x 64 with seed 12 when --eval-large): flexible GCR(16) with the
   network as right preconditioner against plain GCR(16) and the even-odd CGNR
   solve, all to a 1e-10 FP64 true residual: directions/iterations, wall time.

Writes weights (ptc_weights.pt), a JSON summary (learned_preconditioner.json)
and prints the summary.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


# DeGrand-Rossi gamma matrices (the basis the hopping kernels use)
_GAMMA = (
    ((0, 0, 0, 1j), (0, 0, 1j, 0), (0, -1j, 0, 0), (-1j, 0, 0, 0)),
    ((0, 0, 0, -1), (0, 0, 1, 0), (0, 1, 0, 0), (-1, 0, 0, 0)),
    ((0, 0, 1j, 0), (0, 0, 0, -1j), (-1j, 0, 0, 0), (0, 1j, 0, 0)),
    ((0, 0, 1, 0), (0, 0, 0, 1), (1, 0, 0, 0), (0, 1, 0, 0)),
)


def neumann_weights(channels, kappa, seed, scale=0.01):
    """Weights whose network is the degree-(layers) Neumann series
    sum_k (kappa H)^k of D^-1 = (1 - kappa H)^-1, by Horner's rule on two
    channels: channel 0 carries r, channel 1 the partial sum y -> r + kappa H y.
    The hop of H in direction mu is (1 - gamma_mu) forward, (1 + gamma_mu)
    backward.  Small Gaussian entries elsewhere let training use the rest."""
    import numpy as np
    rng = np.random.default_rng(seed)
    I4 = np.eye(4)
    hop = {}
    for mu in range(4):
        g = np.array(_GAMMA[mu], dtype=complex)
        hop[1 + mu] = kappa * (I4 - g)
        hop[5 + mu] = kappa * (I4 + g)
    out = []
    L = len(channels) - 1
    for li, (cin, cout) in enumerate(zip(channels[:-1], channels[1:])):
        W = scale * (rng.standard_normal((cout, cin, 9, 4, 4))
                     + 1j * rng.standard_normal((cout, cin, 9, 4, 4))) / np.sqrt(2 * cin * 9)
        if li < L - 1:                   # carry r in channel 0
            W[0, 0, 0] += I4
        acc = 1 if li < L - 1 else 0     # output channel of the partial sum
        src = 0 if li == 0 else 1        # input channel of the partial sum
        W[acc, 0, 0] += I4               # r + ...
        for k, m in hop.items():
            W[acc, src, k] += m          # ... kappa H y
        out.append(W.ravel())
    return np.concatenate(out)


def identity_weights(channels, seed, scale=0.01):
    import numpy as np
    rng = np.random.default_rng(seed)
    out = []
    for cin, cout in zip(channels[:-1], channels[1:]):
        W = scale * (rng.standard_normal((cout, cin, 9, 4, 4))
                     + 1j * rng.standard_normal((cout, cin, 9, 4, 4))) / np.sqrt(2 * cin * 9)
        W[0, 0, 0] += np.eye(4)
        out.append(W.ravel())
    return np.concatenate(out)


def main():
    import numpy as np
    import torch

    import synthetic as syn
    from paper_1401_2039_gb300 import Fgcr, PtcNet, WilsonDirac

    ap = argparse.ArgumentParser()
    ap.add_argument("--pairs", type=int, default=2000)
    ap.add_argument("--epochs", type=int, default=3)
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--lr", type=float, default=1e-4)
    ap.add_argument("--max-directions", type=int, default=600)
    ap.add_argument("--kappa", type=float, default=0.124)
    ap.add_argument("--out", default=".")
    ap.add_argument("--eval-large", action="store_true")
    ap.add_argument("--data", choices=["residual", "gaussian", "mixed"], default="mixed")
    ap.add_argument("--init", choices=["neumann", "identity"], default="neumann")
    ap.add_argument("--eval-only", action="store_true",
                    help="skip data and training; evaluate the starting weights (the degree-4 "
                         "Neumann network, which validation kept in the training runs)")
    args = ap.parse_args()
    channels = (1, 16, 16, 16, 1)
    ph = syn.workloads.APBC_T
    dims = (16, 16, 16, 32)
    V = syn.volume(dims)
    summary = {"channels": channels, "kappa": args.kappa, "train_lattice": dims,
               "pairs": args.pairs, "epochs": args.epochs, "batch": args.batch, "lr": args.lr}

    if args.eval_only:
        W = torch.from_numpy(neumann_weights(channels, args.kappa, 7)).cuda()
        summary["weights"] = "degree-4 Neumann initialisation (no training)"
        return evaluate(args, summary, channels, ph, W)

    # ---- 1. data
    U = torch.from_numpy(syn.su3_links(dims, eps=0.3, seed=1)).cuda()
    solver = WilsonDirac(dims, args.kappa, ph, prec="f32")
    solver.set_gauge(U)
    exact = WilsonDirac(dims, args.kappa, ph, prec="f64")
    exact.set_gauge(U)
    R = torch.empty((args.pairs, V, 3, 4), dtype=torch.complex64, device="cuda")
    E = torch.empty_like(R)
    t0 = time.perf_counter()
    summary["data"] = args.data
    for i in range(args.pairs):
        b = torch.from_numpy(syn.gaussian_spinor(V, 1000 + i)).cuda()
        x = solver.solve(b, tol=1e-11).x
        if args.data == "gaussian" or (args.data == "mixed" and i % 2 == 0):
            r, e = b, x
        else:
            xn = solver.solve(b, tol=1e-11, maxiter=(8, 16, 32)[i % 3], check=False).x
            e = x - xn
            r = b - exact.apply(xn)
        R[i] = r.to(torch.complex64)
        E[i] = e.to(torch.complex64)
    torch.cuda.synchronize()
    summary["data_seconds"] = time.perf_counter() - t0

    # held-out field for model selection
    Uv = torch.from_numpy(syn.su3_links(dims, eps=0.3, seed=21)).cuda()
    v_lo = WilsonDirac(dims, args.kappa, ph, prec="f32")
    v_hi = WilsonDirac(dims, args.kappa, ph, prec="f64")
    v_lo.set_gauge(Uv)
    v_hi.set_gauge(Uv)
    v_net = PtcNet(dims, ph, channels)
    v_net.set_gauge(Uv)
    v_b = torch.from_numpy(syn.gaussian_spinor(V, 555)).cuda()
    v_solver = Fgcr(v_lo, v_hi, v_net, nkrylov=16)

    def validate(weights):
        v_net.set_weights(weights)
        res = v_solver.solve(v_b, tol=1e-10, maxiter=args.max_directions, check=False)
        return res.info["iters"] if res.status == 0 else 10 ** 9

    # ---- 2. training
    net = PtcNet(dims, ph, channels)
    net.set_gauge(U)
    if args.init == "neumann":
        W0 = torch.from_numpy(neumann_weights(channels, args.kappa, 7)).cuda()
    else:
        W0 = torch.from_numpy(identity_weights(channels, 7)).cuda()
    summary["init"] = args.init
    net.set_weights(W0)
    history = []
    best_w = net.get_weights()
    best_dirs = validate(best_w)
    validation = [best_dirs]
    t0 = time.perf_counter()
    steps = 0
    g = torch.Generator(device="cpu").manual_seed(5)
    for ep in range(args.epochs):
        perm = torch.randperm(args.pairs, generator=g)
        ep_loss = 0.0
        for s in range(0, args.pairs - args.batch + 1, args.batch):
            idx = perm[s:s + args.batch].cuda()
            rb = R[idx].to(torch.complex128).contiguous()
            eb = E[idx].to(torch.complex128).contiguous()
            ep_loss += net.train_step(rb, eb, lr=args.lr)
            steps += 1
        history.append(ep_loss / args.pairs)
        w_ep = net.get_weights()
        dirs = validate(w_ep)
        validation.append(dirs)
        if dirs < best_dirs:
            best_dirs, best_w = dirs, w_ep
        print(f"epoch {ep}: mean loss {history[-1]:.4f}, validation directions {dirs}", flush=True)
    torch.cuda.synchronize()
    summary["train_seconds"] = time.perf_counter() - t0
    summary["train_steps"] = steps
    summary["loss_per_epoch"] = history
    summary["validation_directions"] = validation     # [initial, after each epoch]
    summary["kept"] = "initial" if best_dirs == validation[0] and validation.index(best_dirs) == 0 \
        else f"epoch {validation.index(best_dirs) - 1}"
    W = best_w
    summary["W0"] = W0
    v_solver.close()
    v_net.close()
    v_lo.close()
    v_hi.close()
    os.makedirs(args.out, exist_ok=True)
    torch.save({"channels": channels, "kappa": args.kappa, "weights": W.cpu()},
               os.path.join(args.out, "ptc_weights.pt"))
    net.close()
    solver.close()
    exact.close()
    del R, E
    torch.cuda.empty_cache()
    return evaluate(args, summary, channels, ph, W)


def evaluate(args, summary, channels, ph, W):
    """FGCR with the network, with the untrained Neumann network and without a
    preconditioner, and the even-odd CGNR in FP32 (reliable updates) and plain
    FP64, on unseen gauge fields, to a 1e-10 FP64 true residual."""
    import numpy as np  # noqa: F401
    import torch

    import synthetic as syn
    from paper_1401_2039_gb300 import Fgcr, PtcNet, WilsonDirac

    # ---- 3. evaluation on unseen gauge fields
    evals = []
    cases = [((16, 16, 16, 32), 11)] + ([((32, 32, 32, 64), 12)] if args.eval_large else [])
    W_start = torch.from_numpy(neumann_weights(channels, args.kappa, 7, scale=0.0)).cuda()
    W0 = summary.pop("W0", None)     # the training run's own starting weights
    for edims, seed in cases:
        Ue = torch.from_numpy(syn.su3_links(edims, eps=0.3, seed=seed)).cuda()
        lo = WilsonDirac(edims, args.kappa, ph, prec="f32")
        hi = WilsonDirac(edims, args.kappa, ph, prec="f64")
        lo.set_gauge(Ue)
        hi.set_gauge(Ue)
        enet = PtcNet(edims, ph, channels)
        enet.set_gauge(Ue)
        enet.set_weights(W)
        nnet = PtcNet(edims, ph, channels)          # untrained Neumann polynomial
        nnet.set_gauge(Ue)
        nnet.set_weights(W_start)
        b = torch.from_numpy(syn.gaussian_spinor(syn.volume(edims), 77)).cuda()
        row = {"lattice": "x".join(map(str, edims)), "gauge_seed": seed}

        def timed(fn):
            fn()
            torch.cuda.synchronize()
            t = time.perf_counter()
            out = fn()
            torch.cuda.synchronize()
            return out, (time.perf_counter() - t) * 1e3

        cases_pre = [("fgcr_learned", enet), ("fgcr_neumann4_untrained", nnet), ("gcr_plain", None)]
        snet = None
        if W0 is not None and args.init != "neumann":   # the untrained start of this run
            snet = PtcNet(edims, ph, channels)
            snet.set_gauge(Ue)
            snet.set_weights(W0)
            cases_pre.insert(1, (f"fgcr_{args.init}_untrained", snet))
        for name, pre in cases_pre:
            fg = Fgcr(lo, hi, pre, nkrylov=16)
            res, ms = timed(lambda: fg.solve(b, tol=1e-10, maxiter=args.max_directions,
                                             check=False))
            row[name] = {"directions": res.info["iters"], "restarts": res.info["reliable_updates"],
                         "ms": ms, "true_rel_resid": res.info["true_rel_resid"],
                         "status": res.status}
            fg.close()
        res, ms = timed(lambda: lo.solve(b, tol=1e-10))
        row["cgnr_even_odd_f32"] = {"iterations": res.info["iters"], "ms": ms,
                                    "true_rel_resid": res.info["true_rel_resid"]}
        res, ms = timed(lambda: hi.solve(b, tol=1e-10, maxiter=40000))
        row["cgnr_even_odd_f64"] = {"iterations": res.info["iters"], "ms": ms,
                                    "true_rel_resid": res.info["true_rel_resid"]}
        evals.append(row)
        print(json.dumps(row), flush=True)
        enet.close()
        nnet.close()
        if snet is not None:
            snet.close()
        lo.close()
        hi.close()
        torch.cuda.empty_cache()
    summary["evaluation"] = evals
    os.makedirs(args.out, exist_ok=True)
    with open(os.path.join(args.out, "learned_preconditioner.json"), "w") as f:
        json.dump(summary, f, indent=1)
    print(json.dumps(summary))


if __name__ == "__main__":
    main()

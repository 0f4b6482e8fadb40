"""Flexible GCR with the PTC network as right preconditioner: plain GCR and
preconditioned FGCR reach the FP64 true residual the oracle computes; a
network set to the first Neumann term of D^-1, N = 1 + kappa H, cuts the
number of directions, and so does a network trained on the GPU from the
identity map, on a gauge field it never saw."""
import numpy as np
import pytest
import torch

import oracle
import oracle.ptc as optc
import synthetic as syn

pytestmark = pytest.mark.gpu

APBC = syn.workloads.APBC_T


def neumann_weights(kappa):
    W = np.zeros((1, 1, optc.NK, 4, 4), dtype=complex)
    W[0, 0, 0] = np.eye(4)
    for mu in range(4):
        g = oracle.gamma(mu)
        W[0, 0, 1 + mu] = kappa * (np.eye(4) - g)
        W[0, 0, 5 + mu] = kappa * (np.eye(4) + g)
    return W


def setup(dims, kappa, seed=1):
    from paper_1401_2039_gb300 import WilsonDirac
    U = syn.su3_links(dims, eps=0.3, seed=seed)
    Ut = torch.from_numpy(U).cuda()
    lo = WilsonDirac(dims, kappa, APBC, prec="f32")
    hi = WilsonDirac(dims, kappa, APBC, prec="f64")
    lo.set_gauge(Ut)
    hi.set_gauge(Ut)
    return U, Ut, lo, hi


@pytest.mark.parametrize("dims", [(8, 8, 8, 8), (6, 6, 2, 4)])
def test_gcr_and_neumann_preconditioned_fgcr(dims):
    from paper_1401_2039_gb300 import Fgcr, PtcNet
    kappa = 0.124
    U, Ut, lo, hi = setup(dims, kappa)
    b = syn.gaussian_spinor(syn.volume(dims), 2)
    bt = torch.from_numpy(b).cuda()
    plain = Fgcr(lo, hi, None, nkrylov=16).solve(bt, tol=1e-10)
    net = PtcNet(dims, APBC, (1, 1))
    net.set_gauge(Ut)
    net.set_weights(torch.from_numpy(neumann_weights(kappa).ravel()).cuda())
    pre = Fgcr(lo, hi, net, nkrylov=16).solve(bt, tol=1e-10)
    for res in (plain, pre):
        x = res.x.cpu().numpy()
        r = np.linalg.norm(b - oracle.apply(x, U, dims, kappa, APBC)) / np.linalg.norm(b)
        assert r <= 1.05e-10, (r, res.info)
    assert pre.info["iters"] < 0.8 * plain.info["iters"], (pre.info, plain.info)


def test_trained_network_beats_its_untrained_start_and_plain_gcr():
    """What training gains.  The 1-16-16-16-1 network starts as the identity
    map (FGCR with it is plain GCR) and is trained on the GPU, by the
    library's forward, backward and Adam kernels, on 64 pairs (Gaussian r,
    e = D^-1 r) of one 8^4 gauge field.  On a gauge field it never saw,
    FGCR(16) with the trained weights needs at most half the directions of
    FGCR with the untrained weights and of plain GCR (measured on GB300:
    33 against 138 and 134), and every solve reaches the oracle's FP64 true
    residual of 1e-10."""
    from paper_1401_2039_gb300 import Fgcr, PtcNet, WilsonDirac
    from paper_1401_2039_gb300.train_preconditioner import identity_weights
    dims, kappa, channels = (8, 8, 8, 8), 0.124, optc.LAYERS
    V = syn.volume(dims)
    U = torch.from_numpy(syn.su3_links(dims, eps=0.3, seed=1)).cuda()
    lo = WilsonDirac(dims, kappa, APBC, prec="f32")
    lo.set_gauge(U)
    R = torch.stack([torch.from_numpy(syn.gaussian_spinor(V, 1000 + i)) for i in range(64)]).cuda()
    E = torch.stack([lo.solve(R[i].contiguous(), tol=1e-9).x for i in range(64)])
    net = PtcNet(dims, APBC, channels)
    net.set_gauge(U)
    w0 = torch.from_numpy(identity_weights(channels, 7)).cuda()
    net.set_weights(w0)
    g = torch.Generator().manual_seed(5)
    first = None
    for _ in range(100):
        idx = torch.randperm(64, generator=g)[:8].cuda()
        loss = net.train_step(R[idx].contiguous(), E[idx].contiguous(), lr=1e-3)
        first = loss if first is None else first
    assert loss < 0.2 * first, (first, loss)
    trained = net.get_weights()

    # evaluation on an unseen gauge field and right-hand side
    U_np = syn.su3_links(dims, eps=0.3, seed=21)
    Uv = torch.from_numpy(U_np).cuda()
    lov = WilsonDirac(dims, kappa, APBC, prec="f32")
    hiv = WilsonDirac(dims, kappa, APBC, prec="f64")
    lov.set_gauge(Uv)
    hiv.set_gauge(Uv)
    b = syn.gaussian_spinor(V, 555)
    bt = torch.from_numpy(b).cuda()
    netv = PtcNet(dims, APBC, channels)
    netv.set_gauge(Uv)
    dirs = {}
    for name, w in (("plain", None), ("untrained", w0), ("trained", trained)):
        if w is not None:
            netv.set_weights(w)
        res = Fgcr(lov, hiv, netv if w is not None else None, nkrylov=16).solve(
            bt, tol=1e-10, maxiter=2000)
        x = res.x.cpu().numpy()
        r = np.linalg.norm(b - oracle.apply(x, U_np, dims, kappa, APBC)) / np.linalg.norm(b)
        assert r <= 1.05e-10, (name, r, res.info)
        dirs[name] = res.info["iters"]
    assert dirs["trained"] <= 0.5 * dirs["untrained"], dirs
    assert dirs["trained"] <= 0.5 * dirs["plain"], dirs

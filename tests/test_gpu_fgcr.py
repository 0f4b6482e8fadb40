"""Flexible GCR with the PTC network as right preconditioner: plain GCR and
preconditioned FGCR reach the FP64 true residual the oracle computes, and a
network set to the first Neumann term of D^-1, N = 1 + kappa H, cuts the
number of directions."""
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

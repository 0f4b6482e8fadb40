"""CGNR, CRNE, MCR1 and MCR2 on the CUDA path (the solvers of the paper's
solver comparison, Sec. 5, Fig. algosxp) against the FP64 oracle, through the
C ABI.

* Iterate by iterate: after k iterations from x = 0 the solved parity of the
  GPU's x equals the oracle's k-th iterate of the same method on the same
  Schur system (both FP64; the GPU tracks CRNE through x = A^dag y, the
  oracle through y, so they differ by rounding only).
* Full solves reach the 1e-10 FP64 true residual, judged by the oracle's
  operator, and agree with the oracle's solution.
* CRNE with a twisted mass; MCR refuses one (gamma5-hermiticity).
"""
import numpy as np
import pytest
import torch

import oracle
import synthetic as syn

pytestmark = pytest.mark.gpu

METHODS = ("cgnr", "crne", "mcr1", "mcr2")


def rel(a, b):
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def make(dims, kappa, U, method, mu=0.0, phase=None):
    from paper_1401_2039_gb300 import Krylov, WilsonDirac
    op = WilsonDirac(dims, kappa, syn.workloads.APBC_T if phase is None else phase, prec="f64")
    op.set_gauge(cuda(U))
    if mu:
        op.set_twisted_mass(mu)
    return op, Krylov(op, method)


def oracle_iterate(method, bhat, U, dims, kappa, parity, k):
    if method == "cgnr":
        x, it, _, _ = oracle.cgnr(bhat, U, dims, kappa, syn.workloads.APBC_T, parity=parity,
                                  tol=1e-30, maxiter=k)
    else:
        x, it, _, _ = oracle.cr(bhat, U, dims, kappa, syn.workloads.APBC_T, method,
                                parity=parity, tol=1e-30, maxiter=k)
    assert it == k
    return x


@pytest.mark.parametrize("dims,parity", [((6, 6, 2, 4), 1), ((8, 4, 6, 10), 0)])
@pytest.mark.parametrize("method", METHODS)
def test_iterates_match_oracle(dims, parity, method):
    kappa = 0.124
    U = syn.su3_links(dims, eps=0.3, seed=1)
    b = syn.gaussian_spinor(syn.volume(dims), 7)
    bhat = oracle.schur_prepare(b, U, dims, kappa, syn.workloads.APBC_T, parity)
    op, kr = make(dims, kappa, U, method)
    for k in (1, 3, 8):
        res = kr.solve(cuda(b), tol=1e-30, maxiter=k, parity=parity, check=False)
        assert res.status == 5 and res.info["iters"] == k   # WD_ERR_NOT_CONVERGED
        got = syn.to_half(host(res.x), dims, parity)
        ref = oracle_iterate(method, bhat, U, dims, kappa, parity, k)
        # both FP64; the two sides round in different orders (and CRNE tracks
        # x instead of y), which the recurrences amplify on the indefinite
        # gamma5 A: ~1e-11 after 8 MCR iterations.  A slip in the method
        # moves the iterate by 1e-3 or more.
        assert rel(got, ref) < 1e-9, (method, k, rel(got, ref))
    kr.close()
    op.close()


@pytest.mark.parametrize("method", METHODS)
@pytest.mark.parametrize("dims,parity", [((8, 8, 8, 8), 1), ((4, 6, 8, 10), 0)])
def test_solve_reaches_true_residual(method, dims, parity):
    kappa = 0.124
    U = syn.su3_links(dims, eps=0.3, seed=3)
    b = syn.gaussian_spinor(syn.volume(dims), 4)
    op, kr = make(dims, kappa, U, method)
    res = kr.solve(cuda(b), tol=1e-10, parity=parity)
    x = host(res.x)
    r = np.linalg.norm(b - oracle.apply(x, U, dims, kappa, syn.workloads.APBC_T)) / \
        np.linalg.norm(b)
    assert r <= 1.05e-10, (method, r, res.info)
    assert abs(res.info["true_rel_resid"] - r) <= 1e-2 * r + 1e-15
    if method == "cgnr":
        x_ref, it_ref, ok = oracle.solve(b, U, dims, kappa, syn.workloads.APBC_T, parity,
                                         tol=1e-10)
    else:
        x_ref, it_ref, st = oracle.solve_cr(b, U, dims, kappa, syn.workloads.APBC_T, method,
                                            parity=parity, tol=1e-10)
        ok = st == 0
    assert ok and abs(res.info["iters"] - it_ref) <= 2, (res.info["iters"], it_ref)
    assert rel(x, x_ref) < 1e-8
    kr.close()
    op.close()


def test_crne_with_twisted_mass_and_mcr_refuses_it():
    from paper_1401_2039_gb300 import WDError
    dims, kappa, mu = (8, 8, 4, 8), 0.124, 0.1
    U = syn.su3_links(dims, eps=0.3, seed=5)
    b = syn.gaussian_spinor(syn.volume(dims), 6)
    op, kr = make(dims, kappa, U, "crne", mu=mu)
    res = kr.solve(cuda(b), tol=1e-10)
    x = host(res.x)
    r = np.linalg.norm(b - oracle.apply_tm(x, U, dims, kappa, mu, syn.workloads.APBC_T)) / \
        np.linalg.norm(b)
    assert r <= 1.05e-10
    x_ref, _, st = oracle.solve_cr(b, U, dims, kappa, syn.workloads.APBC_T, "crne", mu=mu,
                                   tol=1e-12)
    assert st == 0 and rel(x, x_ref) < 1e-8
    kr.close()
    from paper_1401_2039_gb300 import Krylov
    kr = Krylov(op, "mcr2")
    with pytest.raises(WDError) as e:
        kr.solve(cuda(b), tol=1e-10)
    assert e.value.status == 1 and "gamma5" in str(e.value)
    kr.close()
    op.close()


def test_initial_guess_limits_and_bad_operator():
    from paper_1401_2039_gb300 import Krylov, WDError, WilsonDirac
    dims, kappa = (8, 4, 4, 8), 0.124
    U = syn.su3_links(dims, eps=0.3, seed=8)
    b = syn.gaussian_spinor(syn.volume(dims), 9)
    op, kr = make(dims, kappa, U, "mcr2")
    x_ref, _, _ = oracle.solve(b, U, dims, kappa, syn.workloads.APBC_T, tol=1e-13)
    res = kr.solve(cuda(b), tol=1e-10, x0=cuda(x_ref))
    assert res.status == 0 and res.info["iters"] == 0
    res = kr.solve(cuda(b), tol=1e-10, maxiter=0, check=False)
    assert res.status == 5 and res.info["iters"] == 0
    # kappa = 0: D = 1, MCR (B = gamma5) needs exactly two iterations, CRNE one
    op0, kr0 = make(dims, 0.0, U, "mcr1")
    assert kr0.solve(cuda(b), tol=1e-12).info["iters"] == 2
    kr0.close()
    kr1 = Krylov(op0, "crne")
    res = kr1.solve(cuda(b), tol=1e-12)
    assert res.info["iters"] == 1 and rel(host(res.x), b) < 1e-14
    kr1.close()
    op0.close()
    lo = WilsonDirac(dims, kappa, syn.workloads.APBC_T, prec="f32")
    with pytest.raises(WDError):
        Krylov(lo, "crne")
    with pytest.raises(ValueError):
        Krylov(op, "bicgstab")
    lo.close()
    kr.close()
    op.close()

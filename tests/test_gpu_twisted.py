"""Twisted mass on the CUDA path (Fig. dirac: D = 1 + 2 i kappa mu gamma5 -
kappa H) against the FP64 oracle's twisted functions, through the C ABI.

The twist enters the hopping-term epilogues: the xpay epilogue multiplies
x by A = 1 + i t gamma5 and the plain one multiplies by A^-1 (t = 2 kappa mu,
-t for adjoints), so the full operator, the Schur operator A - kappa^2 H A^-1
H (storage precision and residual arithmetic) and the solve with its Schur
preparation and reconstruction are checked.  Tolerances as for the Wilson
operator, norm-wise and per site (tests/parity.py); solves by the oracle's
FP64 true residual.
"""
import numpy as np
import pytest
import torch

import oracle
import synthetic as syn
from parity import check

pytestmark = pytest.mark.gpu

PHASE = tuple(np.exp(1j * np.array([0.3, 0.0, -0.9, np.pi])))


def rel(a, b):
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def make_op(dims, kappa, phase, prec, recon, U, mu):
    from paper_1401_2039_gb300 import WilsonDirac
    op = WilsonDirac(dims, kappa, phase, prec=prec, recon=recon)
    op.set_gauge(cuda(U))
    op.set_twisted_mass(mu)
    assert op.mu == mu
    return op


@pytest.mark.parametrize("dims", [(6, 6, 2, 4), (8, 4, 6, 10)])
@pytest.mark.parametrize("prec,recon", [("f64", 18), ("f32", 18), ("f32", 12), ("f16", 12),
                                        ("bf16", 12)])
def test_twisted_operators(dims, prec, recon):
    kappa, mu = 0.124, 0.2
    U = syn.su3_links(dims, eps=0.3, seed=1)
    psi = syn.gaussian_spinor(syn.volume(dims), 101)
    op = make_op(dims, kappa, PHASE, prec, recon, U, mu)
    for dag in (False, True):
        got = host(op.apply(cuda(psi), dagger=dag))
        ref = oracle.apply_tm(psi, U, dims, kappa, mu, PHASE, dag)
        check(got, ref, prec, what=("apply", dag))
        for parity in (0, 1):
            half = syn.to_half(psi, dims, parity)
            ref = oracle.apply_eo_tm(half, U, dims, kappa, mu, PHASE, parity, dag)
            got = host(op.apply_eo(cuda(half), parity, dag))
            check(got, ref, prec, what=("apply_eo", parity, dag))
            got = host(op.apply_eo(cuda(half), parity, dag, residual=True))
            check(got, ref, "f64", what=("residual arithmetic", parity, dag))
    op.close()


def test_twisted_hop_stays_bare():
    """wd_dslash_eo is the hopping term alone, whatever mu the handle has."""
    dims = (6, 6, 2, 4)
    U = syn.su3_links(dims, eps=0.3, seed=1)
    half = syn.to_half(syn.gaussian_spinor(syn.volume(dims), 5), dims, 0)
    op = make_op(dims, 0.12, PHASE, "f64", 18, U, 0.3)
    got = host(op.dslash_eo(cuda(half), 1))
    check(got, oracle.hop_eo(half, U, dims, PHASE, 1), "f64")
    op.close()


@pytest.mark.parametrize("prec,recon", [("f64", 18), ("f32", 18), ("f16", 12)])
def test_twisted_solve(prec, recon):
    dims, kappa, mu = (8, 8, 8, 8), 0.124, 0.1
    U = syn.su3_links(dims, eps=0.3, seed=1)
    b = syn.gaussian_spinor(syn.volume(dims), 2)
    op = make_op(dims, kappa, syn.workloads.APBC_T, prec, recon, U, mu)
    res = op.solve(cuda(b), tol=1e-10)
    x = host(res.x)
    r = np.linalg.norm(b - oracle.apply_tm(x, U, dims, kappa, mu, syn.workloads.APBC_T)) / \
        np.linalg.norm(b)
    assert r <= 1.05e-10, (r, res.info)
    assert abs(res.info["true_rel_resid"] - r) <= 1e-2 * r + 1e-15
    x_ref, _, ok = oracle.solve_tm(b, U, dims, kappa, mu, syn.workloads.APBC_T, tol=1e-13)
    assert ok and rel(x, x_ref) < 1e-8
    # the Wilson solution solves a different system
    x_w, _, _ = oracle.solve(b, U, dims, kappa, syn.workloads.APBC_T, tol=1e-13)
    assert rel(x, x_w) > 1e-3
    op.close()


def test_twisted_mass_can_be_switched():
    """Changing mu rebuilds the captured iteration graphs: Wilson, twisted and
    Wilson again, on one handle."""
    dims, kappa = (8, 4, 4, 8), 0.124
    U = syn.su3_links(dims, eps=0.3, seed=2)
    b = syn.gaussian_spinor(syn.volume(dims), 3)
    op = make_op(dims, kappa, syn.workloads.APBC_T, "f32", 18, U, 0.0)
    x0 = host(op.solve(cuda(b), tol=1e-10).x)
    op.set_twisted_mass(0.25)
    x1 = host(op.solve(cuda(b), tol=1e-10).x)
    r1 = np.linalg.norm(b - oracle.apply_tm(x1, U, dims, kappa, 0.25, syn.workloads.APBC_T))
    assert r1 <= 1.05e-10 * np.linalg.norm(b)
    op.set_twisted_mass(0.0)
    x2 = host(op.solve(cuda(b), tol=1e-10).x)
    assert np.array_equal(x0, x2)
    assert rel(x1, x0) > 1e-3
    op.close()


def test_twisted_mass_argument_checks():
    from paper_1401_2039_gb300 import WDError, WilsonBatch
    dims = (4, 4, 4, 4)
    U = syn.su3_links(dims, seed=1)
    op = make_op(dims, 0.12, syn.workloads.APBC_T, "f32", 18, U, 0.1)
    with pytest.raises(WDError):
        op.set_twisted_mass(float("nan"))
    with pytest.raises(WDError):
        WilsonBatch([op], [1])
    op.close()

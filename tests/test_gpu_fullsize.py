"""Parity at the full benchmark size, 32^3 x 64 (Vh = 1,048,576), in the
launch configuration the benchmark times (autotuned, resident fields).

The oracle computes sampled output sites one by one (hop_sites): random
sites of the output parity plus sites on every wrapping boundary, each
checked on its own (tests/parity.py) as well as norm-wise.  Properties
that hold at any size cover the rest: gamma5-hermiticity of the Schur
operator over the whole field, and the FP64 true residual of the benchmark
solve recomputed by the oracle on the full lattice.
"""
import numpy as np
import pytest
import torch

import oracle
import synthetic as syn
from parity import check

pytestmark = pytest.mark.gpu

W = syn.WORKLOADS["wilson_32x32x32x64_f16r12"]


@pytest.fixture(scope="module")
def field():
    U = syn.su3_links(W.dims, eps=W.eps, seed=W.gauge_seed)
    psi = syn.gaussian_spinor(W.vh, 5)
    return U, psi


def sample_sites(parity, n=20000, seed=3):
    rng = np.random.default_rng(seed)
    X = syn.coords(W.dims)
    par = X.sum(axis=1) % 2 == parity
    cand = np.nonzero(par)[0]
    pick = rng.choice(cand, size=n, replace=False)
    edge = np.nonzero(par & ((X == 0) | (X == np.array(W.dims) - 1)).any(axis=1))[0]
    edge = rng.choice(edge, size=min(1000, len(edge)), replace=False)
    return np.unique(np.concatenate([pick, edge]))


@pytest.mark.parametrize("prec,recon", [("f16", 12), ("f16", 18), ("bf16", 12), ("f32", 18),
                                        ("f32", 12), ("f64", 18)])
def test_dslash_sampled_sites(field, prec, recon):
    from paper_1401_2039_gb300 import WilsonDirac
    U, psi = field
    op = WilsonDirac(W.dims, W.kappa, W.phase, prec=prec, recon=recon)
    op.set_gauge(torch.from_numpy(U).cuda())
    in_parity, out_parity = 0, 1
    op.field_load(0, torch.from_numpy(psi).cuda())
    op.dslash_resident(0, out_parity)
    got = op.field_store(1).cpu().numpy()
    full = np.zeros((syn.volume(W.dims), 3, 4), dtype=complex)
    full[syn.parity_sites(W.dims, in_parity)] = psi
    sites = sample_sites(out_parity)
    ref = oracle.hop_sites(full, U, W.dims, W.phase, sites)
    # norm-wise over the samples and site by site: one wrong site fails
    check(got[sites // 2], ref, prec, what=(prec, recon, op.dslash_tuning()))
    op.close()


@pytest.mark.parametrize("prec,recon,cfg", [("f16", 12, 6), ("bf16", 18, 6), ("f16", 12, 7),
                                            ("bf16", 12, 5)])
def test_dslash_sampled_sites_staged_links(monkeypatch, field, prec, recon, cfg):
    """At full size, the 16-bit hop with its eight link records staged in
    shared memory: spinors two hops ahead (candidate 6) or three (7, the
    pick of both FP16 variants at this size, and 5 with the register cap for
    5 blocks, BF16's pick)."""
    from paper_1401_2039_gb300 import WilsonDirac
    monkeypatch.setenv("WD_DSLASH_CFG", str(cfg))
    U, psi = field
    op = WilsonDirac(W.dims, W.kappa, W.phase, prec=prec, recon=recon)
    op.set_gauge(torch.from_numpy(U).cuda())
    t = op.dslash_tuning()
    assert t["index"] == cfg and t["staged"], t
    op.field_load(0, torch.from_numpy(psi).cuda())
    op.dslash_resident(0, 1)
    got = op.field_store(1).cpu().numpy()
    full = np.zeros((syn.volume(W.dims), 3, 4), dtype=complex)
    full[syn.parity_sites(W.dims, 0)] = psi
    sites = sample_sites(1, seed=4)
    ref = oracle.hop_sites(full, U, W.dims, W.phase, sites)
    check(got[sites // 2], ref, prec, what=(prec, recon, cfg))
    op.close()


def test_schur_operator_gamma5_hermiticity_full_field(field):
    from paper_1401_2039_gb300 import WilsonDirac
    U, psi = field
    op = WilsonDirac(W.dims, W.kappa, W.phase, prec="f32", recon=18)
    op.set_gauge(torch.from_numpy(U).cuda())
    phi = torch.from_numpy(syn.gaussian_spinor(W.vh, 6)).cuda()
    ps = torch.from_numpy(psi).cuda()
    a = torch.vdot(phi.flatten(), op.apply_eo(ps, 1).flatten())
    b = torch.vdot(op.apply_eo(phi, 1, dagger=True).flatten(), ps.flatten())
    assert abs((a - b).item()) < 1e-5 * abs(a.item())
    op.close()


@pytest.mark.parametrize("recovery", ["reliable", "defect"])
def test_benchmark_solve_true_residual_by_oracle(field, recovery):
    """The benchmark's solve (defect correction, inner 1e-3, is the timed
    one) reaches the target FP64 true residual as the oracle recomputes it
    on the full lattice, and reports that residual."""
    from paper_1401_2039_gb300 import WilsonDirac
    U, _ = field
    b = syn.gaussian_spinor(W.volume, W.source_seed)
    op = WilsonDirac(W.dims, W.kappa, W.phase, prec=W.prec, recon=W.recon)
    op.set_gauge(torch.from_numpy(U).cuda())
    if recovery == "defect":
        op.set_recovery("defect", 1e-3)
    res = op.solve(torch.from_numpy(b).cuda(), tol=W.tol)
    x = res.x.cpu().numpy()
    r = np.linalg.norm(b - oracle.apply(x, U, W.dims, W.kappa, W.phase)) / np.linalg.norm(b)
    assert r <= 1.05 * W.tol, (r, res.info)
    assert abs(res.info["true_rel_resid"] - r) <= 1e-3 * r
    op.close()

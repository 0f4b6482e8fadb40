"""Batched systems (many right-hand sides, uneven lattices in one persistent
launch) against the FP64 oracle and the single-system solver.

Tolerances as in test_gpu_parity.py: hopping term norm-wise 1e-13 (FP64),
1e-6 (FP32), 2e-2 (FP16) and per site (tests/parity.py); every solved system meets the FP64 true residual
1e-10 computed by the oracle and lies within 1e-8 of the oracle's solution.
"""
import numpy as np
import pytest
import torch

import oracle
import synthetic as syn
from parity import check

pytestmark = pytest.mark.gpu

APBC = syn.workloads.APBC_T
# uneven lattices, ragged last tiles, 1-3 right-hand sides each
PROBLEMS = [((4, 4, 4, 4), 3, 0.12), ((6, 6, 2, 4), 2, 0.124), ((8, 4, 6, 10), 1, 0.13)]


def rel(a, b):
    return np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel())


def make(prec, recon, problems=PROBLEMS, phase=APBC):
    from paper_1401_2039_gb300 import WilsonBatch, WilsonDirac
    ops, Us = [], []
    for k, (dims, n, kappa) in enumerate(problems):
        U = syn.su3_links(dims, eps=0.3, seed=40 + k)
        op = WilsonDirac(dims, kappa, phase, prec=prec, recon=recon)
        op.set_gauge(torch.from_numpy(U).cuda())
        ops.append(op)
        Us.append(U)
    return WilsonBatch(ops, [n for _, n, _ in problems]), ops, Us


@pytest.mark.parametrize("prec", ["f64", "f32", "f16"])
@pytest.mark.parametrize("recon", [18, 12])
def test_batch_dslash(prec, recon):
    bt, ops, Us = make(prec, recon)
    for out_parity in (0, 1):
        for dagger in (False, True):
            ins = []
            for k, (dims, n, _) in enumerate(PROBLEMS):
                ins.append(np.stack([syn.gaussian_spinor(syn.volume(dims) // 2, 100 + 7 * k + r)
                                     for r in range(n)]))
            outs = bt.dslash([torch.from_numpy(a).cuda() for a in ins], out_parity, dagger)
            torch.cuda.synchronize()
            for k, (dims, n, _) in enumerate(PROBLEMS):
                got = outs[k].cpu().numpy()
                for r in range(n):
                    ref = oracle.hop_eo(ins[k][r], Us[k], dims, APBC, out_parity, dagger)
                    check(got[r], ref, prec, what=(k, r, out_parity, dagger))


# trivial (exactly 1) and complex boundary phases mixed: the hop kernels skip
# the multiplication only in the directions whose phase is 1
TWISTED = tuple(np.exp(1j * np.array([0.0, 0.7, 0.0, -2.1])))


@pytest.mark.parametrize("prec,recon,cfg", [("f64", 18, 0), ("f32", 18, 0), ("f32", 12, 5),
                                            ("f16", 12, 0)])
def test_batch_dslash_twisted_phases(monkeypatch, prec, recon, cfg):
    monkeypatch.setenv("WD_BATCH_CFG", str(cfg))
    bt, ops, Us = make(prec, recon, PAIR_PROBLEMS, phase=TWISTED)
    ins = [np.stack([syn.gaussian_spinor(syn.volume(dims) // 2, 700 + 7 * k + r)
                     for r in range(n)]) for k, (dims, n, _) in enumerate(PAIR_PROBLEMS)]
    for out_parity in (0, 1):
        for dagger in (False, True):
            outs = bt.dslash([torch.from_numpy(a).cuda() for a in ins], out_parity, dagger)
            torch.cuda.synchronize()
            for k, (dims, n, _) in enumerate(PAIR_PROBLEMS):
                got = outs[k].cpu().numpy()
                for r in range(n):
                    ref = oracle.hop_eo(ins[k][r], Us[k], dims, TWISTED, out_parity, dagger)
                    check(got[r], ref, prec, what=(k, r, out_parity, dagger))


@pytest.mark.parametrize("prec,recon", [("f64", 18), ("f32", 18), ("f16", 12)])
def test_batch_solve(prec, recon):
    bt, ops, Us = make(prec, recon)
    bs = [np.stack([syn.gaussian_spinor(syn.volume(dims), 200 + 5 * k + r) for r in range(n)])
          for k, (dims, n, _) in enumerate(PROBLEMS)]
    xs, rc, infos = bt.solve([torch.from_numpy(b).cuda() for b in bs], tol=1e-10, maxiter=5000)
    assert rc == 0
    s = 0
    for k, (dims, n, kappa) in enumerate(PROBLEMS):
        x = xs[k].cpu().numpy()
        for r in range(n):
            b = bs[k][r]
            rt = np.linalg.norm(b - oracle.apply(x[r], Us[k], dims, kappa, APBC)) / np.linalg.norm(b)
            assert rt <= 1.05e-10, (k, r, rt, infos[s])
            assert abs(infos[s]["true_rel_resid"] - rt) <= 1e-3 * rt + 1e-15
            x_ref, _, ok = oracle.solve(b, Us[k], dims, kappa, APBC, tol=1e-13)
            assert ok and rel(x[r], x_ref) < 1e-8
            s += 1


def test_batch_matches_single_solves_and_freezes_converged():
    """Twelve point sources (every spin and colour) on one lattice, plus a
    zero right-hand side that is converged from the start."""
    from paper_1401_2039_gb300 import WilsonBatch, WilsonDirac
    dims, kappa = (4, 4, 4, 6), 0.124
    U = syn.su3_links(dims, seed=3)
    op = WilsonDirac(dims, kappa, APBC, prec="f32", recon=18)
    op.set_gauge(torch.from_numpy(U).cuda())
    srcs = [syn.point_source(dims, 5, c, s) for c in range(3) for s in range(4)]
    srcs.append(np.zeros_like(srcs[0]))
    bt = WilsonBatch([op], [len(srcs)])
    xs, rc, infos = bt.solve([torch.from_numpy(np.stack(srcs)).cuda()], tol=1e-10)
    assert rc == 0
    x = xs[0].cpu().numpy()
    assert np.count_nonzero(x[-1]) == 0 and infos[-1]["iters"] == 0
    for k in range(12):
        single = op.solve(torch.from_numpy(srcs[k]).cuda(), tol=1e-10).x.cpu().numpy()
        assert rel(x[k], single) < 1e-8
        r = np.linalg.norm(srcs[k] - oracle.apply(x[k], U, dims, kappa, APBC))
        assert r <= 1.05e-10 * np.linalg.norm(srcs[k])


def test_batch_rejects_mixed_precisions():
    from paper_1401_2039_gb300 import WDError, WilsonBatch, WilsonDirac
    U = torch.from_numpy(syn.su3_links((4, 4, 4, 4))).cuda()
    a = WilsonDirac((4, 4, 4, 4), 0.12, APBC, prec="f32")
    b = WilsonDirac((4, 4, 4, 4), 0.12, APBC, prec="f16")
    a.set_gauge(U)
    b.set_gauge(U)
    with pytest.raises(WDError):
        WilsonBatch([a, b], [1, 1])


def test_one_call_multi_solve_equals_the_batch_handle():
    """wd_solve_cg_multi (create, solve, destroy in one call) gives bitwise the
    batch handle's solutions and meets the oracle's FP64 true residual."""
    from paper_1401_2039_gb300 import WDError, solve_cg_multi
    bt, ops, Us = make("f32", 18)
    bs = [torch.from_numpy(np.stack([syn.gaussian_spinor(syn.volume(dims), 300 + 3 * k + r)
                                     for r in range(n)])).cuda()
          for k, (dims, n, _) in enumerate(PROBLEMS)]
    xs_h, rc_h, _ = bt.solve(bs, tol=1e-10)
    xs, rc, infos = solve_cg_multi(ops, [n for _, n, _ in PROBLEMS], bs, tol=1e-10)
    assert rc == rc_h == 0 and len(infos) == sum(n for _, n, _ in PROBLEMS)
    for k, (dims, n, kappa) in enumerate(PROBLEMS):
        assert torch.equal(xs[k], xs_h[k])
        x, b = xs[k].cpu().numpy(), bs[k].cpu().numpy()
        for r in range(n):
            rt = np.linalg.norm(b[r] - oracle.apply(x[r], Us[k], dims, kappa, APBC))
            assert rt <= 1.05e-10 * np.linalg.norm(b[r])
    ops[0].set_twisted_mass(0.1)   # batches have no twisted mass: an argument error
    with pytest.raises(WDError):
        solve_cg_multi(ops, [n for _, n, _ in PROBLEMS], bs, tol=1e-10)


@pytest.mark.parametrize("prec,recon", [("f32", 18), ("f16", 12)])
def test_batch_autotuner_keeps_the_fastest_configuration(prec, recon):
    """The batched hop's launch configuration (block, register cap, grid) is
    picked per batch by timing every candidate on its own lattices; the
    choice is the fastest candidate and its grid is a resident-capacity grid
    (a multiple of the SM count) no larger than needed."""
    bt, ops, Us = make(prec, recon)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    for norm in (False, True):
        t = bt.tuning(norm=norm)
        us = t["us"]
        # one item per thread: always timed; two (rhs pairs): not for odd nrhs
        assert len(us) == 9 and all(u > 0 for u in us[:5]) and all(u == 0 for u in us[5:]), t
        assert t["index"] == int(np.argmin(us[:5])) and t["rhs_per_thread"] == 1, t
        assert t["block"] in (128, 256) and t["min_blocks"] >= 1, t
        assert t["grid"] >= 1 and (t["grid"] % sms == 0 or t["grid"] < sms * t["min_blocks"]), t


# even right-hand-side counts: the pair candidates (two rhs per thread) apply
PAIR_PROBLEMS = [((4, 4, 4, 4), 4, 0.12), ((6, 6, 2, 4), 2, 0.124), ((8, 4, 6, 10), 6, 0.13)]


def test_batch_autotuner_times_the_pair_candidates():
    """With FP32 storage and even nrhs everywhere, all nine candidates are
    timed (five with one (site, rhs) item per thread, four with two) and the
    fastest is kept."""
    bt, ops, Us = make("f32", 18, PAIR_PROBLEMS)
    for norm in (False, True):
        t = bt.tuning(norm=norm)
        us = t["us"]
        assert len(us) == 9 and all(u > 0 for u in us), t
        assert t["index"] == int(np.argmin(us)), t
        assert t["rhs_per_thread"] == (2 if t["index"] >= 5 else 1), t


@pytest.mark.parametrize("recon", [18, 12])
@pytest.mark.parametrize("cfg", [5, 6, 7, 8])
def test_batch_pair_dslash(monkeypatch, recon, cfg):
    """Two right-hand sides per thread (packed FP32 pair arithmetic): every
    site against the oracle at the FP32 tolerance, and bitwise the output of
    the one-item-per-thread kernel (the same operations in the same order per
    lane), on uneven lattices with ragged last tiles, both parities and both
    daggers."""
    ins = [np.stack([syn.gaussian_spinor(syn.volume(dims) // 2, 500 + 7 * k + r)
                     for r in range(n)]) for k, (dims, n, _) in enumerate(PAIR_PROBLEMS)]
    res = {}
    for c in (0, cfg):
        monkeypatch.setenv("WD_BATCH_CFG", str(c))
        bt, ops, Us = make("f32", recon, PAIR_PROBLEMS)
        assert bt.tuning()["index"] == c and bt.tuning(norm=True)["index"] == c
        res[c] = {}
        for out_parity in (0, 1):
            for dagger in (False, True):
                outs = bt.dslash([torch.from_numpy(a).cuda() for a in ins], out_parity, dagger)
                torch.cuda.synchronize()
                res[c][out_parity, dagger] = [o.cpu() for o in outs]
        bt.close()
    for (out_parity, dagger), outs in res[cfg].items():
        for k, (dims, n, _) in enumerate(PAIR_PROBLEMS):
            assert torch.equal(outs[k], res[0][out_parity, dagger][k]), (k, out_parity, dagger)
            got = outs[k].numpy()
            for r in range(n):
                ref = oracle.hop_eo(ins[k][r], Us[k], dims, APBC, out_parity, dagger)
                check(got[r], ref, "f32", what=(k, r, out_parity, dagger))


@pytest.mark.parametrize("recovery", [("reliable", 0.1), ("defect", 1e-3)])
def test_batch_pair_solve(monkeypatch, recovery):
    """A batched solve whose hops take two right-hand sides per thread: every
    system meets the oracle's FP64 true residual and lies within 1e-8 of the
    oracle's solution."""
    monkeypatch.setenv("WD_BATCH_CFG", "6")
    bt, ops, Us = make("f32", 18, PAIR_PROBLEMS)
    assert bt.tuning()["rhs_per_thread"] == 2
    ops[0].set_recovery(*recovery)
    bs = [np.stack([syn.gaussian_spinor(syn.volume(dims), 600 + 5 * k + r) for r in range(n)])
          for k, (dims, n, _) in enumerate(PAIR_PROBLEMS)]
    xs, status, infos = bt.solve([torch.from_numpy(b).cuda() for b in bs], tol=1e-10)
    assert status == 0
    for k, (dims, n, kappa) in enumerate(PAIR_PROBLEMS):
        x = xs[k].cpu().numpy()
        for r in range(n):
            res = np.linalg.norm(bs[k][r] - oracle.apply(x[r], Us[k], dims, kappa, APBC))
            assert res <= 1.05e-10 * np.linalg.norm(bs[k][r]), (k, r, res)
            x_ref, _, ok = oracle.solve(bs[k][r], Us[k], dims, kappa, APBC, parity=1, tol=1e-13)
            assert ok and rel(x[r], x_ref) < 1e-8


@pytest.mark.parametrize("prec,recon", [("f32", 18), ("f16", 12)])
def test_batch_solve_with_defect_correction(prec, recon):
    """Batched systems with defect correction (every refresh restarts all
    inner CGNRs): each system meets the oracle's FP64 true residual and lies
    within 1e-8 of the oracle's solution."""
    bt, ops, Us = make(prec, recon)
    ops[0].set_recovery("defect", 1e-3)
    bs = []
    for k, (dims, n, _) in enumerate(PROBLEMS):
        bs.append(np.stack([syn.gaussian_spinor(syn.volume(dims), 300 + 5 * k + r) for r in range(n)]))
    xs, status, infos = bt.solve([torch.from_numpy(b).cuda() for b in bs], tol=1e-10)
    assert status == 0
    for k, (dims, n, kappa) in enumerate(PROBLEMS):
        x = xs[k].cpu().numpy()
        for r in range(n):
            res = np.linalg.norm(bs[k][r] - oracle.apply(x[r], Us[k], dims, kappa, APBC))
            assert res <= 1.05e-10 * np.linalg.norm(bs[k][r]), (k, r, res)
            x_ref, _, ok = oracle.solve(bs[k][r], Us[k], dims, kappa, APBC, parity=1, tol=1e-13)
            assert ok and rel(x[r], x_ref) < 1e-8

"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Norm-wise relative tolerances ||gpu - oracle|| / ||oracle|| by storage
precision: FP64 1e-13, FP32 1e-6, FP16/BF16 2e-2; every operator
application is also bounded site by site (tests/parity.py: FP16 4e-3 per
site, the other formats their norm-wise tolerance).  Solves are judged by
the FP64 true residual ||b - D x|| / ||b|| the oracle computes, and by the
distance to the oracle's solution.

Lattices span several 128-site thread blocks with a ragged last block
(e.g. 6x6x2x4: Vh = 144), the 2^4 lattice where x+mu and x-mu coincide,
anisotropic shapes and both boundary-phase kinds.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import synthetic as syn
from parity import check

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-13, "f32": 1e-6, "f16": 2e-2, "bf16": 2e-2}
PRECS = ["f64", "f32", "f16", "bf16"]
DIMS = [(4, 4, 4, 4), (6, 6, 2, 4), (2, 2, 2, 2), (16, 8, 8, 8), (8, 4, 6, 10)]
PHASES = {"apbc": syn.workloads.APBC_T,
          "twisted": tuple(np.exp(1j * np.array([0.3, 0.0, -0.9, np.pi])))}


def rel(a, b):
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


_fields = {}


def fields(dims, seed=1):
    key = (dims, seed)
    if key not in _fields:
        U = syn.su3_links(dims, eps=0.3, seed=seed)
        psi = syn.gaussian_spinor(syn.volume(dims), seed + 100)
        _fields[key] = (U, psi)
    return _fields[key]


def make_op(dims, kappa, phase, prec, recon, U):
    from paper_1401_2039_gb300 import WilsonDirac
    op = WilsonDirac(dims, kappa, phase, prec=prec, recon=recon)
    op.set_gauge(cuda(U))
    return op


# --------------------------------------------------------------------- hopping term
@pytest.mark.parametrize("dims", DIMS)
@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("recon", [18, 12])
def test_dslash_eo(dims, prec, recon):
    U, psi = fields(dims)
    for phname, phase in PHASES.items():
        op = make_op(dims, 0.12, phase, prec, recon, U)
        for out_parity in (0, 1):
            src = syn.to_half(psi, dims, 1 - out_parity)
            for dagger in (False, True):
                ref = oracle.hop_eo(src, U, dims, phase, out_parity, dagger)
                got = host(op.dslash_eo(cuda(src), out_parity, dagger))
                check(got, ref, prec, what=(phname, out_parity, dagger))
        op.close()


@pytest.mark.parametrize("prec", ["f16", "bf16"])
@pytest.mark.parametrize("recon", [18, 12])
@pytest.mark.parametrize("cfg", [1, 5, 6, 7])
def test_dslash_eo_each_16bit_path(monkeypatch, prec, recon, cfg):
    """Every hop path of 16-bit storage against the oracle, site by site:
    link and spinor words in registers one hop ahead (candidate 1), and the
    eight link records staged in shared memory by cp.async with the spinors
    two hops ahead (candidate 6) or three (candidates 5 and 7, register caps
    for 5 and 6 blocks).  Lattices: odd Lx/2 with a ragged last block, 2^4
    (x + mu = x - mu), and an anisotropic one; twisted boundary phases."""
    monkeypatch.setenv("WD_DSLASH_CFG", str(cfg))
    for dims in [(6, 6, 2, 4), (2, 2, 2, 2), (8, 4, 6, 10)]:
        U, psi = fields(dims)
        op = make_op(dims, 0.12, PHASES["twisted"], prec, recon, U)
        t = op.dslash_tuning()
        assert t["staged"] == (cfg >= 5) and t["stage"] == {1: 0, 5: 2, 6: 1, 7: 2}[cfg]
        for out_parity in (0, 1):
            src = syn.to_half(psi, dims, 1 - out_parity)
            for dagger in (False, True):
                ref = oracle.hop_eo(src, U, dims, PHASES["twisted"], out_parity, dagger)
                got = host(op.dslash_eo(cuda(src), out_parity, dagger))
                check(got, ref, prec, what=(dims, cfg, out_parity, dagger))
        op.close()


def test_dslash_generic_links_f64():
    """18-real links need not be unitary: random complex matrices."""
    dims = (6, 4, 2, 4)
    rng = np.random.default_rng(5)
    V = syn.volume(dims)
    U = (rng.standard_normal((V, 4, 3, 3)) + 1j * rng.standard_normal((V, 4, 3, 3)))
    psi = syn.gaussian_spinor(V, 6)
    op = make_op(dims, 0.1, PHASES["twisted"], "f64", 18, U)
    for par in (0, 1):
        for dag in (False, True):
            src = syn.to_half(psi, dims, 1 - par)
            check(host(op.dslash_eo(cuda(src), par, dag)),
                  oracle.hop_eo(src, U, dims, PHASES["twisted"], par, dag), "f64", what=(par, dag))


# --------------------------------------------------------------------- operators
@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 6, 2, 4), (8, 4, 6, 10)])
@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("recon", [18, 12])
def test_apply_full(dims, prec, recon):
    U, psi = fields(dims)
    kappa = 0.124
    phase = PHASES["apbc"]
    op = make_op(dims, kappa, phase, prec, recon, U)
    for dagger in (False, True):
        ref = oracle.apply(psi, U, dims, kappa, phase, dagger)
        got = host(op.apply(cuda(psi), dagger))
        check(got, ref, prec, what=dagger)


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 6, 2, 4), (2, 2, 2, 2)])
@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("recon", [18, 12])
def test_apply_eo(dims, prec, recon):
    U, psi = fields(dims)
    kappa = 0.13
    phase = PHASES["twisted"]
    op = make_op(dims, kappa, phase, prec, recon, U)
    for parity in (0, 1):
        src = syn.to_half(psi, dims, parity)
        for dagger in (False, True):
            ref = oracle.apply_eo(src, U, dims, kappa, phase, parity, dagger)
            got = host(op.apply_eo(cuda(src), parity, dagger))
            check(got, ref, prec, what=(parity, dagger))


def test_kappa_zero_is_identity():
    dims = (4, 4, 2, 2)
    U, psi = fields(dims)
    op = make_op(dims, 0.0, PHASES["apbc"], "f64", 18, U)
    assert np.array_equal(host(op.apply(cuda(psi))), psi)
    half = syn.to_half(psi, dims, 1)
    assert np.array_equal(host(op.apply_eo(cuda(half), 1)), half)


# --------------------------------------------------------------------- solves
@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("dims,kappa,recon", [((4, 4, 4, 4), 0.12, 18),
                                              ((8, 8, 8, 8), 0.124, 18),
                                              ((8, 8, 8, 8), 0.124, 12),
                                              ((6, 6, 2, 4), 0.124, 12)])
def test_solve_matches_oracle(prec, dims, kappa, recon):
    U, _ = fields(dims)
    phase = PHASES["apbc"]
    b = syn.gaussian_spinor(syn.volume(dims), 2)
    op = make_op(dims, kappa, phase, prec, recon, U)
    res = op.solve(cuda(b), tol=1e-10, maxiter=5000, parity=1)
    x = host(res.x)
    r_true = np.linalg.norm(b - oracle.apply(x, U, dims, kappa, phase)) / np.linalg.norm(b)
    assert r_true <= 1.05e-10, (r_true, res.info)
    assert abs(res.info["true_rel_resid"] - r_true) <= 1e-3 * r_true + 1e-15
    x_ref, _, ok = oracle.solve(b, U, dims, kappa, phase, parity=1, tol=1e-13)
    assert ok
    assert rel(x, x_ref) < 1e-8
    if prec != "f64":
        assert res.info["reliable_updates"] >= 2


@pytest.mark.parametrize("prec", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("inner_tol", [0.1, 1e-3])
@pytest.mark.parametrize("dims,recon", [((8, 8, 8, 8), 12), ((6, 6, 2, 4), 18)])
def test_defect_correction_solve_matches_oracle(prec, inner_tol, dims, recon):
    """Defect correction (outer residual in the residual arithmetic, inner
    storage-precision CGNR restarted on every new residual): the oracle's
    FP64 true residual and its solution, as for reliable updates."""
    U, _ = fields(dims)
    kappa, phase = 0.124, PHASES["apbc"]
    b = syn.gaussian_spinor(syn.volume(dims), 2)
    op = make_op(dims, kappa, phase, prec, recon, U)
    op.set_recovery("defect", inner_tol)
    assert op.recovery == ("defect", inner_tol)
    res = op.solve(cuda(b), tol=1e-10, maxiter=5000, parity=1)
    x = host(res.x)
    r_true = np.linalg.norm(b - oracle.apply(x, U, dims, kappa, phase)) / np.linalg.norm(b)
    assert r_true <= 1.05e-10, (r_true, res.info)
    assert abs(res.info["true_rel_resid"] - r_true) <= 1e-3 * r_true + 1e-15
    x_ref, _, ok = oracle.solve(b, U, dims, kappa, phase, parity=1, tol=1e-13)
    assert ok and rel(x, x_ref) < 1e-8
    # several outer steps, none of them a stagnation restart
    assert res.info["reliable_updates"] >= 2 and res.info["restarts"] == 0


def test_recovery_mode_rejects_bad_arguments():
    from paper_1401_2039_gb300.wd import WDError
    U, _ = fields((4, 4, 4, 4))
    op = make_op((4, 4, 4, 4), 0.12, PHASES["apbc"], "f16", 12, U)
    for mode, tol in (("defect", 0.0), ("defect", 1.0), ("defect", float("nan"))):
        with pytest.raises(WDError):
            op.set_recovery(mode, tol)
    assert op.recovery[0] == "reliable"


def test_solve_even_parity_and_initial_guess():
    dims, kappa = (6, 6, 2, 4), 0.124
    U, _ = fields(dims)
    phase = PHASES["twisted"]
    b = syn.gaussian_spinor(syn.volume(dims), 3)
    op = make_op(dims, kappa, phase, "f32", 18, U)
    res = op.solve(cuda(b), tol=1e-10, parity=0)
    x = host(res.x)
    assert np.linalg.norm(b - oracle.apply(x, U, dims, kappa, phase)) <= 1.05e-10 * np.linalg.norm(b)
    # starting from the solution needs no iteration
    res2 = op.solve(cuda(b), tol=1e-8, parity=0, x0=res.x)
    assert res2.info["iters"] == 0 and res2.status == 0


def test_solve_zero_rhs_and_kappa_zero():
    dims = (4, 4, 4, 4)
    U, psi = fields(dims)
    op = make_op(dims, 0.12, PHASES["apbc"], "f32", 18, U)
    res = op.solve(cuda(np.zeros_like(psi)), tol=1e-10)
    assert res.status == 0 and np.count_nonzero(host(res.x)) == 0
    op0 = make_op(dims, 0.0, PHASES["apbc"], "f64", 18, U)
    res0 = op0.solve(cuda(psi), tol=1e-12)
    # D = I: the first iteration is exact; the rest of its graph batch is a no-op
    assert res0.status == 0 and res0.info["true_rel_resid"] == 0.0
    assert res0.info["iters"] <= 8
    assert rel(host(res0.x), psi) < 1e-15


def test_solve_reports_not_converged():
    from paper_1401_2039_gb300.wd import WD_ERR_NOT_CONVERGED
    dims = (8, 8, 8, 8)
    U, _ = fields(dims)
    b = syn.gaussian_spinor(syn.volume(dims), 2)
    op = make_op(dims, 0.124, PHASES["apbc"], "f32", 18, U)
    res = op.solve(cuda(b), tol=1e-10, maxiter=5, check=False)
    assert res.status == WD_ERR_NOT_CONVERGED
    assert res.info["iters"] == 5
    assert 1e-10 < res.info["true_rel_resid"] < 1.0


@pytest.mark.parametrize("prec,recon", [("f32", 18), ("f16", 12)])
def test_host_stream_solves_match_single_host_solves(prec, recon):
    """A stream of host-memory solves (b_{k+1} uploaded during solve k, x_k
    downloaded during solve k+1, two device staging buffers for b) gives
    bitwise the solutions of one-at-a-time zero-guess host solves, each at
    the oracle's FP64 true residual; pinned and pageable buffers, both
    staging buffers reused (five sources), n = 0, and a null pointer."""
    dims, kappa = (8, 6, 6, 10), 0.124
    U, _ = fields(dims)
    op = make_op(dims, kappa, PHASES["twisted"], prec, recon, U)
    bs = [syn.gaussian_spinor(syn.volume(dims), 40 + k) for k in range(5)]
    singles = []
    for b in bs:
        bh = torch.from_numpy(b).pin_memory()
        xh = torch.zeros_like(bh).pin_memory()
        r = op.solve_host(xh, bh, tol=1e-10, guess=False)
        singles.append((xh.numpy().copy(), r.info["iters"]))
    bhs = [torch.from_numpy(b).pin_memory() for b in bs]
    bhs[3] = torch.from_numpy(bs[3].copy())   # one pageable source
    xhs = [torch.full_like(bhs[0], complex(float("nan"), 1.0)) for _ in bs]
    xhs = [x.pin_memory() if k != 1 else x for k, x in enumerate(xhs)]
    res = op.solve_host_stream(xhs, bhs, tol=1e-10)
    assert len(res) == 5
    for k, (r, (xs, it)) in enumerate(zip(res, singles)):
        assert np.array_equal(r.x.numpy(), xs), k
        assert r.info["iters"] == it and r.info["seconds"] > 0
        rt = np.linalg.norm(bs[k] - oracle.apply(r.x.numpy(), U, dims, kappa, PHASES["twisted"]))
        assert rt <= 1.05e-10 * np.linalg.norm(bs[k])
    assert op.solve_host_stream([], [], tol=1e-10) == []
    lib, n = op.lib, 2
    xp = (ctypes.c_void_p * n)(xhs[0].data_ptr(), None)
    bp = (ctypes.c_void_p * n)(bhs[0].data_ptr(), bhs[1].data_ptr())
    assert lib.wd_solve_cg_host_stream(op.handle, n, xp, bp, 1e-10, 100, 1, None) == 1
    assert lib.wd_solve_cg_host_stream(op.handle, -1, xp, bp, 1e-10, 100, 1, None) == 1
    op.close()


def test_host_memory_solve_matches_device_solve():
    dims, kappa = (8, 8, 8, 8), 0.124
    U, _ = fields(dims)
    b = syn.gaussian_spinor(syn.volume(dims), 2)
    op = make_op(dims, kappa, PHASES["apbc"], "f32", 18, U)
    dev = op.solve(cuda(b), tol=1e-10)
    bh = torch.from_numpy(b).pin_memory()
    xh = torch.zeros_like(bh).pin_memory()
    res = op.solve_host(xh, bh, tol=1e-10)
    assert np.array_equal(res.x.numpy(), host(dev.x))   # same kernels, same order: bitwise
    assert res.info["iters"] == dev.info["iters"]
    # no initial guess: x_host is not read (garbage in it changes nothing)
    xg = torch.full_like(bh, complex(float("nan"), 1.0)).pin_memory()
    res0 = op.solve_host(xg, bh, tol=1e-10, guess=False)
    assert np.array_equal(res0.x.numpy(), host(dev.x))
    # pageable host memory takes the staged-copy path, with the same result
    bp = torch.from_numpy(b.copy())
    xp = torch.full_like(bp, complex(float("nan"), 1.0))
    assert not bp.is_pinned() and not xp.is_pinned()
    resp = op.solve_host(xp, bp, tol=1e-10, guess=False)
    assert np.array_equal(resp.x.numpy(), host(dev.x))
    resq = op.solve_host(torch.zeros_like(bp), bp, tol=1e-10)
    assert np.array_equal(resq.x.numpy(), host(dev.x))
    # b arrives in eight t-slabs and the first hop runs slab by slab (one
    # slice each at Lt = 8; some empty at Lt = 6); with the twisted mass the
    # solve waits for all of b
    op.set_twisted_mass(0.05)
    dev_tm = op.solve(cuda(b), tol=1e-10)
    res_tm = op.solve_host(xh, bh, tol=1e-10, guess=False)
    assert np.array_equal(res_tm.x.numpy(), host(dev_tm.x))
    op.close()
    dims4 = (4, 4, 4, 6)
    U4, _ = fields(dims4)
    b4 = syn.gaussian_spinor(syn.volume(dims4), 2)
    op4 = make_op(dims4, kappa, PHASES["apbc"], "f16", 12, U4)
    dev4 = op4.solve(cuda(b4), tol=1e-10)
    b4h = torch.from_numpy(b4).pin_memory()
    res4 = op4.solve_host(torch.zeros_like(b4h).pin_memory(), b4h, tol=1e-10, guess=False)
    assert np.array_equal(res4.x.numpy(), host(dev4.x))
    op4.close()
    # Lt = 2: six of the eight slabs are empty, and the wrap-around slice 0
    # needs slice 1 from the last one
    dims2 = (2, 2, 2, 2)
    U2, _ = fields(dims2)
    b2 = syn.gaussian_spinor(syn.volume(dims2), 2)
    op2 = make_op(dims2, kappa, PHASES["twisted"], "f32", 18, U2)
    dev2 = op2.solve(cuda(b2), tol=1e-10)
    b2h = torch.from_numpy(b2).pin_memory()
    res2 = op2.solve_host(torch.zeros_like(b2h).pin_memory(), b2h, tol=1e-10, guess=False)
    assert np.array_equal(res2.x.numpy(), host(dev2.x))
    x2 = res2.x.numpy()
    r2 = np.linalg.norm(b2 - oracle.apply(x2, U2, dims2, kappa, PHASES["twisted"])) / np.linalg.norm(b2)
    assert r2 <= 1.05e-10, r2
    op2.close()


def test_resident_dslash_matches_canonical():
    dims = (8, 4, 6, 10)
    U, psi = fields(dims)
    for prec, recon in (("f32", 18), ("f16", 12)):
        op = make_op(dims, 0.12, PHASES["apbc"], prec, recon, U)
        src = syn.to_half(psi, dims, 0)
        op.field_load(0, cuda(src))
        op.dslash_resident(0, 1)
        got = host(op.field_store(1))
        check(got, oracle.hop_eo(src, U, dims, PHASES["apbc"], 1), prec)
        assert op.dslash_bytes == syn.volume(dims) // 2 * (48 + 8 * recon) * (4 if prec == "f32" else 2)


@pytest.mark.parametrize("prec,recon", [("f32", 18), ("f16", 12)])
def test_residual_precision_modes(prec, recon):
    """Reliable updates in native FP64 and in double-float reach the same
    FP64 true residual; switching converts the FP64-side links in place."""
    dims, kappa = (8, 8, 8, 8), 0.124
    U, _ = fields(dims)
    b = syn.gaussian_spinor(syn.volume(dims), 2)
    op = make_op(dims, kappa, PHASES["apbc"], prec, recon, U)
    xs = {}
    for mode in ("f64", "df64", "f64"):
        op.set_residual_precision(mode)
        res = op.solve(cuda(b), tol=1e-10)
        x = host(res.x)
        r = np.linalg.norm(b - oracle.apply(x, U, dims, kappa, PHASES["apbc"])) / np.linalg.norm(b)
        assert r <= 1.05e-10, (mode, r)
        xs.setdefault(mode, x)
    x_ref, _, _ = oracle.solve(b, U, dims, kappa, PHASES["apbc"], tol=1e-13)
    for mode, x in xs.items():
        assert rel(x, x_ref) < 1e-8, mode


@pytest.mark.parametrize("dims", [(6, 6, 2, 4), (8, 4, 6, 10), (2, 2, 2, 2)])
@pytest.mark.parametrize("mode", ["df64", "f64"])
def test_residual_arithmetic_schur_operator(dims, mode):
    """Mhat_p and its dagger in the arithmetic of the reliable updates agree
    with the FP64 oracle to 1e-13: native FP64, and double-float (48-bit
    significands, compensated sums rounded once per output)."""
    U, psi = fields(dims)
    kappa = 0.124
    for phase in PHASES.values():
        op = make_op(dims, kappa, phase, "f16", 12, U)
        op.set_residual_precision(mode)
        for parity in (0, 1):
            src = syn.to_half(psi, dims, parity)
            for dag in (False, True):
                ref = oracle.apply_eo(src, U, dims, kappa, phase, parity, dag)
                got = host(op.apply_eo(cuda(src), parity, dag, residual=True))
                check(got, ref, "f64", what=(mode, parity, dag))
        op.close()


@pytest.mark.parametrize("dims", [(6, 6, 2, 4), (8, 4, 6, 10), (2, 2, 2, 2)])
def test_early_refresh_schur_operator(dims):
    """Mhat_p and its dagger in the arithmetic of the early refreshes (FP32
    on the double-float fields and links) agree with the FP64 oracle to the
    FP32 tolerance, norm-wise and site by site, with the twisted mass too;
    on a handle with FP64 residuals the early form is the FP64 one."""
    U, psi = fields(dims)
    kappa = 0.124
    for phase in PHASES.values():
        op = make_op(dims, kappa, phase, "f16", 12, U)
        for mu in (0.0, 0.05):
            op.set_twisted_mass(mu)
            for parity in (0, 1):
                src = syn.to_half(psi, dims, parity)
                for dag in (False, True):
                    apply = oracle.apply_eo_tm if mu else oracle.apply_eo
                    args = (src, U, dims, kappa, mu, phase, parity, dag) if mu else \
                        (src, U, dims, kappa, phase, parity, dag)
                    ref = apply(*args)
                    got = host(op.apply_eo(cuda(src), parity, dag, residual="early"))
                    check(got, ref, "f32", what=(mu, parity, dag))
        op.set_residual_precision("f64")
        src = syn.to_half(psi, dims, 1)
        ref = oracle.apply_eo(src, U, dims, kappa, phase, 1, False)
        op.set_twisted_mass(0.0)
        got = host(op.apply_eo(cuda(src), 1, False, residual="early"))
        check(got, ref, "f64", what="f64 handle")
        op.close()


@pytest.mark.parametrize("prec,recon", [("f16", 12), ("bf16", 18), ("f32", 18)])
def test_solve_bitwise_identical_across_launch_configurations(monkeypatch, prec, recon):
    """Fused norms add in one order under every launch configuration, so
    the iterates and the solution are bitwise identical whichever
    configuration the tuner picks (ragged last chunk: Vh = 1440).  The
    link-staging candidates (5..7) apply to 16-bit storage only; elsewhere
    forcing one falls back to candidate 0."""
    dims = (8, 6, 6, 10)
    U, _ = fields(dims)
    b = syn.gaussian_spinor(syn.volume(dims), 3)
    runs = []
    for k in range(8):
        monkeypatch.setenv("WD_DSLASH_CFG", str(k))
        op = make_op(dims, 0.124, PHASES["apbc"], prec, recon, U)
        t = op.dslash_tuning()
        assert t["index"] == (k if prec in ("f16", "bf16") or k < 5 else 0)
        assert t["staged"] == (prec in ("f16", "bf16") and k >= 5)
        res = op.solve(cuda(b), tol=1e-10)
        runs.append((host(res.x), res.info["iters"], res.info["reliable_updates"]))
        op.close()
    for x, it, ru in runs[1:]:
        assert (it, ru) == runs[0][1:]
        assert np.array_equal(x, runs[0][0])


def test_f64_operator_rejects_double_float_residuals():
    from paper_1401_2039_gb300 import WDError
    dims = (4, 4, 4, 4)
    U, _ = fields(dims)
    op = make_op(dims, 0.12, PHASES["apbc"], "f64", 18, U)
    with pytest.raises(WDError):
        op.set_residual_precision("df64")

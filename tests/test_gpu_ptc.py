"""The learned preconditioner on the GPU: the tensor-core GEMM against an
FP32 matrix product of the same BF16 operands, and the network forward pass
against the FP64 oracle (BF16 operands: norm-wise 3e-2), on small lattices
in full and on the 16^3 x 32 production shape at sampled sites."""
import numpy as np
import pytest
import torch

import oracle.ptc as optc
import synthetic as syn

pytestmark = pytest.mark.gpu

APBC = syn.workloads.APBC_T
# per-site bound of the BF16 network output: 8 u with u = 2^-8 the BF16 unit
# roundoff (measured on GB300 at 16^3 x 32: at most 1.05e-2 per site,
# 5.3e-3 norm-wise)
PTC_SITE_TOL = 3e-2


@pytest.mark.parametrize("M,N,K", [(128, 16, 64), (256, 128, 128), (1024, 128, 1152), (384, 16, 64)])
def test_tensor_core_gemm(M, N, K):
    from paper_1401_2039_gb300 import PtcNet
    net = PtcNet((4, 4, 4, 4), APBC, (1, 2, 1))
    g = torch.Generator(device="cuda").manual_seed(M + N + K)
    A = torch.randn(M, K, device="cuda", generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, device="cuda", generator=g).to(torch.bfloat16)
    D = net.gemm(A, B)
    ref = A.float() @ B.float().T
    err = ((D - ref).norm() / ref.norm()).item()
    assert err < 1e-5, err


@pytest.mark.parametrize("R,M,N", [(64, 128, 16), (256, 128, 128), (6400, 384, 128),
                                   (4096, 1152, 128), (192, 256, 16)])
def test_tensor_core_gemm_transposed(R, M, N):
    """The weight-gradient GEMM D = A^T B (MN-major operand tiles, reduction
    split over CTAs and summed in a fixed order) against an FP32 product of
    the same BF16 operands; the result is the same bits on a second call."""
    from paper_1401_2039_gb300 import PtcNet
    net = PtcNet((4, 4, 4, 4), APBC, (1, 2, 1))
    g = torch.Generator(device="cuda").manual_seed(R + M + N)
    A = torch.randn(R, M, device="cuda", generator=g).to(torch.bfloat16)
    B = torch.randn(R, N, device="cuda", generator=g).to(torch.bfloat16)
    D = net.gemm_tn(A, B)
    ref = A.float().T @ B.float()
    err = ((D - ref).norm() / ref.norm()).item()
    assert err < 1e-5, err
    assert torch.equal(net.gemm_tn(A, B), D)
    net.close()


def test_gemm_bounded_wait_runs_out_and_the_gpu_stays_usable():
    """The test hook makes the GEMM issue no MMA, so its first mbarrier wait
    (limited to 2000 polls) runs out with nothing in flight: the call
    returns WD_ERR_TIMEOUT, TMEM is freed, and the next GEMM on the same
    handle, with the default limit, is correct."""
    from paper_1401_2039_gb300 import PtcNet
    from paper_1401_2039_gb300.wd import WD_ERR_TIMEOUT, WDError
    net = PtcNet((4, 4, 4, 4), APBC, (1, 2, 1))
    A = torch.randn(512, 256, device="cuda").to(torch.bfloat16)
    B = torch.randn(128, 256, device="cuda").to(torch.bfloat16)
    net.set_wait_limit(2000, withhold_mma=True)
    for fn in (lambda: net.gemm(A, B), lambda: net.gemm_tn(A, A[:, :128].contiguous())):
        with pytest.raises(WDError) as exc:
            fn()
        assert exc.value.status == WD_ERR_TIMEOUT
    net.set_wait_limit()
    D = net.gemm(A, B)
    ref = A.float() @ B.float().T
    assert ((D - ref).norm() / ref.norm()).item() < 1e-5
    with pytest.raises(WDError):
        net.set_wait_limit(0)
    net.close()


@pytest.mark.parametrize("dims", [(8, 8, 8, 8), (6, 6, 2, 4), (4, 4, 4, 4)])
@pytest.mark.parametrize("channels,norm_tol,site_tol", [((1, 16, 16, 1), 1e-4, 5e-3),
                                                        ((1, 16, 16, 16, 1), 1e-3, 1e-2)])
def test_fused_layers_match_the_gathered_layers(dims, channels, norm_tol, site_tol):
    """The fused 16 -> 16 layers (transports straight into the tensor cores'
    shared-memory tiles, TMEM accumulators per colour) against the gathered
    operand + GEMM form of the same network: the same BF16 products summed
    in another FP32 order.  The order changes the FP32 output by ~1e-7; the
    next layer rounds its operand to BF16 again, and a small fraction of
    those roundings then lands one BF16 ulp (2^-8) apart, so the bound grows
    with the layers that follow a fused one (one: 1e-4; two: 1e-3, measured
    2e-4).  Shapes with a ragged last 128-site tile (V = 288) and a partial
    one (4^4: V = 256 in two tiles)."""
    from paper_1401_2039_gb300 import PtcNet
    from parity import check
    U = syn.su3_links(dims, eps=0.3, seed=9)
    Ws = optc.identity_init(6, scale=0.5, layers=channels)
    net = PtcNet(dims, APBC, channels)
    net.set_gauge(torch.from_numpy(U).cuda())
    net.set_weights(torch.from_numpy(_to_flat(Ws)).cuda())
    r = torch.from_numpy(syn.gaussian_spinor(syn.volume(dims), 12)).cuda()
    y_fused = net.apply(r).cpu().numpy()
    net.set_fused(False)
    y_gather = net.apply(r).cpu().numpy()
    check(y_fused, y_gather, norm_tol=norm_tol, site_tol=site_tol)
    net.set_fused(True)
    assert np.array_equal(net.apply(r).cpu().numpy(), y_fused)   # deterministic
    net.close()


def test_fused_layer_bounded_wait_runs_out_and_the_gpu_stays_usable():
    from paper_1401_2039_gb300 import PtcNet
    from paper_1401_2039_gb300.wd import WD_ERR_TIMEOUT, WDError
    dims = (8, 8, 8, 8)
    U = syn.su3_links(dims, eps=0.3, seed=9)
    net = PtcNet(dims, APBC, optc.LAYERS)
    net.set_gauge(torch.from_numpy(U).cuda())
    net.set_weights(torch.from_numpy(_to_flat(optc.identity_init(6, scale=0.5))).cuda())
    r = torch.from_numpy(syn.gaussian_spinor(syn.volume(dims), 12)).cuda()
    y = net.apply(r).cpu().numpy()
    net.set_wait_limit(2000, withhold_mma=True)
    with pytest.raises(WDError) as exc:
        net.apply(r)
    assert exc.value.status == WD_ERR_TIMEOUT
    net.set_wait_limit()
    assert np.array_equal(net.apply(r).cpu().numpy(), y)
    net.close()


def _to_flat(Ws):
    return np.concatenate([W.ravel() for W in Ws])


@pytest.mark.parametrize("dims,channels", [((4, 4, 4, 4), (1, 16, 16, 16, 1)),
                                           ((6, 4, 2, 4), (1, 4, 1))])
def test_ptc_forward_matches_oracle(dims, channels):
    from paper_1401_2039_gb300 import PtcNet
    U = syn.su3_links(dims, eps=0.3, seed=2)
    Ws = optc.identity_init(3, scale=0.5, layers=channels)
    net = PtcNet(dims, APBC, channels)
    net.set_gauge(torch.from_numpy(U).cuda())
    net.set_weights(torch.from_numpy(_to_flat(Ws)).cuda())
    back = net.get_weights().cpu().numpy()
    assert np.abs(back - _to_flat(Ws)).max() < 1e-6 * np.abs(_to_flat(Ws)).max()
    r = syn.gaussian_spinor(syn.volume(dims), 5)
    y = net.apply(torch.from_numpy(r).cuda()).cpu().numpy()
    ref = optc.net_forward(r, Ws, U, dims, APBC)
    err = np.linalg.norm(y - ref) / np.linalg.norm(ref)
    assert err < 3e-2, err


def test_ptc_loss_and_gradient_match_oracle():
    from paper_1401_2039_gb300 import PtcNet
    dims, channels = (4, 4, 2, 4), (1, 4, 4, 1)
    U = syn.su3_links(dims, eps=0.3, seed=4)
    Ws = optc.identity_init(11, scale=0.5, layers=channels)
    V = syn.volume(dims)
    rs = np.stack([syn.gaussian_spinor(V, 30 + i) for i in range(2)])
    es = np.stack([syn.gaussian_spinor(V, 40 + i) for i in range(2)])
    net = PtcNet(dims, APBC, channels)
    net.set_gauge(torch.from_numpy(U).cuda())
    net.set_weights(torch.from_numpy(_to_flat(Ws)).cuda())
    loss, g = net.loss_grad(torch.from_numpy(rs).cuda(), torch.from_numpy(es).cuda())
    L_ref, g_ref = optc.loss_and_grad(list(rs), list(es), Ws, U, dims, APBC)
    assert abs(loss - L_ref) < 2e-2 * L_ref, (loss, L_ref)
    g = g.cpu().numpy()
    g_ref = _to_flat(g_ref)
    err = np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref)
    assert err < 5e-2, err
    # layer by layer too (catches a transposed block in one layer)
    off = 0
    for W in Ws:
        n = W.size
        e_l = np.linalg.norm(g[off:off + n] - g_ref[off:off + n]) / np.linalg.norm(g_ref[off:off + n])
        assert e_l < 5e-2, e_l
        off += n


def test_ptc_training_reduces_the_loss():
    """A few Adam steps fit N(r) to e = D^-1 r on a small lattice."""
    import oracle
    from paper_1401_2039_gb300 import PtcNet
    dims, channels, kappa = (4, 4, 4, 4), (1, 4, 4, 1), 0.12
    U = syn.su3_links(dims, eps=0.3, seed=5)
    V = syn.volume(dims)
    rs = np.stack([syn.gaussian_spinor(V, 50 + i) for i in range(4)])
    es = np.stack([oracle.solve(r, U, dims, kappa, APBC, tol=1e-12)[0] for r in rs])
    net = PtcNet(dims, APBC, channels)
    net.set_gauge(torch.from_numpy(U).cuda())
    net.set_weights(torch.from_numpy(_to_flat(optc.identity_init(1, 0.01, channels))).cuda())
    R, E = torch.from_numpy(rs).cuda(), torch.from_numpy(es).cuda()
    first = net.train_step(R, E, lr=3e-3)
    for _ in range(60):
        last = net.train_step(R, E, lr=3e-3)
    assert last < 0.5 * first, (first, last)


# ------------------------------------------------------------- production shape
PROD_DIMS = (16, 16, 16, 32)          # M = 3 V = 393,216 GEMM rows, 3,072 row tiles


def _prod_sites(n_random=128, seed=7):
    rng = np.random.default_rng(seed)
    V = syn.volume(PROD_DIMS)
    X = syn.coords(PROD_DIMS)
    edge = np.nonzero(((X == 0) | (X == np.array(PROD_DIMS) - 1)).any(axis=1))[0]
    pick = rng.choice(V, size=n_random, replace=False)
    last = np.array([V - 1, V - 2, V - 3 * 128])          # the last GEMM row tiles
    return np.unique(np.concatenate([pick, rng.choice(edge, 32, replace=False), last]))


def test_ptc_forward_at_production_shape_on_sampled_sites():
    """The full 1-16-16-16-1 network on 16^3 x 32 (every GEMM tile, the
    gather's full-size indexing) against the oracle evaluated on the
    receptive fields of sampled sites: norm-wise 3e-2 and per site."""
    from paper_1401_2039_gb300 import PtcNet
    from parity import check
    U = syn.su3_links(PROD_DIMS, eps=0.3, seed=2)
    Ws = optc.identity_init(3, scale=0.5)
    net = PtcNet(PROD_DIMS, APBC, optc.LAYERS)
    net.set_gauge(torch.from_numpy(U).cuda())
    net.set_weights(torch.from_numpy(_to_flat(Ws)).cuda())
    r = syn.gaussian_spinor(syn.volume(PROD_DIMS), 5)
    y = net.apply(torch.from_numpy(r).cuda()).cpu().numpy()
    sites = _prod_sites()
    ref = optc.net_forward_sites(r, Ws, U, PROD_DIMS, APBC, sites)
    check(y[sites], ref, norm_tol=3e-2, site_tol=PTC_SITE_TOL)
    net.close()


def test_ptc_gradient_at_production_shape_by_exact_central_difference():
    """The network is linear in each layer's weights, so the loss is a
    quadratic function of them and (L(W + d) - L(W - d)) / 2 equals the
    directional derivative <grad, d> exactly for a perturbation d of one
    layer.  Checks the backward pass (tensor-core and weight-gradient GEMMs,
    adjoint transports) over every tile of the 16^3 x 32 shape, layer by
    layer; both sides run on the GPU, so only BF16 rounding separates them."""
    from paper_1401_2039_gb300 import PtcNet
    U = syn.su3_links(PROD_DIMS, eps=0.3, seed=2)
    Ws = optc.identity_init(4, scale=0.5)
    V = syn.volume(PROD_DIMS)
    net = PtcNet(PROD_DIMS, APBC, optc.LAYERS)
    net.set_gauge(torch.from_numpy(U).cuda())
    w0 = _to_flat(Ws)
    net.set_weights(torch.from_numpy(w0).cuda())
    r = torch.from_numpy(syn.gaussian_spinor(V, 21)[None]).cuda()
    e = torch.from_numpy(syn.gaussian_spinor(V, 22)[None]).cuda()
    _, g = net.loss_grad(r, e)
    g = g.cpu().numpy()
    rng = np.random.default_rng(8)
    off = 0
    for W in Ws:
        n = W.size
        d = np.zeros_like(w0)
        d[off:off + n] = 0.3 * np.abs(W).mean() * (rng.standard_normal(n) + 1j * rng.standard_normal(n))
        net.set_weights(torch.from_numpy(w0 + d).cuda())
        lp, _ = net.loss_grad(r, e)
        net.set_weights(torch.from_numpy(w0 - d).cuda())
        lm, _ = net.loss_grad(r, e)
        fd = (lp - lm) / 2
        an = float(np.real(np.vdot(g, d)))
        assert abs(fd - an) < 3e-2 * abs(fd) + 1e-3 * (lp + lm) / 2, (off, fd, an, lp, lm)
        off += n
    net.close()

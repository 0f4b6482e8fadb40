"""The learned preconditioner on the GPU: the tensor-core GEMM against an
FP32 matrix product of the same BF16 operands, and the network forward pass
against the FP64 oracle (BF16 operands: norm-wise 3e-2)."""
import numpy as np
import pytest
import torch

import oracle.ptc as optc
import synthetic as syn

pytestmark = pytest.mark.gpu

APBC = syn.workloads.APBC_T


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

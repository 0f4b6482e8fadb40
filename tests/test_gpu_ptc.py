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

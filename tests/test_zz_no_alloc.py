"""wd_apply_eo_noalloc: the Schur operator for callers that cannot allocate
device memory (code inside a host framework's stream capture, plug-ins
whose host owns all device memory, real-time paths that must stay out of
the allocator).  It keeps its intermediate field in a fixed device array
inside libwd, so its results must equal those of wd_apply_eo, which works
through an operator handle and its own allocations.

Collected last on purpose: a run that stops at the first failure has run
every other test before this one.
"""
import ctypes

import numpy as np
import pytest

import synthetic as syn
from parity import check

KAPPA = 0.124
PHASE = tuple(np.exp(1j * np.array([0.2, 0.0, -0.5, np.pi])))


def _lib():
    from paper_1401_2039_gb300 import load_library
    lib = load_library()
    vp = ctypes.c_void_p
    lib.wd_apply_eo_noalloc.restype = ctypes.c_int
    lib.wd_apply_eo_noalloc.argtypes = [vp, vp, vp, ctypes.POINTER(ctypes.c_int),
                                        ctypes.c_double, ctypes.POINTER(ctypes.c_double),
                                        ctypes.c_int, ctypes.c_int, vp]
    lib.wd_noalloc_last_error.restype = ctypes.c_char_p
    return lib


def _phase8():
    flat = []
    for p in PHASE:
        flat += [p.real, p.imag]
    return (ctypes.c_double * 8)(*flat)


def test_noalloc_rejects_lattices_above_its_maximum():
    """Size check happens before any CUDA call, so it runs without a GPU."""
    lib = _lib()
    dims = (ctypes.c_int * 4)(16, 16, 16, 34)          # V/2 = 69632 > 65536
    dummy = ctypes.c_void_p(16)
    rc = lib.wd_apply_eo_noalloc(dummy, dummy, dummy, dims, KAPPA, _phase8(), 1, 0, None)
    assert rc == 2
    assert b"exceeds the no-allocation maximum of 65536" in lib.wd_noalloc_last_error()
    rc = lib.wd_apply_eo_noalloc(None, dummy, dummy, dims, KAPPA, _phase8(), 1, 0, None)
    assert rc == 1


@pytest.mark.parametrize("dims", [(65536, 65536, 65536, 65536),   # product wraps to 0
                                  (2, 2, 2**30, 2**30),           # product wraps in 64 bits
                                  (1 << 17, 2, 2, 2)])             # one extent alone too large
def test_noalloc_rejects_extents_whose_product_overflows(dims):
    """A volume that would wrap around in 64-bit arithmetic is rejected
    with WD_ERR_DIMS before any kernel is queued (no GPU needed)."""
    lib = _lib()
    dummy = ctypes.c_void_p(16)
    rc = lib.wd_apply_eo_noalloc(dummy, dummy, dummy, (ctypes.c_int * 4)(*dims), KAPPA,
                                 _phase8(), 1, 0, None)
    assert rc == 2
    assert b"exceeds the no-allocation maximum" in lib.wd_noalloc_last_error()


@pytest.mark.gpu
@pytest.mark.parametrize("dims", [(6, 6, 2, 4), (16, 16, 16, 32)])   # the latter: V/2 = maximum
def test_noalloc_matches_apply_eo_on_consecutive_calls(dims):
    import torch
    from paper_1401_2039_gb300 import WilsonDirac
    lib = _lib()
    U_np = syn.su3_links(dims, eps=0.3, seed=7)
    U = torch.from_numpy(U_np).cuda()
    op = WilsonDirac(dims, KAPPA, PHASE, prec="f64", recon=18)
    op.set_gauge(U)
    dims_c = (ctypes.c_int * 4)(*dims)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    V = syn.volume(dims)
    # two calls in a row with different inputs, parities and dagger flags:
    # the second reuses the device array the first one left filled
    for parity, dagger, seed in ((1, 0, 21), (0, 1, 22)):
        psi = torch.from_numpy(syn.gaussian_spinor(V // 2, seed)).cuda()
        ref = op.apply_eo(psi, parity, bool(dagger))
        out = torch.full_like(psi, float("nan"))
        rc = lib.wd_apply_eo_noalloc(ctypes.c_void_p(out.data_ptr()),
                                     ctypes.c_void_p(psi.data_ptr()),
                                     ctypes.c_void_p(U.data_ptr()), dims_c, KAPPA, _phase8(),
                                     parity, dagger, stream)
        assert rc == 0, lib.wd_noalloc_last_error()
        torch.cuda.synchronize()
        check(out.cpu().numpy(), ref.cpu().numpy(), "f64", what=(parity, dagger))
    op.close()


@pytest.mark.gpu
def test_noalloc_calls_captured_in_a_cuda_graph():
    """The call allocates nothing and, after one call outside the capture
    has loaded its kernels, makes no call that a stream capture forbids:
    calls with both dagger flags captured in one torch.cuda.graph and
    replayed give the results of wd_apply_eo."""
    import torch
    from paper_1401_2039_gb300 import WilsonDirac
    lib = _lib()
    dims = (6, 6, 2, 4)
    U_np = syn.su3_links(dims, eps=0.3, seed=9)
    U = torch.from_numpy(U_np).cuda()
    op = WilsonDirac(dims, KAPPA, PHASE, prec="f64", recon=18)
    op.set_gauge(U)
    dims_c = (ctypes.c_int * 4)(*dims)
    V = syn.volume(dims)
    cases = ((1, 0, 31), (0, 1, 32))
    ins = [torch.from_numpy(syn.gaussian_spinor(V // 2, seed)).cuda() for _, _, seed in cases]
    outs = [torch.empty_like(t) for t in ins]
    refs = [op.apply_eo(t, parity, bool(dagger)) for t, (parity, dagger, _) in zip(ins, cases)]

    def call(i, stream):
        parity, dagger, _ = cases[i]
        return lib.wd_apply_eo_noalloc(ctypes.c_void_p(outs[i].data_ptr()),
                                       ctypes.c_void_p(ins[i].data_ptr()),
                                       ctypes.c_void_p(U.data_ptr()), dims_c, KAPPA, _phase8(),
                                       parity, dagger, ctypes.c_void_p(stream))

    assert call(0, torch.cuda.current_stream().cuda_stream) == 0   # warm call, not captured
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    rcs = []
    with torch.cuda.graph(graph):
        s = torch.cuda.current_stream().cuda_stream
        rcs = [call(0, s), call(1, s)]
    assert rcs == [0, 0], lib.wd_noalloc_last_error()
    for o in outs:
        o.fill_(float("nan"))
    graph.replay()
    torch.cuda.synchronize()
    for i, (parity, dagger, _) in enumerate(cases):
        check(outs[i].cpu().numpy(), refs[i].cpu().numpy(), "f64", what=(parity, dagger))
    op.close()

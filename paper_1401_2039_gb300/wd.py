"""ctypes binding of libwd (include/wd.h): argument marshalling only.

Every operation runs in the CUDA kernels of libwd; PyTorch provides device
memory and streams.  There is no CPU fallback: constructing an operator
without a CUDA device, or without the compiled library, raises.

Arrays are torch complex128 tensors in the canonical layout of the C ABI:
full spinors ``[V, 3, 4]``, half-lattice spinors ``[V/2, 3, 4]`` (entry
``lex // 2`` of each site of one parity), gauge fields ``[V, 4, 3, 3]``.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import torch

from . import build as _build

WD_OK, WD_ERR_ARG, WD_ERR_DIMS, WD_ERR_CUDA, WD_ERR_NOMEM = 0, 1, 2, 3, 4
WD_ERR_NOT_CONVERGED, WD_ERR_BREAKDOWN, WD_ERR_TIMEOUT, WD_ERR_STATE = 5, 6, 7, 8
PRECISIONS = {"f64": 0, "f32": 1, "f16": 2, "bf16": 3}
RECOVERY = {"reliable": 0, "defect": 1}
# launch candidates of the batched hop (include/wd.h, wd_batch_tuning): the
# ones from BATCH_PAIR_FIRST on take two right-hand sides per thread
BATCH_CANDIDATES = 9
BATCH_PAIR_FIRST = 5


class WDError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"libwd status {status}: {message}")
        self.status = status


class SolveInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("reliable_updates", ctypes.c_int),
                ("true_rel_resid", ctypes.c_double), ("seconds", ctypes.c_double),
                ("dslash_lo", ctypes.c_double), ("dslash_hi", ctypes.c_double),
                ("bytes", ctypes.c_double), ("launches", ctypes.c_double),
                ("restarts", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def load_library() -> ctypes.CDLL:
    """Load (building first if stale) libwd.so from the package's _build directory."""
    global _lib
    if _lib is None:
        path = _build.build_library()
        lib = ctypes.CDLL(path)
        vp, dp, ip = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)
        i, d = ctypes.c_int, ctypes.c_double
        sig = {
            "wd_op_create": (i, [ctypes.POINTER(vp), ip, d, dp, i, i, vp]),
            "wd_op_destroy": (None, [vp]),
            "wd_op_set_gauge": (i, [vp, vp]),
            "wd_apply": (i, [vp, vp, vp, i]),
            "wd_apply_eo": (i, [vp, vp, vp, i, i]),
            "wd_apply_eo_residual": (i, [vp, vp, vp, i, i]),
            "wd_apply_eo_residual_early": (i, [vp, vp, vp, i, i]),
            "wd_op_set_twisted_mass": (i, [vp, ctypes.c_double]),
            "wd_op_twisted_mass": (ctypes.c_double, [vp]),
            "wd_dslash_eo": (i, [vp, vp, vp, i, i]),
            "wd_solve_cg": (i, [vp, vp, vp, d, i, i, ctypes.POINTER(SolveInfo)]),
            "wd_solve_cg_host": (i, [vp, vp, vp, d, i, i, ctypes.POINTER(SolveInfo)]),
            "wd_solve_cg_host_zero_guess": (i, [vp, vp, vp, d, i, i, ctypes.POINTER(SolveInfo)]),
            "wd_solve_cg_host_stream": (i, [vp, i, ctypes.POINTER(vp), ctypes.POINTER(vp), d, i, i,
                                            ctypes.POINTER(SolveInfo)]),
            "wd_field_load": (i, [vp, i, vp]),
            "wd_field_store": (i, [vp, i, vp]),
            "wd_dslash_resident": (i, [vp, i, i, i]),
            "wd_op_stream": (vp, [vp]),
            "wd_op_half_volume": (ctypes.c_long, [vp]),
            "wd_op_set_solver": (i, [vp, d, i]),
            "wd_op_set_recovery": (i, [vp, i, d]),
            "wd_op_recovery": (i, [vp, dp]),
            "wd_op_set_residual_precision": (i, [vp, i]),
            "wd_dslash_tuning": (i, [vp, i, dp, i, ip, ip, ip, ip]),
            "wd_dslash_bytes": (d, [vp]),
            "wd_status_string": (ctypes.c_char_p, [i]),
            "wd_last_error": (ctypes.c_char_p, []),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def _check(rc: int):
    if rc != WD_OK:
        lib = load_library()
        raise WDError(rc, lib.wd_last_error().decode() or lib.wd_status_string(rc).decode())


def _dev(t: torch.Tensor, shape, name: str) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != torch.complex128 or tuple(t.shape) != tuple(shape) or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous complex128 tensor of shape {tuple(shape)}")
    return t


def phases_array(phase) -> ctypes.Array:
    ph = [complex(p) for p in phase]
    if len(ph) != 4:
        raise ValueError("phase needs one complex number per direction")
    flat = []
    for p in ph:
        flat += [p.real, p.imag]
    return (ctypes.c_double * 8)(*flat)


@dataclass
class SolveResult:
    x: torch.Tensor
    status: int
    info: dict


class WilsonDirac:
    """Wilson-Dirac operator D = 1 - kappa H on one GPU (handle on a wd_op)."""

    def __init__(self, dims, kappa: float, phase=(1, 1, 1, -1), prec: str = "f64",
                 recon: int = 18, stream: torch.cuda.Stream | None = None):
        if not torch.cuda.is_available():
            raise RuntimeError("WilsonDirac needs a CUDA device; there is no CPU fallback")
        self.lib = load_library()
        self.dims = tuple(int(v) for v in dims)
        self.V = 1
        for v in self.dims:
            self.V *= v
        self.Vh = self.V // 2
        self.kappa = float(kappa)
        self.prec = prec
        self.recon = int(recon)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        handle = ctypes.c_void_p()
        dims_c = (ctypes.c_int * 4)(*self.dims)
        rc = self.lib.wd_op_create(ctypes.byref(handle), dims_c, self.kappa, phases_array(phase),
                                   PRECISIONS[prec], self.recon,
                                   ctypes.c_void_p(self.stream.cuda_stream))
        _check(rc)
        self.handle = handle

    # ------------------------------------------------------------------ life cycle
    def close(self):
        if getattr(self, "handle", None):
            self.lib.wd_op_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def work_stream(self) -> int:
        """cudaStream_t (as an int) that libwd queues this operator's kernels on."""
        return int(self.lib.wd_op_stream(self.handle) or 0)

    @property
    def dslash_bytes(self) -> float:
        return float(self.lib.wd_dslash_bytes(self.handle))

    # ------------------------------------------------------------------ operations
    def set_gauge(self, U: torch.Tensor):
        _dev(U, (self.V, 4, 3, 3), "U")
        _check(self.lib.wd_op_set_gauge(self.handle, ctypes.c_void_p(U.data_ptr())))

    def apply(self, psi: torch.Tensor, dagger: bool = False, out=None) -> torch.Tensor:
        _dev(psi, (self.V, 3, 4), "psi")
        out = torch.empty_like(psi) if out is None else _dev(out, (self.V, 3, 4), "out")
        _check(self.lib.wd_apply(self.handle, ctypes.c_void_p(out.data_ptr()),
                                 ctypes.c_void_p(psi.data_ptr()), int(bool(dagger))))
        return out

    def apply_eo(self, psi: torch.Tensor, parity: int = 1, dagger: bool = False,
                 out=None, residual: bool = False) -> torch.Tensor:
        """Mhat_p psi; residual=True evaluates it in the residual arithmetic
        of the reliable updates (FP64 or double-float) instead of storage
        precision, residual="early" in that of the early refreshes (FP32 on
        the double-float fields)."""
        _dev(psi, (self.Vh, 3, 4), "psi")
        out = torch.empty_like(psi) if out is None else _dev(out, (self.Vh, 3, 4), "out")
        fn = (self.lib.wd_apply_eo_residual_early if residual == "early" else
              self.lib.wd_apply_eo_residual if residual else self.lib.wd_apply_eo)
        _check(fn(self.handle, ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(psi.data_ptr()),
                  int(parity), int(bool(dagger))))
        return out

    def dslash_eo(self, psi: torch.Tensor, out_parity: int, dagger: bool = False,
                  out=None) -> torch.Tensor:
        _dev(psi, (self.Vh, 3, 4), "psi")
        out = torch.empty_like(psi) if out is None else _dev(out, (self.Vh, 3, 4), "out")
        _check(self.lib.wd_dslash_eo(self.handle, ctypes.c_void_p(out.data_ptr()),
                                     ctypes.c_void_p(psi.data_ptr()), int(out_parity),
                                     int(bool(dagger))))
        return out

    def solve(self, b: torch.Tensor, tol: float = 1e-10, maxiter: int = 20000, parity: int = 1,
              x0: torch.Tensor | None = None, check: bool = True) -> SolveResult:
        _dev(b, (self.V, 3, 4), "b")
        x = torch.zeros_like(b) if x0 is None else _dev(x0, (self.V, 3, 4), "x0").clone()
        info = SolveInfo()
        rc = self.lib.wd_solve_cg(self.handle, ctypes.c_void_p(x.data_ptr()),
                                  ctypes.c_void_p(b.data_ptr()), float(tol), int(maxiter),
                                  int(parity), ctypes.byref(info))
        if check and rc not in (WD_OK,):
            _check(rc)
        return SolveResult(x, rc, info.as_dict())

    def solve_host(self, x_host: torch.Tensor, b_host: torch.Tensor, tol: float = 1e-10,
                   maxiter: int = 20000, parity: int = 1, guess: bool = True) -> SolveResult:
        """Solve with x and b in host memory (pinned for asynchronous copies).
        guess=False starts from x = 0 and never reads x_host (output only)."""
        for t, n in ((x_host, "x"), (b_host, "b")):
            if t.is_cuda or t.dtype != torch.complex128 or tuple(t.shape) != (self.V, 3, 4) \
                    or not t.is_contiguous():
                raise ValueError(f"{n} must be a contiguous complex128 host tensor [V, 3, 4]")
        info = SolveInfo()
        fn = self.lib.wd_solve_cg_host if guess else self.lib.wd_solve_cg_host_zero_guess
        rc = fn(self.handle, ctypes.c_void_p(x_host.data_ptr()), ctypes.c_void_p(b_host.data_ptr()),
                float(tol), int(maxiter), int(parity), ctypes.byref(info))
        _check(rc)
        return SolveResult(x_host, rc, info.as_dict())

    def solve_host_stream(self, xs_host, bs_host, tol: float = 1e-10, maxiter: int = 20000,
                          parity: int = 1) -> list:
        """A stream of host-memory solves from x = 0 (wd_solve_cg_host_stream):
        b_{k+1} goes up while solve k runs and x_k comes down while solve k+1
        runs.  xs_host[k], bs_host[k]: contiguous complex128 host tensors
        [V, 3, 4] (pinned for asynchronous copies).  Returns one SolveResult
        per source."""
        n = len(bs_host)
        if len(xs_host) != n:
            raise ValueError("as many solution tensors as sources")
        for t in list(xs_host) + list(bs_host):
            if t.is_cuda or t.dtype != torch.complex128 or tuple(t.shape) != (self.V, 3, 4) \
                    or not t.is_contiguous():
                raise ValueError("spinors must be contiguous complex128 host tensors [V, 3, 4]")
        xp = (ctypes.c_void_p * max(n, 1))(*[t.data_ptr() for t in xs_host])
        bp = (ctypes.c_void_p * max(n, 1))(*[t.data_ptr() for t in bs_host])
        infos = (SolveInfo * max(n, 1))()
        rc = self.lib.wd_solve_cg_host_stream(self.handle, n, xp, bp, float(tol), int(maxiter),
                                              int(parity), infos)
        _check(rc)
        return [SolveResult(xs_host[k], rc, infos[k].as_dict()) for k in range(n)]

    def set_solver(self, ru_delta: float = 0.1, stall_iters: int = 200):
        """Reliable-update threshold and stagnation restart of the mixed-precision solve."""
        _check(self.lib.wd_op_set_solver(self.handle, float(ru_delta), int(stall_iters)))

    def set_recovery(self, mode: str = "reliable", inner_tol: float = 0.1):
        """Accuracy recovery of the mixed-precision solve: "reliable" (reliable
        updates, the default) or "defect" (defect correction with inner CGNR
        solves that each reduce the residual by inner_tol)."""
        _check(self.lib.wd_op_set_recovery(self.handle, RECOVERY[mode], float(inner_tol)))

    @property
    def recovery(self) -> tuple:
        tol = ctypes.c_double()
        k = self.lib.wd_op_recovery(self.handle, ctypes.byref(tol))
        return ({v: n for n, v in RECOVERY.items()}[k], tol.value)

    def set_twisted_mass(self, mu: float):
        """D = 1 + 2 i kappa mu gamma5 - kappa H (Fig. dirac); mu = 0 is the
        Wilson operator.  Applies to apply, apply_eo and solve."""
        _check(self.lib.wd_op_set_twisted_mass(self.handle, float(mu)))

    @property
    def mu(self) -> float:
        return float(self.lib.wd_op_twisted_mass(self.handle))

    def set_residual_precision(self, mode: str = "df64"):
        """Residual arithmetic of the reliable updates: "f64" or "df64" (double-float)."""
        _check(self.lib.wd_op_set_residual_precision(self.handle, {"f64": 0, "df64": 1}[mode]))

    def dslash_tuning(self, hi: bool = False, norm: bool = False) -> dict:
        """The autotuner's choice for the hopping term and its per-candidate
        timings (us): storage precision (default), residual arithmetic
        (hi=True), or the storage-precision variant with xpay and fused norm
        (norm=True)."""
        us = (ctypes.c_double * 8)()
        blk, mb, spt, stg = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        variant = 2 if norm else int(bool(hi))
        k = self.lib.wd_dslash_tuning(self.handle, variant, us, 8, ctypes.byref(blk),
                                      ctypes.byref(mb), ctypes.byref(spt), ctypes.byref(stg))
        return {"index": k, "block": blk.value, "min_blocks": mb.value,
                "sites_per_thread": spt.value, "staged": bool(stg.value), "stage": stg.value,
                "us": [round(v, 2) for v in us]}

    # resident fields, for timing the hopping term alone
    def field_load(self, slot: int, half: torch.Tensor):
        _dev(half, (self.Vh, 3, 4), "half")
        _check(self.lib.wd_field_load(self.handle, int(slot), ctypes.c_void_p(half.data_ptr())))

    def field_store(self, slot: int, out: torch.Tensor | None = None) -> torch.Tensor:
        if out is None:
            out = torch.empty((self.Vh, 3, 4), dtype=torch.complex128, device="cuda")
        _dev(out, (self.Vh, 3, 4), "out")
        _check(self.lib.wd_field_store(self.handle, int(slot), ctypes.c_void_p(out.data_ptr())))
        return out

    def dslash_resident(self, in_slot: int, out_parity: int, dagger: bool = False):
        _check(self.lib.wd_dslash_resident(self.handle, int(in_slot), int(out_parity),
                                           int(bool(dagger))))


def solve_cg_multi(ops, nrhs, bs, tol: float = 1e-10, maxiter: int = 20000, parity: int = 1,
                   x0s=None, check: bool = True):
    """One-call batched solve (wd_solve_cg_multi): bs[k] is [nrhs_k, V_k, 3, 4]
    for operator ops[k].  Returns (xs, status, infos) like WilsonBatch.solve."""
    lib = load_library()
    _setup_batch_signatures(lib)
    if len(ops) != len(nrhs) or len(bs) != len(ops):
        raise ValueError("one nrhs and one right-hand-side tensor per operator")
    nrhs = [int(n) for n in nrhs]
    shapes = [(n, op.V, 3, 4) for n, op in zip(nrhs, ops)]
    for t, shp in zip(bs, shapes):
        _dev(t, shp, "b")
    xs = [torch.zeros(sh, dtype=torch.complex128, device="cuda") for sh in shapes] \
        if x0s is None else [x.clone() for x in x0s]
    for t, shp in zip(xs, shapes):
        _dev(t, shp, "x0")
    vpa = ctypes.c_void_p * len(ops)
    infos = (SolveInfo * sum(nrhs))()
    rc = lib.wd_solve_cg_multi(vpa(*[op.handle for op in ops]), len(ops),
                               vpa(*[x.data_ptr() for x in xs]), vpa(*[b.data_ptr() for b in bs]),
                               (ctypes.c_int * len(ops))(*nrhs), float(tol), int(maxiter),
                               int(parity), infos)
    if check and rc != WD_OK:
        raise WDError(rc, lib.wd_batch_last_error().decode())
    return xs, rc, [i.as_dict() for i in infos]


class WilsonBatch:
    """Lockstep batch of systems: several operators (lattices of any size, same
    storage precision) with nrhs right-hand sides each (handle on a wd_batch)."""

    def __init__(self, ops, nrhs):
        self.lib = load_library()
        _setup_batch_signatures(self.lib)
        if len(ops) != len(nrhs):
            raise ValueError("one nrhs per operator")
        self.ops = list(ops)
        self.nrhs = [int(n) for n in nrhs]
        arr = (ctypes.c_void_p * len(ops))(*[op.handle for op in ops])
        nr = (ctypes.c_int * len(ops))(*self.nrhs)
        handle = ctypes.c_void_p()
        rc = self.lib.wd_batch_create(ctypes.byref(handle), arr, nr, len(ops))
        if rc != WD_OK:
            raise WDError(rc, self.lib.wd_batch_last_error().decode())
        self.handle = handle

    def close(self):
        if getattr(self, "handle", None):
            self.lib.wd_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def nsystems(self) -> int:
        return sum(self.nrhs)

    def _ptrs(self, tensors, shapes, name):
        if len(tensors) != len(self.ops):
            raise ValueError(f"{name}: one tensor per operator")
        for t, shp in zip(tensors, shapes):
            _dev(t, shp, name)
        return (ctypes.c_void_p * len(tensors))(*[t.data_ptr() for t in tensors])

    def dslash(self, ins, out_parity: int, dagger: bool = False):
        """Hopping term of every system: ins[k] is [nrhs_k, V_k/2, 3, 4] on parity 1 - out_parity."""
        shapes = [(n, op.Vh, 3, 4) for n, op in zip(self.nrhs, self.ops)]
        outs = [torch.empty(s, dtype=torch.complex128, device="cuda") for s in shapes]
        rc = self.lib.wd_batch_dslash(self.handle, self._ptrs(outs, shapes, "out"),
                                      self._ptrs(ins, shapes, "in"), int(out_parity),
                                      int(bool(dagger)))
        if rc != WD_OK:
            raise WDError(rc, self.lib.wd_batch_last_error().decode())
        return outs

    def tuning(self, norm: bool = False) -> dict:
        """The autotuner's choice for the batched hop (norm=True: the xpay hop
        with fused norms) and every candidate's microseconds per launch."""
        us = (ctypes.c_double * BATCH_CANDIDATES)()
        blk, mb, gr = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        k = self.lib.wd_batch_tuning(self.handle, int(bool(norm)), us, BATCH_CANDIDATES,
                                     ctypes.byref(blk), ctypes.byref(mb), ctypes.byref(gr))
        return {"index": k, "block": blk.value, "min_blocks": mb.value, "grid": gr.value,
                "rhs_per_thread": 2 if k >= BATCH_PAIR_FIRST else 1,
                "us": [us[i] for i in range(BATCH_CANDIDATES)]}

    def dslash_resident(self, out_parity: int, dagger: bool = False):
        rc = self.lib.wd_batch_dslash_resident(self.handle, int(out_parity), int(bool(dagger)))
        if rc != WD_OK:
            raise WDError(rc, self.lib.wd_batch_last_error().decode())

    def solve(self, bs, tol: float = 1e-10, maxiter: int = 20000, parity: int = 1, x0s=None,
              check: bool = True):
        """Solve every system; bs[k] is [nrhs_k, V_k, 3, 4].  Returns (xs, status, infos)."""
        shapes = [(n, op.V, 3, 4) for n, op in zip(self.nrhs, self.ops)]
        xs = [torch.zeros(s, dtype=torch.complex128, device="cuda") for s in shapes] \
            if x0s is None else [x.clone() for x in x0s]
        infos = (SolveInfo * self.nsystems)()
        rc = self.lib.wd_batch_solve(self.handle, self._ptrs(xs, shapes, "x"),
                                     self._ptrs(bs, shapes, "b"), float(tol), int(maxiter),
                                     int(parity), infos)
        if check and rc != WD_OK:
            raise WDError(rc, self.lib.wd_batch_last_error().decode())
        return xs, rc, [i.as_dict() for i in infos]


_batch_sigs_done = False


def _setup_batch_signatures(lib):
    global _batch_sigs_done
    if _batch_sigs_done:
        return
    vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    pp = ctypes.POINTER(ctypes.c_void_p)
    sig = {
        "wd_batch_create": (i, [ctypes.POINTER(vp), pp, ctypes.POINTER(i), i]),
        "wd_batch_destroy": (None, [vp]),
        "wd_batch_dslash": (i, [vp, pp, pp, i, i]),
        "wd_batch_dslash_resident": (i, [vp, i, i]),
        "wd_batch_tuning": (i, [vp, i, ctypes.POINTER(d), i, ctypes.POINTER(i),
                                ctypes.POINTER(i), ctypes.POINTER(i)]),
        "wd_batch_solve": (i, [vp, pp, pp, d, i, i, ctypes.POINTER(SolveInfo)]),
        "wd_batch_last_error": (ctypes.c_char_p, []),
        "wd_solve_cg_multi": (i, [pp, i, pp, pp, ctypes.POINTER(i), d, i, i,
                                  ctypes.POINTER(SolveInfo)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _batch_sigs_done = True


class PtcNet:
    """Parallel-transport convolution network (handle on a wd_ptc): the learned
    right preconditioner.  Weights are one flat complex128 vector, layers in
    order, each [C_out, C_in, 9, 4, 4]."""

    def __init__(self, dims, phase=(1, 1, 1, -1), channels=(1, 16, 16, 16, 1),
                 stream: torch.cuda.Stream | None = None):
        if not torch.cuda.is_available():
            raise RuntimeError("PtcNet needs a CUDA device; there is no CPU fallback")
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.lib = load_library()
        _setup_ptc_signatures(self.lib)
        self.dims = tuple(int(d) for d in dims)
        self.V = 1
        for d in self.dims:
            self.V *= d
        self.channels = tuple(int(c) for c in channels)
        handle = ctypes.c_void_p()
        ch = (ctypes.c_int * len(self.channels))(*self.channels)
        rc = self.lib.wd_ptc_create(ctypes.byref(handle), (ctypes.c_int * 4)(*self.dims),
                                    phases_array(phase), len(self.channels) - 1, ch,
                                    ctypes.c_void_p(self.stream.cuda_stream))
        if rc != WD_OK:
            raise WDError(rc, self.lib.wd_ptc_last_error().decode())
        self.handle = handle
        self.n_weights = int(self.lib.wd_ptc_weight_count(self.handle))

    def _chk(self, rc):
        if rc != WD_OK:
            raise WDError(rc, self.lib.wd_ptc_last_error().decode())

    def close(self):
        if getattr(self, "handle", None):
            self.lib.wd_ptc_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_gauge(self, U: torch.Tensor):
        _dev(U, (self.V, 4, 3, 3), "U")
        self._chk(self.lib.wd_ptc_set_gauge(self.handle, ctypes.c_void_p(U.data_ptr())))

    def set_weights(self, W: torch.Tensor):
        _dev(W, (self.n_weights,), "W")
        self._chk(self.lib.wd_ptc_set_weights(self.handle, ctypes.c_void_p(W.data_ptr())))

    def get_weights(self) -> torch.Tensor:
        W = torch.empty(self.n_weights, dtype=torch.complex128, device="cuda")
        self._chk(self.lib.wd_ptc_get_weights(self.handle, ctypes.c_void_p(W.data_ptr())))
        return W

    def apply(self, r: torch.Tensor, out=None) -> torch.Tensor:
        _dev(r, (self.V, 3, 4), "r")
        y = torch.empty_like(r) if out is None else out
        torch.cuda.synchronize()
        self._chk(self.lib.wd_ptc_apply(self.handle, ctypes.c_void_p(y.data_ptr()),
                                        ctypes.c_void_p(r.data_ptr())))
        return y

    def loss_grad(self, r: torch.Tensor, e: torch.Tensor):
        """Loss sum_i |N(r_i) - e_i|^2 / |e_i|^2 over samples r, e [n, V, 3, 4] and its
        packed gradient dL/dRe W + i dL/dIm W (complex128 [n_weights])."""
        n = r.shape[0]
        _dev(r, (n, self.V, 3, 4), "r")
        _dev(e, (n, self.V, 3, 4), "e")
        g = torch.empty(self.n_weights, dtype=torch.complex128, device="cuda")
        loss = ctypes.c_double()
        torch.cuda.synchronize()
        self._chk(self.lib.wd_ptc_loss_grad(self.handle, ctypes.c_void_p(r.data_ptr()),
                                            ctypes.c_void_p(e.data_ptr()), n, ctypes.byref(loss),
                                            ctypes.c_void_p(g.data_ptr())))
        return loss.value, g

    def train_step(self, r: torch.Tensor, e: torch.Tensor, lr: float = 1e-3) -> float:
        """One Adam step on the samples; returns the loss before the step."""
        n = r.shape[0]
        _dev(r, (n, self.V, 3, 4), "r")
        _dev(e, (n, self.V, 3, 4), "e")
        loss = ctypes.c_double()
        torch.cuda.synchronize()
        self._chk(self.lib.wd_ptc_train_step(self.handle, ctypes.c_void_p(r.data_ptr()),
                                             ctypes.c_void_p(e.data_ptr()), n, float(lr),
                                             ctypes.byref(loss)))
        return loss.value

    def gemm_tn(self, A: torch.Tensor, B: torch.Tensor) -> torch.Tensor:
        """D = A^T B on the transposed (weight-gradient) tensor-core GEMM, for tests."""
        R, M = A.shape
        N = B.shape[1]
        D = torch.empty((M, N), dtype=torch.float32, device="cuda")
        torch.cuda.synchronize()
        self._chk(self.lib.wd_tc_gemm_bf16_tn(self.handle, ctypes.c_void_p(A.data_ptr()),
                                              ctypes.c_void_p(B.data_ptr()),
                                              ctypes.c_void_p(D.data_ptr()), R, M, N))
        return D

    def set_fused(self, on: bool = True):
        """Layers of apply() with 16 input channels as one fused transport +
        tensor-core kernel (default), or gathered operand + GEMM (on=False)."""
        self._chk(self.lib.wd_ptc_set_fused(self.handle, int(bool(on))))

    def set_wait_limit(self, polls: int = 1 << 26, withhold_mma: bool = False):
        """Polls per bounded GEMM wait; withhold_mma (tests) makes the GEMMs issue no MMA."""
        self._chk(self.lib.wd_ptc_set_wait_limit(self.handle, int(polls), int(withhold_mma)))

    def gemm(self, A: torch.Tensor, B: torch.Tensor) -> torch.Tensor:
        """D = A B^T on the tensor-core GEMM (bf16 in, fp32 out), for tests."""
        M, K = A.shape
        N = B.shape[0]
        D = torch.empty((M, N), dtype=torch.float32, device="cuda")
        torch.cuda.synchronize()
        self._chk(self.lib.wd_tc_gemm_bf16(self.handle, ctypes.c_void_p(A.data_ptr()),
                                           ctypes.c_void_p(B.data_ptr()),
                                           ctypes.c_void_p(D.data_ptr()), M, N, K))
        return D


_ptc_sigs_done = False


def _setup_ptc_signatures(lib):
    global _ptc_sigs_done
    if _ptc_sigs_done:
        return
    vp, i, d, l = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_long
    sig = {
        "wd_ptc_create": (i, [ctypes.POINTER(vp), ctypes.POINTER(i), ctypes.POINTER(d), i,
                              ctypes.POINTER(i), vp]),
        "wd_ptc_destroy": (None, [vp]),
        "wd_ptc_set_gauge": (i, [vp, vp]),
        "wd_ptc_set_weights": (i, [vp, vp]),
        "wd_ptc_get_weights": (i, [vp, vp]),
        "wd_ptc_weight_count": (l, [vp]),
        "wd_ptc_apply": (i, [vp, vp, vp]),
        "wd_tc_gemm_bf16": (i, [vp, vp, vp, vp, l, i, i]),
        "wd_tc_gemm_bf16_tn": (i, [vp, vp, vp, vp, l, i, i]),
        "wd_ptc_set_wait_limit": (i, [vp, ctypes.c_uint, i]),
        "wd_ptc_set_fused": (i, [vp, i]),
        "wd_ptc_loss_grad": (i, [vp, vp, vp, i, ctypes.POINTER(d), vp]),
        "wd_ptc_train_step": (i, [vp, vp, vp, i, d, ctypes.POINTER(d)]),
        "wd_ptc_last_error": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _ptc_sigs_done = True


class Fgcr:
    """Flexible GCR on the full system with an optional learned right
    preconditioner (handle on a wd_fgcr)."""

    def __init__(self, op_lo: WilsonDirac, op_hi: WilsonDirac, net: "PtcNet | None" = None,
                 nkrylov: int = 16):
        self.lib = load_library()
        _setup_ptc_signatures(self.lib)
        vp, i = ctypes.c_void_p, ctypes.c_int
        for name, res, args in (("wd_fgcr_create", i, [ctypes.POINTER(vp), vp, vp, vp, i]),
                                ("wd_fgcr_destroy", None, [vp]),
                                ("wd_fgcr_solve", i, [vp, vp, vp, ctypes.c_double, i,
                                                      ctypes.POINTER(SolveInfo)]),
                                ("wd_fgcr_last_error", ctypes.c_char_p, [])):
            f = getattr(self.lib, name)
            f.restype = res
            f.argtypes = args
        self.ops = (op_lo, op_hi, net)     # keep them alive
        self.V = op_lo.V
        handle = ctypes.c_void_p()
        rc = self.lib.wd_fgcr_create(ctypes.byref(handle), op_lo.handle, op_hi.handle,
                                     net.handle if net is not None else None, int(nkrylov))
        if rc != WD_OK:
            raise WDError(rc, self.lib.wd_fgcr_last_error().decode())
        self.handle = handle

    def close(self):
        if getattr(self, "handle", None):
            self.lib.wd_fgcr_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, b: torch.Tensor, tol: float = 1e-10, maxiter: int = 2000, check=True):
        _dev(b, (self.V, 3, 4), "b")
        x = torch.empty_like(b)
        info = SolveInfo()
        torch.cuda.synchronize()
        rc = self.lib.wd_fgcr_solve(self.handle, ctypes.c_void_p(x.data_ptr()),
                                    ctypes.c_void_p(b.data_ptr()), float(tol), int(maxiter),
                                    ctypes.byref(info))
        if check and rc != WD_OK:
            raise WDError(rc, self.lib.wd_fgcr_last_error().decode())
        return SolveResult(x, rc, info.as_dict())


KRYLOV_METHODS = {"cgnr": 0, "crne": 1, "mcr1": 2, "mcr2": 3}


class Krylov:
    """CGNR, CRNE, MCR1 or MCR2 on the Schur system of a WD_F64 operator
    (the solvers of the paper's solver comparison; handle on a wd_krylov)."""

    def __init__(self, op: WilsonDirac, method: str):
        if method not in KRYLOV_METHODS:
            raise ValueError(f"method must be one of {sorted(KRYLOV_METHODS)}, got {method!r}")
        self.lib = load_library()
        vp, i = ctypes.c_void_p, ctypes.c_int
        for name, res, args in (("wd_krylov_create", i, [ctypes.POINTER(vp), vp, i]),
                                ("wd_krylov_destroy", None, [vp]),
                                ("wd_krylov_solve", i, [vp, vp, vp, ctypes.c_double, i, i,
                                                        ctypes.POINTER(SolveInfo)]),
                                ("wd_krylov_last_error", ctypes.c_char_p, [])):
            f = getattr(self.lib, name)
            f.restype = res
            f.argtypes = args
        self.op = op                      # keep it alive
        self.method = method
        self.V = op.V
        handle = ctypes.c_void_p()
        rc = self.lib.wd_krylov_create(ctypes.byref(handle), op.handle, KRYLOV_METHODS[method])
        if rc != WD_OK:
            raise WDError(rc, self.lib.wd_krylov_last_error().decode())
        self.handle = handle

    def close(self):
        if getattr(self, "handle", None):
            self.lib.wd_krylov_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, b: torch.Tensor, tol: float = 1e-10, maxiter: int = 20000, parity: int = 1,
              x0: torch.Tensor | None = None, check: bool = True) -> SolveResult:
        _dev(b, (self.V, 3, 4), "b")
        x = torch.zeros_like(b) if x0 is None else _dev(x0, (self.V, 3, 4), "x0").clone()
        info = SolveInfo()
        torch.cuda.synchronize()
        rc = self.lib.wd_krylov_solve(self.handle, ctypes.c_void_p(x.data_ptr()),
                                      ctypes.c_void_p(b.data_ptr()), float(tol), int(maxiter),
                                      int(parity), ctypes.byref(info))
        if check and rc != WD_OK:
            raise WDError(rc, self.lib.wd_krylov_last_error().decode())
        return SolveResult(x, rc, info.as_dict())

"""FP64 CPU oracle for the Wilson-Dirac hot path (arXiv:1401.2039).

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import this package.  The CUDA
library never loads it and shares no code with it.

The arithmetic lives in ``wilson_oracle.c`` (plain C, FP64, OpenMP over
sites); this module loads it through ctypes and adds the dense-matrix
builder used by the LU pins.  Every array is a numpy complex128 array in the
canonical layout:

* full-lattice spinor  ``[V, 3, 4]`` (colour, spin), site ``lex`` with x fastest
* half-lattice spinor  ``[V/2, 3, 4]``, entry ``lex // 2`` of each site of the parity
* gauge field          ``[V, 4, 3, 3]`` (direction mu = x, y, z, t; row; column)

Parity: every function here is pinned by ``tests/test_oracle_*.py``
(free-field closed form, gamma5-hermiticity, gauge covariance, Schur
identity, dense LU, kappa = 0; the conjugate-residual solvers by the dense
least-squares minimiser over their Krylov spaces); none is "parity
unpinned".
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .build import build_oracle, library_path

__all__ = [
    "gamma", "hop", "hop_sites", "apply", "apply_eo", "hop_eo", "schur_prepare",
    "schur_reconstruct", "cgnr", "solve", "dense_matrix", "num_threads", "set_num_threads",
    "build_oracle", "CR_METHODS", "cr", "solve_cr",
]

_lib = None


def _load():
    global _lib
    if _lib is None:
        build_oracle()
        lib = ctypes.CDLL(library_path())
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        lib.oracle_gamma.argtypes = [ctypes.c_int, dp]
        lib.oracle_hop.argtypes = [dp, dp, dp, ip, dp, ctypes.c_int]
        lib.oracle_hop_sites.argtypes = [dp, dp, dp, ip, dp, ctypes.c_int,
                                         ctypes.POINTER(ctypes.c_long), ctypes.c_long]
        lib.oracle_apply.argtypes = [dp, dp, dp, ip, ctypes.c_double, dp, ctypes.c_int]
        lib.oracle_apply_eo.argtypes = [dp, dp, dp, ip, ctypes.c_double, dp, ctypes.c_int, ctypes.c_int]
        lib.oracle_hop_eo.argtypes = [dp, dp, dp, ip, dp, ctypes.c_int, ctypes.c_int]
        lib.oracle_schur_prepare.argtypes = [dp, dp, dp, ip, ctypes.c_double, dp, ctypes.c_int]
        lib.oracle_schur_reconstruct.argtypes = [dp, dp, dp, dp, ip, ctypes.c_double, dp, ctypes.c_int]
        lib.oracle_cgnr.argtypes = [dp, dp, dp, ip, ctypes.c_double, dp, ctypes.c_int,
                                    ctypes.c_double, ctypes.c_int, ip, dp]
        lib.oracle_cgnr.restype = ctypes.c_int
        lib.oracle_solve.argtypes = [dp, dp, dp, ip, ctypes.c_double, dp, ctypes.c_int,
                                     ctypes.c_double, ctypes.c_int, ip]
        lib.oracle_solve.restype = ctypes.c_int
        d = ctypes.c_double
        lib.oracle_twist.argtypes = [dp, dp, ctypes.c_long, d, d, ctypes.c_int]
        lib.oracle_twist.restype = ctypes.c_int
        lib.oracle_apply_tm.argtypes = [dp, dp, dp, ip, d, d, dp, ctypes.c_int]
        lib.oracle_apply_eo_tm.argtypes = [dp, dp, dp, ip, d, d, dp, ctypes.c_int, ctypes.c_int]
        lib.oracle_schur_prepare_tm.argtypes = [dp, dp, dp, ip, d, d, dp, ctypes.c_int]
        lib.oracle_schur_reconstruct_tm.argtypes = [dp, dp, dp, dp, ip, d, d, dp, ctypes.c_int]
        lib.oracle_cgnr_tm.argtypes = [dp, dp, dp, ip, d, d, dp, ctypes.c_int, d, ctypes.c_int,
                                       ip, dp]
        lib.oracle_cgnr_tm.restype = ctypes.c_int
        lib.oracle_solve_tm.argtypes = [dp, dp, dp, ip, d, d, dp, ctypes.c_int, d, ctypes.c_int,
                                        ip]
        lib.oracle_solve_tm.restype = ctypes.c_int
        lib.oracle_cr.argtypes = [dp, dp, dp, ip, d, d, dp, ctypes.c_int, ctypes.c_int, d,
                                  ctypes.c_int, ip, dp]
        lib.oracle_cr.restype = ctypes.c_int
        lib.oracle_solve_cr.argtypes = [dp, dp, dp, ip, d, d, dp, ctypes.c_int, ctypes.c_int, d,
                                        ctypes.c_int, ip]
        lib.oracle_solve_cr.restype = ctypes.c_int
        lib.oracle_num_threads.restype = ctypes.c_int
        lib.oracle_set_num_threads.argtypes = [ctypes.c_int]
        _lib = lib
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _c128(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.complex128)


def _dims(dims) -> ctypes.Array:
    d = [int(v) for v in dims]
    if len(d) != 4 or any(v <= 0 for v in d) or d[0] % 2:
        raise ValueError(f"dims must be 4 positive ints with Lx even, got {dims}")
    return (ctypes.c_int * 4)(*d)


def _phase(phase) -> np.ndarray:
    ph = np.asarray(phase, dtype=np.complex128).reshape(4)
    return np.ascontiguousarray(np.stack([ph.real, ph.imag], axis=1).reshape(8))


def _vol(dims) -> int:
    return int(np.prod([int(v) for v in dims]))


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def set_num_threads(n: int) -> None:
    """OpenMP threads of the oracle's loops (for timing it on fewer cores)."""
    _load().oracle_set_num_threads(int(n))


def gamma(mu: int) -> np.ndarray:
    """gamma_mu (mu = 0..3 for x, y, z, t; 4 for gamma5) as a 4x4 complex matrix."""
    out = np.zeros(32, dtype=np.float64)
    _load().oracle_gamma(int(mu), _dp(out))
    return out.view(np.complex128).reshape(4, 4)


def hop(psi, U, dims, phase, dagger=False) -> np.ndarray:
    """Full-lattice hopping term H psi (or H^dag psi)."""
    psi, U = _c128(psi), _c128(U)
    out = np.empty_like(psi)
    ph = _phase(phase)
    _load().oracle_hop(_dp(out), _dp(psi), _dp(U), _dims(dims), _dp(ph), int(bool(dagger)))
    return out


def hop_sites(psi, U, dims, phase, sites, dagger=False) -> np.ndarray:
    """(H psi)(x) at the listed lex sites only, shape [len(sites), 3, 4]."""
    psi, U = _c128(psi), _c128(U)
    sites = np.ascontiguousarray(sites, dtype=np.int64)
    out = np.empty((len(sites), 3, 4), dtype=np.complex128)
    ph = _phase(phase)
    _load().oracle_hop_sites(_dp(out), _dp(psi), _dp(U), _dims(dims), _dp(ph), int(bool(dagger)),
                             sites.ctypes.data_as(ctypes.POINTER(ctypes.c_long)), len(sites))
    return out


def apply(psi, U, dims, kappa, phase, dagger=False) -> np.ndarray:
    """Full Wilson-Dirac operator D psi = psi - kappa H psi (Fig. dirac, mu = 0)."""
    psi, U = _c128(psi), _c128(U)
    out = np.empty_like(psi)
    ph = _phase(phase)
    _load().oracle_apply(_dp(out), _dp(psi), _dp(U), _dims(dims), float(kappa), _dp(ph),
                         int(bool(dagger)))
    return out


def hop_eo(psi_half, U, dims, phase, out_parity, dagger=False) -> np.ndarray:
    """P_p H P_q^t psi: hopping term from parity q = 1 - p onto parity p."""
    psi_half, U = _c128(psi_half), _c128(U)
    out = np.empty_like(psi_half)
    ph = _phase(phase)
    _load().oracle_hop_eo(_dp(out), _dp(psi_half), _dp(U), _dims(dims), _dp(ph),
                          int(out_parity), int(bool(dagger)))
    return out


def apply_eo(psi_half, U, dims, kappa, phase, parity=1, dagger=False) -> np.ndarray:
    """Schur operator Mhat_p = I - kappa^2 P_p H P_q^t P_q H P_p^t (Alg. schur)."""
    psi_half, U = _c128(psi_half), _c128(U)
    out = np.empty_like(psi_half)
    ph = _phase(phase)
    _load().oracle_apply_eo(_dp(out), _dp(psi_half), _dp(U), _dims(dims), float(kappa),
                            _dp(ph), int(parity), int(bool(dagger)))
    return out


def schur_prepare(b_full, U, dims, kappa, phase, parity=1) -> np.ndarray:
    """bhat_p = b_p + kappa P_p H P_q^t b_q (Alg. schur)."""
    b_full, U = _c128(b_full), _c128(U)
    out = np.empty((_vol(dims) // 2, 3, 4), dtype=np.complex128)
    ph = _phase(phase)
    _load().oracle_schur_prepare(_dp(out), _dp(b_full), _dp(U), _dims(dims), float(kappa),
                                 _dp(ph), int(parity))
    return out


def schur_reconstruct(x_half, b_full, U, dims, kappa, phase, parity=1) -> np.ndarray:
    """Full solution from x_p: x_q = b_q + kappa P_q H P_p^t x_p (Alg. schur)."""
    x_half, b_full, U = _c128(x_half), _c128(b_full), _c128(U)
    out = np.empty_like(b_full)
    ph = _phase(phase)
    _load().oracle_schur_reconstruct(_dp(out), _dp(x_half), _dp(b_full), _dp(U), _dims(dims),
                                     float(kappa), _dp(ph), int(parity))
    return out


def cgnr(b_half, U, dims, kappa, phase, parity=1, tol=1e-12, maxiter=10000):
    """Alg. CGNR on Mhat_p.  Returns (x, iterations, converged, ||r_k|| history)."""
    b_half, U = _c128(b_half), _c128(U)
    x = np.empty_like(b_half)
    it = ctypes.c_int(0)
    hist = np.zeros(maxiter + 1, dtype=np.float64)
    ph = _phase(phase)
    rc = _load().oracle_cgnr(_dp(x), _dp(b_half), _dp(U), _dims(dims), float(kappa), _dp(ph),
                             int(parity), float(tol), int(maxiter), ctypes.byref(it), _dp(hist))
    return x, it.value, rc == 0, hist[: it.value + 1].copy()


def solve(b_full, U, dims, kappa, phase, parity=1, tol=1e-12, maxiter=10000):
    """Goal xx = Dirac^-1 bb with templates "CGNR schur".  Returns (x, iterations, converged)."""
    b_full, U = _c128(b_full), _c128(U)
    x = np.empty_like(b_full)
    it = ctypes.c_int(0)
    ph = _phase(phase)
    rc = _load().oracle_solve(_dp(x), _dp(b_full), _dp(U), _dims(dims), float(kappa), _dp(ph),
                              int(parity), float(tol), int(maxiter), ctypes.byref(it))
    return x, it.value, rc == 0


def dense_matrix(U, dims, kappa, phase, dagger=False, mu=None) -> np.ndarray:
    """D as a dense (12V x 12V) matrix, built column by column from ``apply``
    (``apply_tm`` with the twisted mass mu when given).
    Row/column index = lex * 12 + colour * 4 + spin.  Small lattices only."""
    n = 12 * _vol(dims)
    if n > 12 * 4 ** 4:
        raise ValueError("dense_matrix is meant for lattices of at most 4^4 sites")
    M = np.empty((n, n), dtype=np.complex128)
    e = np.zeros(n, dtype=np.complex128)
    for j in range(n):
        e[:] = 0
        e[j] = 1
        v = e.reshape(-1, 3, 4)
        col = (apply(v, U, dims, kappa, phase, dagger) if mu is None
               else apply_tm(v, U, dims, kappa, mu, phase, dagger))
        M[:, j] = col.reshape(n)
    return M


# ---------------------------------------------------------------- twisted mass
# Fig. "dirac" with mu != 0: D = I + 2 i kappa mu gamma_5 - kappa H, whose
# diagonal parity blocks A = I + 2 i kappa mu gamma_5 enter Alg. "schur".

def twist(psi, kappa, mu, inverse=False) -> np.ndarray:
    """A psi (or A^-1 psi) site by site, A = I + 2 i kappa mu gamma_5."""
    psi = _c128(psi)
    out = np.empty_like(psi)
    rc = _load().oracle_twist(_dp(out), _dp(psi), psi.size // 12, float(kappa), float(mu),
                              int(bool(inverse)))
    if rc != 0:
        raise RuntimeError("gamma_5 of the oracle's basis is not diagonal")
    return out


def apply_tm(psi, U, dims, kappa, mu, phase, dagger=False) -> np.ndarray:
    """D psi = A psi - kappa H psi (dagger: A(-mu) psi - kappa H^dag psi)."""
    psi, U = _c128(psi), _c128(U)
    out = np.empty_like(psi)
    _load().oracle_apply_tm(_dp(out), _dp(psi), _dp(U), _dims(dims), float(kappa), float(mu),
                            _dp(_phase(phase)), int(bool(dagger)))
    return out


def apply_eo_tm(psi_half, U, dims, kappa, mu, phase, parity=1, dagger=False) -> np.ndarray:
    """Mhat_p = A - kappa^2 P_p H P_q^t A^-1 P_q H P_p^t (dagger: H^dag, -mu)."""
    psi_half, U = _c128(psi_half), _c128(U)
    out = np.empty_like(psi_half)
    _load().oracle_apply_eo_tm(_dp(out), _dp(psi_half), _dp(U), _dims(dims), float(kappa),
                               float(mu), _dp(_phase(phase)), int(parity), int(bool(dagger)))
    return out


def schur_prepare_tm(b_full, U, dims, kappa, mu, phase, parity=1) -> np.ndarray:
    """bhat_p = b_p + kappa P_p H P_q^t A^-1 b_q."""
    b_full, U = _c128(b_full), _c128(U)
    out = np.empty((_vol(dims) // 2, 3, 4), dtype=np.complex128)
    _load().oracle_schur_prepare_tm(_dp(out), _dp(b_full), _dp(U), _dims(dims), float(kappa),
                                    float(mu), _dp(_phase(phase)), int(parity))
    return out


def schur_reconstruct_tm(x_half, b_full, U, dims, kappa, mu, phase, parity=1) -> np.ndarray:
    """Full solution from x_p: x_q = A^-1 (b_q + kappa P_q H P_p^t x_p)."""
    x_half, b_full, U = _c128(x_half), _c128(b_full), _c128(U)
    out = np.empty_like(b_full)
    _load().oracle_schur_reconstruct_tm(_dp(out), _dp(x_half), _dp(b_full), _dp(U), _dims(dims),
                                        float(kappa), float(mu), _dp(_phase(phase)), int(parity))
    return out


def cgnr_tm(b_half, U, dims, kappa, mu, phase, parity=1, tol=1e-12, maxiter=10000):
    """Alg. CGNR on the twisted-mass Mhat_p.  Returns (x, iterations, converged, history)."""
    b_half, U = _c128(b_half), _c128(U)
    x = np.empty_like(b_half)
    it = ctypes.c_int(0)
    hist = np.zeros(maxiter + 1, dtype=np.float64)
    rc = _load().oracle_cgnr_tm(_dp(x), _dp(b_half), _dp(U), _dims(dims), float(kappa), float(mu),
                                _dp(_phase(phase)), int(parity), float(tol), int(maxiter),
                                ctypes.byref(it), _dp(hist))
    return x, it.value, rc == 0, hist[: it.value + 1].copy()


def solve_tm(b_full, U, dims, kappa, mu, phase, parity=1, tol=1e-12, maxiter=10000):
    """x = D^-1 b with the twisted mass ("CGNR schur").  Returns (x, iterations, converged)."""
    b_full, U = _c128(b_full), _c128(U)
    x = np.empty_like(b_full)
    it = ctypes.c_int(0)
    rc = _load().oracle_solve_tm(_dp(x), _dp(b_full), _dp(U), _dims(dims), float(kappa), float(mu),
                                 _dp(_phase(phase)), int(parity), float(tol), int(maxiter),
                                 ctypes.byref(it))
    return x, it.value, rc == 0


# ------------------------------------------------------- conjugate residual
# Sec. 5 compares CRNE, MCR1 and MCR2 with CGNR on the Schur system without
# defining them; wilson_oracle.c states the textbook readings (CR of Saad,
# Alg. 6.20, on A A^dag and on gamma_5 A).

CR_METHODS = {"crne": 1, "mcr1": 2, "mcr2": 3}


def cr(b_half, U, dims, kappa, phase, method, mu=0.0, parity=1, tol=1e-12, maxiter=10000):
    """CRNE / MCR1 / MCR2 on Mhat_p (twisted mass mu, CRNE only: MCR needs
    gamma5-hermiticity).  Returns (x, iterations, status, ||r_k|| history);
    status 0 converged, 1 maxiter, 2 breakdown."""
    b_half, U = _c128(b_half), _c128(U)
    x = np.empty_like(b_half)
    it = ctypes.c_int(0)
    hist = np.zeros(maxiter + 1, dtype=np.float64)
    rc = _load().oracle_cr(_dp(x), _dp(b_half), _dp(U), _dims(dims), float(kappa), float(mu),
                           _dp(_phase(phase)), int(parity), CR_METHODS[method], float(tol),
                           int(maxiter), ctypes.byref(it), _dp(hist))
    if rc < 0:
        raise ValueError("oracle_cr: unknown method, MCR with mu != 0 or non-diagonal gamma_5")
    return x, it.value, rc, hist[: it.value + 1].copy()


def solve_cr(b_full, U, dims, kappa, phase, method, mu=0.0, parity=1, tol=1e-12, maxiter=10000):
    """x = D^-1 b with Alg. "schur" around CRNE / MCR1 / MCR2.
    Returns (x, iterations, status)."""
    b_full, U = _c128(b_full), _c128(U)
    x = np.empty_like(b_full)
    it = ctypes.c_int(0)
    rc = _load().oracle_solve_cr(_dp(x), _dp(b_full), _dp(U), _dims(dims), float(kappa),
                                 float(mu), _dp(_phase(phase)), int(parity), CR_METHODS[method],
                                 float(tol), int(maxiter), ctypes.byref(it))
    if rc < 0:
        raise ValueError("oracle_solve_cr: unknown method, MCR with mu != 0 or non-diagonal "
                         "gamma_5")
    return x, it.value, rc

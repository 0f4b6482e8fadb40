"""Seeded synthetic inputs: SU(3) gauge fields, Gaussian and point sources.

This module is the one piece shared by the oracle side and the CUDA side: it
draws inputs and holds none of the Wilson-Dirac arithmetic.  Everything is
numpy complex128 in the canonical layout

* gauge field ``[V, 4, 3, 3]`` (site lex with x fastest; mu = x, y, z, t; row; col)
* spinor      ``[V, 3, 4]``    (colour, spin)

The paper measures on real gauge configurations that are not available;
these seeded fields stand in for them:

* links ``U = exp(i eps H)``, ``H = sum_a c_a lambda_a / 2`` over the eight
  Gell-Mann matrices, ``c_a ~ N(0, 1)``, then re-unitarised (Gram-Schmidt of
  rows 0 and 1, row 2 = conj(row0 x row1)) so that det U = 1 to rounding;
* sources: complex Gaussian with E|z|^2 = 1 (real and imaginary parts
  N(0, 1/2)), or unit point sources.
"""
from __future__ import annotations

import os

import numpy as np

_CHUNK = 1 << 16  # matrices per generator chunk (part of the field's definition)


def volume(dims) -> int:
    return int(np.prod([int(d) for d in dims]))


def gell_mann() -> np.ndarray:
    """The eight Gell-Mann matrices, shape (8, 3, 3)."""
    lam = np.zeros((8, 3, 3), dtype=np.complex128)
    lam[0][0, 1] = lam[0][1, 0] = 1
    lam[1][0, 1], lam[1][1, 0] = -1j, 1j
    lam[2][0, 0], lam[2][1, 1] = 1, -1
    lam[3][0, 2] = lam[3][2, 0] = 1
    lam[4][0, 2], lam[4][2, 0] = -1j, 1j
    lam[5][1, 2] = lam[5][2, 1] = 1
    lam[6][1, 2], lam[6][2, 1] = -1j, 1j
    lam[7][0, 0] = lam[7][1, 1] = 1 / np.sqrt(3)
    lam[7][2, 2] = -2 / np.sqrt(3)
    return lam


def _mm_soa(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Products of batches of 3x3 matrices stored as [3, 3, n] (long contiguous
    vectors per entry, so every numpy call streams n elements)."""
    c = np.empty_like(a)
    for i in range(3):
        for k in range(3):
            c[i, k] = a[i, 0] * b[0, k] + a[i, 1] * b[1, k] + a[i, 2] * b[2, k]
    return c


def _expm_soa(X: np.ndarray) -> np.ndarray:
    """exp(X) for [3, 3, n] batches: scaling and squaring (2^-4) with a
    degree-8 Taylor polynomial; for ||X|| < 2 the truncation is below 1e-14
    and the re-unitarisation that follows removes it from the group."""
    s = 4
    Y = X / (1 << s)
    eye = np.zeros_like(X)
    for i in range(3):
        eye[i, i] = 1
    E = eye.copy()
    term = eye
    for k in range(1, 9):
        term = _mm_soa(term, Y) / k
        E += term
    for _ in range(s):
        E = _mm_soa(E, E)
    return E


def reunitarise(U: np.ndarray) -> np.ndarray:
    """Project a batch of near-SU(3) matrices [..., 3, 3] onto SU(3):
    orthonormalise rows 0 and 1, then row 2 = conj(row0 x row1)."""
    r0 = U[..., 0, :]
    r0 = r0 / np.linalg.norm(r0, axis=-1, keepdims=True)
    r1 = U[..., 1, :]
    r1 = r1 - np.sum(np.conj(r0) * r1, axis=-1, keepdims=True) * r0
    r1 = r1 / np.linalg.norm(r1, axis=-1, keepdims=True)
    r2 = np.conj(np.cross(r0, r1))
    return np.stack([r0, r1, r2], axis=-2)


def _reunitarise_soa(U: np.ndarray) -> np.ndarray:
    """reunitarise for [3, 3, n] batches, returned as [n, 3, 3]."""
    r0, r1 = U[0], U[1]
    r0 = r0 / np.sqrt((np.abs(r0) ** 2).sum(axis=0))
    r1 = r1 - (np.conj(r0) * r1).sum(axis=0) * r0
    r1 = r1 / np.sqrt((np.abs(r1) ** 2).sum(axis=0))
    r2 = np.conj(np.stack([r0[1] * r1[2] - r0[2] * r1[1],
                           r0[2] * r1[0] - r0[0] * r1[2],
                           r0[0] * r1[1] - r0[1] * r1[0]]))
    return np.ascontiguousarray(np.stack([r0, r1, r2]).transpose(2, 0, 1))


def _links_chunk(args):
    seed, k, n, eps = args
    rng = np.random.default_rng((seed, k))
    c = rng.standard_normal((n, 8))
    H = np.einsum("aij,na->ijn", gell_mann() / 2, c)          # [3, 3, n]
    return _reunitarise_soa(_expm_soa(1j * eps * H))


def su3_links(dims, eps: float = 0.3, seed: int = 1, workers: int | None = None) -> np.ndarray:
    """Seeded gauge field U_mu(x) = exp(i eps sum_a c_a lambda_a / 2), [V, 4, 3, 3].

    The 4V matrices are drawn in fixed chunks of 2^16, chunk k from the
    generator seeded by (seed, k), so the field does not depend on how many
    threads build it (numpy releases the GIL inside its array kernels)."""
    V = volume(dims)
    n = 4 * V
    jobs = [(seed, k, min(_CHUNK, n - a), eps) for k, a in enumerate(range(0, n, _CHUNK))]
    out = np.empty((n, 3, 3), dtype=np.complex128)

    def run(k):
        out[k * _CHUNK:k * _CHUNK + jobs[k][2]] = _links_chunk(jobs[k])

    if workers is None:
        workers = min(16, os.cpu_count() or 1)
    if workers > 1 and len(jobs) > 1:
        from concurrent.futures import ThreadPoolExecutor
        with ThreadPoolExecutor(workers) as ex:
            list(ex.map(run, range(len(jobs))))
    else:
        for k in range(len(jobs)):
            run(k)
    return out.reshape(V, 4, 3, 3)


def unit_links(dims) -> np.ndarray:
    """Free field: every link is the identity."""
    V = volume(dims)
    U = np.zeros((V, 4, 3, 3), dtype=np.complex128)
    U[..., 0, 0] = U[..., 1, 1] = U[..., 2, 2] = 1
    return U


def random_su3(n: int, seed: int) -> np.ndarray:
    """n Haar-like random SU(3) matrices (QR of complex Gaussians, phase-fixed)."""
    rng = np.random.default_rng(seed)
    Z = (rng.standard_normal((n, 3, 3)) + 1j * rng.standard_normal((n, 3, 3))) / np.sqrt(2)
    Q, R = np.linalg.qr(Z)
    d = np.diagonal(R, axis1=-2, axis2=-1)
    Q = Q * (d / np.abs(d))[:, None, :]
    det = np.linalg.det(Q)
    Q[:, :, 2] = Q[:, :, 2] / det[:, None]  # det 1; column scale by a unit phase keeps unitarity
    return Q


def gaussian_spinor(n_sites: int, seed: int) -> np.ndarray:
    """Complex Gaussian spinor field [n_sites, 3, 4] with E|z|^2 = 1."""
    rng = np.random.default_rng(seed)
    re = rng.standard_normal((n_sites, 3, 4))
    im = rng.standard_normal((n_sites, 3, 4))
    return (re + 1j * im) / np.sqrt(2)


def point_source(dims, site: int, colour: int, spin: int) -> np.ndarray:
    """delta_{x, site} delta_{c, colour} delta_{s, spin}, [V, 3, 4]."""
    b = np.zeros((volume(dims), 3, 4), dtype=np.complex128)
    b[site, colour, spin] = 1
    return b


def coords(dims) -> np.ndarray:
    """Coordinates (x, y, z, t) of every lex site, shape [V, 4]."""
    Lx, Ly, Lz, Lt = (int(d) for d in dims)
    t, z, y, x = np.meshgrid(np.arange(Lt), np.arange(Lz), np.arange(Ly), np.arange(Lx),
                             indexing="ij")
    return np.stack([x.ravel(), y.ravel(), z.ravel(), t.ravel()], axis=1)


def parity_sites(dims, parity: int) -> np.ndarray:
    """Lex indices of the sites of one parity, in half-lattice order (lex // 2)."""
    c = coords(dims)
    return np.nonzero(c.sum(axis=1) % 2 == parity)[0]


def to_half(full: np.ndarray, dims, parity: int) -> np.ndarray:
    return np.ascontiguousarray(full[parity_sites(dims, parity)])


def from_halves(even: np.ndarray, odd: np.ndarray, dims) -> np.ndarray:
    out = np.empty((volume(dims),) + even.shape[1:], dtype=even.dtype)
    out[parity_sites(dims, 0)] = even
    out[parity_sites(dims, 1)] = odd
    return out

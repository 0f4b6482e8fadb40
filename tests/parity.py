"""Comparison of a GPU field with the oracle's: norm-wise and site by site.

Norm-wise: ||gpu - oracle|| / ||oracle|| over the whole field.  On a field
of N sites this hides a wrong site whose error is about tol * sqrt(N) of a
site's norm, so every operator comparison also bounds each site:

    max_x ||gpu(x) - oracle(x)|| / max(||oracle(x)||, floor),

with floor = 0.1 * the root-mean-square site norm (it only matters for
sparse fields such as point sources, whose zero sites must stay near zero;
Gaussian fields have no site below 0.45 of the RMS norm).

Per-site tolerances come from the unit roundoff u of the storage format:
an output site sums eight transported neighbours, each carrying the storage
rounding of its spinor and link (and, with FP16, the FP16 projection sum),
and is rounded once when stored, about 4 u per term; for the random fields
of these tests the terms' norms add to about sqrt(8) times the site's norm,
so 11 u bounds a site.  Measured on GB300 over several lattices and the
full 32^3 x 64 field: FP16 1.9 u (9.3e-4), BF16 1.4 u (5.5e-3), FP32
(u = 2^-24) 3.3 u, FP64 4.3 u.  FP16 takes 8 u = 3.9e-3 per site, tighter
than its norm-wise 2e-2; the other formats keep their norm-wise tolerance
per site (BF16 8 u = 3.1e-2 would be looser than 2e-2).
"""
from __future__ import annotations

import numpy as np

NORM_TOL = {"f64": 1e-13, "f32": 1e-6, "f16": 2e-2, "bf16": 2e-2}
SITE_TOL = {"f64": 1e-13, "f32": 1e-6, "f16": 4e-3, "bf16": 2e-2}
SITE_REALS = 24   # one site: 3 colours x 4 spins complex


def _sites(a: np.ndarray) -> np.ndarray:
    a = np.asarray(a)
    if np.iscomplexobj(a):
        return a.reshape(-1, SITE_REALS // 2)
    return a.reshape(-1, SITE_REALS)


def norm_error(got, ref) -> float:
    got = np.asarray(got).ravel()
    ref = np.asarray(ref).ravel()
    return float(np.linalg.norm(got - ref) / np.linalg.norm(ref))


def site_errors(got, ref) -> np.ndarray:
    """Per-site relative errors, with the floor described above."""
    g, r = _sites(got), _sites(ref)
    assert g.shape == r.shape, (g.shape, r.shape)
    n = np.linalg.norm(r, axis=1)
    floor = 0.1 * np.sqrt(np.mean(n ** 2))
    return np.linalg.norm(g - r, axis=1) / np.maximum(n, floor)


def check(got, ref, prec: str | None = None, norm_tol: float | None = None,
          site_tol: float | None = None, what=()):
    """Assert both bounds; tolerances default to the precision's."""
    nt = NORM_TOL[prec] if norm_tol is None else norm_tol
    st = SITE_TOL[prec] if site_tol is None else site_tol
    e = norm_error(got, ref)
    assert e < nt, ("norm-wise", what, e, nt)
    s = site_errors(got, ref)
    worst = int(np.argmax(s))
    assert s[worst] < st, ("per site", what, "site", worst, float(s[worst]), st)
    return e, float(s[worst])

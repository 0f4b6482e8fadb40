"""The seeded workloads (lattice shapes, kappa, boundary phases, seeds).

Shapes follow the paper's 24^3 x 48 benchmark lattice (Sec. 5) and the
sizes around it; the gauge configurations are synthetic (``fields.su3_links``).
"""
from __future__ import annotations

from dataclasses import dataclass, field

# Periodic in space, antiperiodic in time: phi = (1, 1, 1, -1).
APBC_T = (1.0 + 0j, 1.0 + 0j, 1.0 + 0j, -1.0 + 0j)


@dataclass(frozen=True)
class Workload:
    name: str
    dims: tuple          # (Lx, Ly, Lz, Lt)
    kappa: float
    prec: str            # storage precision of the inner Dslash
    recon: int           # 18 or 12 reals per link
    eps: float = 0.3     # gauge-field roughness
    gauge_seed: int = 1
    source_seed: int = 2
    phase: tuple = field(default=APBC_T)
    tol: float = 1e-10   # FP64 true residual ||b - D x|| / ||b||

    @property
    def volume(self) -> int:
        v = 1
        for d in self.dims:
            v *= d
        return v

    @property
    def vh(self) -> int:
        return self.volume // 2


WORKLOADS = {
    # plain FP64 apply + CG, the small case the oracle finishes in seconds
    "wilson_4x4x4x4_f64": Workload("wilson_4x4x4x4_f64", (4, 4, 4, 4), 0.12, "f64", 18),
    # even-odd, FP32 Dslash with FP64 reliable-update CG
    "wilson_16x16x16x32_f32": Workload("wilson_16x16x16x32_f32", (16, 16, 16, 32), 0.124,
                                       "f32", 18),
    # even-odd, half-precision storage with 12-real links
    "wilson_32x32x32x64_f16r12": Workload("wilson_32x32x32x64_f16r12", (32, 32, 32, 64), 0.124,
                                          "f16", 12),
    "wilson_32x32x32x64_f32": Workload("wilson_32x32x32x64_f32", (32, 32, 32, 64), 0.124,
                                       "f32", 18),
    # the paper's benchmark lattice (Sec. 5, 24^3 x 48)
    "wilson_24x24x24x48_f32": Workload("wilson_24x24x24x48_f32", (24, 24, 24, 48), 0.12,
                                       "f32", 18),
}

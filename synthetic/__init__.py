"""Seeded synthetic workloads shared by the oracle tests and the CUDA path.

Holds input generation only (gauge fields, sources, the workload table);
none of the Wilson-Dirac arithmetic lives here.
"""
from .fields import (coords, from_halves, gaussian_spinor, gell_mann, parity_sites,  # noqa: F401
                     point_source, random_su3, reunitarise, su3_links, to_half, unit_links,
                     volume)
from .workloads import WORKLOADS, Workload  # noqa: F401

"""GB300-native Wilson-Dirac hot path (arXiv:1401.2039): hopping term,
even-odd Schur operator and CGNR solve with mixed-precision reliable
updates, all in the CUDA library libwd (include/wd.h)."""
from .build import build_library  # noqa: F401
from .wd import (KRYLOV_METHODS, PRECISIONS, Fgcr, Krylov, PtcNet, SolveInfo,  # noqa: F401
                 SolveResult, WDError, WilsonBatch, WilsonDirac, load_library, solve_cg_multi)

__all__ = ["WilsonDirac", "WilsonBatch", "PtcNet", "Fgcr", "Krylov", "KRYLOV_METHODS", "solve_cg_multi", "WDError", "SolveInfo", "SolveResult", "PRECISIONS", "build_library",
           "load_library"]

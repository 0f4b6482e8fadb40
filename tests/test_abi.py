"""The C ABI library builds, loads and exports every function include/wd.h
declares, and rejects bad arguments before touching a GPU (CPU only)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include"))
           if f.endswith(".h")]


@pytest.fixture(scope="module")
def lib():
    from paper_1401_2039_gb300 import load_library
    return load_library()


def declared_functions():
    names = set()
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(wd_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("wd_apply", "wd_apply_eo", "wd_solve_cg", "wd_op_create",
                     "wd_op_set_gauge", "wd_dslash_eo"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings(lib):
    lib.wd_status_string.restype = ctypes.c_char_p
    assert lib.wd_status_string(0) == b"ok"
    assert lib.wd_status_string(2) == b"invalid lattice dimensions"
    assert lib.wd_status_string(99) == b"unknown status"


def _create(lib, dims, prec=0, recon=18, kappa=0.12, phase=(1, 0, 1, 0, 1, 0, -1, 0)):
    h = ctypes.c_void_p()
    d = (ctypes.c_int * 4)(*dims)
    ph = (ctypes.c_double * 8)(*phase)
    lib.wd_op_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_int),
                                 ctypes.c_double, ctypes.POINTER(ctypes.c_double), ctypes.c_int,
                                 ctypes.c_int, ctypes.c_void_p]
    return lib.wd_op_create(ctypes.byref(h), d, kappa, ph, prec, recon, None), h


@pytest.mark.parametrize("dims", [(3, 4, 4, 4), (4, 4, 5, 4), (4, 4, 4, 0), (0, 2, 2, 2),
                                  (4, -2, 4, 4), (4, 4, 4, 1)])
def test_create_rejects_bad_dims(lib, dims):
    rc, h = _create(lib, dims)
    assert rc == 2 and not h.value


@pytest.mark.parametrize("prec,recon", [(7, 18), (-1, 18), (0, 13), (1, 0)])
def test_create_rejects_bad_precision_or_recon(lib, prec, recon):
    rc, h = _create(lib, (4, 4, 4, 4), prec, recon)
    assert rc == 1 and not h.value


def test_create_rejects_non_finite(lib):
    rc, _ = _create(lib, (4, 4, 4, 4), kappa=float("nan"))
    assert rc == 1
    rc, _ = _create(lib, (4, 4, 4, 4), phase=(1, 0, 1, 0, 1, float("inf"), -1, 0))
    assert rc == 1


def test_null_handles_are_rejected(lib):
    lib.wd_apply.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_int]
    lib.wd_apply_eo.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_int, ctypes.c_int]
    lib.wd_solve_cg.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_double, ctypes.c_int,
                                                        ctypes.c_int, ctypes.c_void_p]
    assert lib.wd_apply(None, None, None, 0) == 1
    assert lib.wd_apply_eo(None, None, None, 1, 0) == 1
    assert lib.wd_solve_cg(None, None, None, 1e-10, 100, 1, None) == 1
    lib.wd_last_error.restype = ctypes.c_char_p
    assert b"null" in lib.wd_last_error()
    lib.wd_op_destroy(None)   # no-op
    lib.wd_apply_eo_residual.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_int, ctypes.c_int]
    assert lib.wd_apply_eo_residual(None, None, None, 1, 0) == 1
    lib.wd_apply_eo_residual_early.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_int, ctypes.c_int]
    assert lib.wd_apply_eo_residual_early(None, None, None, 1, 0) == 1
    lib.wd_op_set_twisted_mass.argtypes = [ctypes.c_void_p, ctypes.c_double]
    assert lib.wd_op_set_twisted_mass(None, 0.1) == 1
    lib.wd_op_twisted_mass.argtypes = [ctypes.c_void_p]
    lib.wd_op_twisted_mass.restype = ctypes.c_double
    assert lib.wd_op_twisted_mass(None) == 0.0
    lib.wd_dslash_tuning.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                                     ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_void_p]
    assert lib.wd_dslash_tuning(None, 0, None, 0, None, None, None, None) == -1
    lib.wd_krylov_create.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
    assert lib.wd_krylov_create(None, None, 1) == 1
    h = ctypes.c_void_p()
    assert lib.wd_krylov_create(ctypes.byref(h), None, 1) == 1 and not h.value
    lib.wd_krylov_solve.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_double, ctypes.c_int,
                                                            ctypes.c_int, ctypes.c_void_p]
    assert lib.wd_krylov_solve(None, None, None, 1e-10, 100, 1, None) == 1
    lib.wd_krylov_last_error.restype = ctypes.c_char_p
    assert b"null" in lib.wd_krylov_last_error()
    lib.wd_krylov_destroy(None)   # no-op
    lib.wd_solve_cg_multi.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                      ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double,
                                      ctypes.c_int, ctypes.c_int, ctypes.c_void_p]
    assert lib.wd_solve_cg_multi(None, 1, None, None, None, 1e-10, 100, 1, None) == 1
    lib.wd_solve_cg_host_stream.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                            ctypes.c_void_p, ctypes.c_double, ctypes.c_int,
                                            ctypes.c_int, ctypes.c_void_p]
    assert lib.wd_solve_cg_host_stream(None, 1, None, None, 1e-10, 100, 1, None) == 1


def test_product_path_has_no_cpu_fallback():
    import torch
    from paper_1401_2039_gb300 import WilsonDirac
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(RuntimeError, match="CUDA"):
        WilsonDirac((4, 4, 4, 4), 0.12)


def test_product_package_does_not_import_oracle():
    pkg = os.path.join(ROOT, "paper_1401_2039_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in src.lower(), f


def _header_enum(name):
    """{enumerator: value} of the typedef enum `name` in include/wd.h."""
    text = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "wd.h")).read(), flags=re.S)
    m = re.search(r"typedef enum\s*\{([^}]*)\}\s*" + name + r"\s*;", text)
    assert m, name
    return {k: int(v) for k, v in re.findall(r"(WD_[A-Z0-9_]+)\s*=\s*(-?\d+)", m.group(1))}


def test_binding_constants_match_the_header():
    """The binding's integer constants are the header's enums (a mismatch
    would send the wrong precision, method or status across the ABI)."""
    from paper_1401_2039_gb300 import wd
    prec = _header_enum("wd_prec")
    assert {k: prec["WD_" + k.upper()] for k in wd.PRECISIONS} == wd.PRECISIONS
    methods = _header_enum("wd_krylov_method")
    assert {k: methods["WD_KRYLOV_" + k.upper()] for k in wd.KRYLOV_METHODS} == wd.KRYLOV_METHODS
    assert len(methods) == len(wd.KRYLOV_METHODS)
    rec = _header_enum("wd_recovery")
    assert {k: rec["WD_RECOVER_" + k.upper()] for k in wd.RECOVERY} == wd.RECOVERY
    assert len(rec) == len(wd.RECOVERY)
    status = _header_enum("wd_status")
    for name, value in status.items():
        assert getattr(wd, name) == value, name


def test_solve_cg_multi_checks_lengths_before_any_call():
    from paper_1401_2039_gb300 import solve_cg_multi
    with pytest.raises(ValueError):
        solve_cg_multi([object()], [1, 2], [None])


def test_recovery_mode_arguments_are_checked(lib):
    """wd_op_set_recovery rejects a null handle, unknown modes and inner
    tolerances outside (0, 1) before any GPU work."""
    vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    lib.wd_op_set_recovery.argtypes = [vp, i, d]
    lib.wd_op_recovery.argtypes = [vp, ctypes.POINTER(d)]
    assert lib.wd_op_set_recovery(None, 1, 0.1) == 1
    assert lib.wd_op_recovery(None, None) == -1

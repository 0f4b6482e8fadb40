"""The oracle's pins have teeth: plant a plausible mistake in a copy of the
oracle source (on the CPU, in a temporary directory), build it, and check
that the pins of ``test_oracle_pins.py`` reject it.  The real oracle is
never modified."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "wilson_oracle.c")

# (description, original text, planted text)
MUTANTS = [
    ("projector sign swapped", "double sf = dagger ? +1.0 : -1.0;",
     "double sf = dagger ? -1.0 : +1.0;"),
    ("backward hop uses U instead of U^dag", "sum += wb * conj(Ub[3 * b + a])",
     "sum += wb * Ub[3 * a + b]"),
    ("backward phase not conjugated", "wb = conj(ph);", "wb = ph;"),
    ("forward link taken at x+mu", "const cplx *Uf = U + (site * 4 + mu) * 9;",
     "const cplx *Uf = U + (lf * 4 + mu) * 9;"),
    ("kappa^2 dropped in the Schur operator", "out[i] = in[i] - kappa * kappa * t[i];",
     "out[i] = in[i] - kappa * t[i];"),
    ("literal 2 kappa in the schur reconstruction", "xq[i] = bq[i] + kappa * hx[i];",
     "xq[i] = 2 * kappa * bq[i] + kappa * hx[i];"),
    ("CGNR beta inverted", "double beta = nz1 / nz;", "double beta = nz / nz1;"),
    ("gamma_x sign slip", "g[0][3] = I;  g[1][2] = I;", "g[0][3] = -I;  g[1][2] = I;"),
    ("twisted mass without its factor 2", "const cplx a = 1.0 + 2.0 * I * kappa * mu * g5[s][s];",
     "const cplx a = 1.0 + I * kappa * mu * g5[s][s];"),
    ("adjoint keeps the sign of mu", "double m = dagger ? -mu : mu;", "double m = mu;"),
    ("A instead of A^-1 in the reconstruction",
     "oracle_twist((double *)xq, (double *)v, vh, kappa, mu, 1);",
     "oracle_twist((double *)xq, (double *)v, vh, kappa, mu, 0);"),
]

# The conjugate-residual solvers sit on top of the operator that the pins
# above already hold; their mutants are run against the solver pins alone (a
# subset of the full set, so rejection by it implies rejection by all).
CR_MUTANTS = [
    ("MCR without gamma5 on the right-hand side", "if (method != 1) cr_gamma5(&c, r);",
     "if (method == 0) cr_gamma5(&c, r);"),
    ("CR step length from (r|r)", "const double alpha = rBr / nBp;",
     "const double alpha = nr / nBp;"),
    ("CR beta inverted", "const double beta = rBr1 / rBr;", "const double beta = rBr / rBr1;"),
    ("CRNE returns y instead of A^dag y", "if (method == 1)                                     /*",
     "if (method == 0)                                     /*"),
    ("CR recurrence for B p drops beta", "Bp[i] = Br[i] + beta * Bp[i];", "Bp[i] = Br[i] + Bp[i];"),
]

FAST_PINS = ("test_gamma_basis_clifford or test_free_field_plane_waves or "
             "test_gamma5_hermiticity or test_gauge_covariance or "
             "test_schur_blocks_dense or test_cgnr_schur_solve_matches_lu or "
             "test_twisted_free_field or test_twisted_adjoint_flips_mu or "
             "test_twisted_solve_matches_lu")
CR_PINS = ("test_cr_iterates_minimise_over_krylov_space or test_cr_solves_match_lu or "
           "test_cr_special_cases")


@pytest.mark.parametrize("desc,orig,planted,pins",
                         [m + (FAST_PINS,) for m in MUTANTS] + [m + (CR_PINS,) for m in CR_MUTANTS],
                         ids=[m[0] for m in MUTANTS + CR_MUTANTS])
def test_pins_reject_mutant(tmp_path, desc, orig, planted, pins):
    src = open(SRC).read()
    assert src.count(orig) == 1, f"mutation anchor not found: {orig}"
    mut = tmp_path / "mut.c"
    mut.write_text(src.replace(orig, planted))
    lib = tmp_path / "libmut.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", str(mut), "-o",
                    str(lib), "-lm"], check=True)
    env = dict(os.environ, WD_ORACLE_LIB=str(lib), OMP_NUM_THREADS="4")
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py"), "-k", pins],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 1 and "1 failed" in r.stdout, (desc, r.stdout[-2000:])

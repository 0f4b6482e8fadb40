"""The comparison the GPU tests use (tests/parity.py), exercised on the CPU
with planted errors: the per-site bound catches one wrong site that the
norm-wise tolerance lets through."""
import numpy as np
import pytest

from parity import check, site_errors

N_SITES = 4096   # the (16, 8, 8, 8) test lattice's half volume


def _field(seed):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((N_SITES, 3, 4)) + 1j * rng.standard_normal((N_SITES, 3, 4)))


def test_one_wrong_site_passes_norm_wise_but_fails_per_site():
    ref = _field(1)
    got = ref.copy()
    got[1234] = 0.0                          # a tail-tile bug that drops one site
    norm_err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert norm_err < 2e-2                   # hidden by the field-wide FP16 tolerance
    with pytest.raises(AssertionError, match="per site"):
        check(got, ref, "f16")
    assert int(np.argmax(site_errors(got, ref))) == 1234


def test_rounding_level_noise_passes():
    ref = _field(2)
    rng = np.random.default_rng(3)
    u = 2.0 ** -11
    got = ref * (1 + u * rng.uniform(-1, 1, ref.shape))   # one FP16 rounding per entry
    check(got, ref, "f16")


def test_zero_sites_of_a_sparse_field_are_held_near_zero():
    ref = np.zeros((N_SITES, 3, 4), dtype=complex)
    ref[:16] = _field(4)[:16]                # point-like source: most sites zero
    got = ref.copy()
    check(got, ref, "f64")
    got[2000, 1, 2] = 0.2                    # a stray value on a zero site (1% norm-wise)
    with pytest.raises(AssertionError, match="per site"):
        check(got, ref, "f16")

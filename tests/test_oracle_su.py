"""Pins of the truncated-sweep oracle (Sec. 4) against the exact methods and invariants.

When chi and chi_mps exceed every bond the sweep can produce, nothing is truncated and
the result must equal the exact transfer matrix; as chi grows it must converge to it.
"""
import numpy as np
import pytest

from td_inputs import point_sector_3d, rotated_phenomenological, repetition_phenomenological, sample_shots
from oracle import exact, su


@pytest.mark.parametrize("make", [
    lambda: point_sector_3d(3, 0.05),
    lambda: rotated_phenomenological(3, 2, 0.05, 0.04),
    lambda: repetition_phenomenological(5, 3, 0.07, 0.03),
])
def test_untruncated_sweep_is_exact(make):
    dem = make()
    det, _ = sample_shots(dem, 10, seed=21)
    tm = exact.transfer_matrix(dem, det)
    s4 = su.su_logprob(dem, det, chi=256, chi_mps=1024)
    np.testing.assert_allclose(s4, tm, rtol=0, atol=1e-10)


@pytest.mark.parametrize("deform", [False, True])
def test_class_tracking_forms_agree(deform):
    """Counter legs on every bottom site (observable as given) and the top readout
    (observable + all rows of H, class offset by the parity of m) give the same exact
    coset probabilities."""
    dem = point_sector_3d(3, 0.06)
    det, _ = sample_shots(dem, 8, seed=4)
    plan = su.SUPlan(dem, deform=deform)
    assert (len(plan.counter_sites) == 0) == deform
    s4 = su.su_logprob(dem, det, chi=256, chi_mps=1024, plan=plan)
    tm = exact.transfer_matrix(dem, det)
    np.testing.assert_allclose(s4, tm, atol=1e-10)


def test_sweep_half_rate_closed_form():
    dem = point_sector_3d(3, 0.5)
    det, _ = sample_shots(dem, 6, seed=2)
    s4 = su.su_logprob(dem, det, chi=64, chi_mps=256)
    np.testing.assert_allclose(s4, -(18 + 1) * np.log(2), atol=1e-10)


def test_convergence_in_chi():
    """Error against the exact value shrinks as chi grows (d = 4: bonds reach 8 untruncated)."""
    dem = point_sector_3d(4, 0.08)
    det, _ = sample_shots(dem, 6, seed=5)
    tm = exact.transfer_matrix(dem, det)
    errs = [np.abs(su.su_logprob(dem, det, chi=c, chi_mps=512) - tm).max() for c in (2, 4, 8)]
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 1e-10


def test_convergence_in_chi_mps():
    dem = point_sector_3d(4, 0.08)
    det, _ = sample_shots(dem, 4, seed=6)
    tm = exact.transfer_matrix(dem, det)
    errs = [np.abs(su.su_logprob(dem, det, chi=8, chi_mps=c) - tm).max() for c in (16, 64, 512)]
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 1e-10


def test_keep_count_rules():
    s = np.array([1.0, 0.5, 0.5 - 1e-12, 0.2, 1e-14])
    assert su.keep_count(s, 10, 1e-12, 1e-8) == 4          # cutoff drops 1e-14
    assert su.keep_count(s, 4, 1e-12, 1e-8) == 4
    assert su.keep_count(s, 2, 1e-12, 1e-8) == 1           # cut inside the 0.5 doublet
    assert su.keep_count(s, 3, 1e-12, 1e-8) == 3
    assert su.keep_count(np.ones(4), 2, 1e-12, 1e-8) == 2  # all degenerate: keep chi


def test_planted_mistake_is_caught():
    """Dropping the weights of the vertical mechanisms (a plausible slip) breaks the
    exactness pin by far more than its tolerance."""
    dem = rotated_phenomenological(3, 2, 0.05, 0.04)
    det, _ = sample_shots(dem, 4, seed=8)
    plan = su.SUPlan(dem)
    for t in range(plan.T - 1):
        plan.post[t] = [np.eye(plan.P[s]) for s in range(plan.S)]
    bad = su.su_logprob(dem, det, chi=256, chi_mps=1024, plan=plan)
    tm = exact.transfer_matrix(dem, det)
    assert np.abs(bad - tm).max() > 1e-2

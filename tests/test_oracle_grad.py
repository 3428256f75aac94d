"""Pins of the exact gradient d log P(m) / d p_j (P(m) = sum_L p_{m,L})."""
import numpy as np

from td_inputs import repetition_phenomenological, rotated_phenomenological, sample_shots
from oracle import exact


def _posterior_marginals(dem, m):
    """P(x_j = 1 | m) by enumerating every error pattern (tiny problems)."""
    n = dem.n_mech
    X = ((np.arange(1 << n)[:, None] >> np.arange(n)[None, :]) & 1).astype(np.uint8)
    H = dem.H_dense()
    ok = np.all((X @ H.T) % 2 == m[None, :], axis=1)
    p = dem.p
    w = np.prod(np.where(X == 1, p, 1 - p), axis=1) * ok
    return (w[:, None] * X).sum(axis=0) / w.sum()


def test_gradient_matches_posterior_marginals():
    """d log P / d p_j = pi_j / p_j - (1 - pi_j) / (1 - p_j), pi_j the posterior marginal."""
    dem = repetition_phenomenological(4, 2, 0.08, 0.05)
    rng = np.random.default_rng(3)
    dem = dem.with_rates(rng.uniform(0.01, 0.2, dem.n_mech))
    det, _ = sample_shots(dem, 5, seed=13)
    g = exact.grad_total_logprob(dem, det)
    for b in range(len(det)):
        pi = _posterior_marginals(dem, det[b])
        expect = pi / dem.p - (1 - pi) / (1 - dem.p)
        np.testing.assert_allclose(g[b], expect, rtol=1e-9, atol=1e-9)


def test_gradient_matches_central_differences():
    dem = rotated_phenomenological(3, 1, 0.05, 0.03)
    rng = np.random.default_rng(4)
    dem = dem.with_rates(np.exp(rng.uniform(np.log(1e-3), np.log(1e-2), dem.n_mech)) * 5)
    det, _ = sample_shots(dem, 3, seed=14)
    g = exact.grad_total_logprob(dem, det)
    lay = exact.Layering(dem)
    for j in (0, 5, 17, dem.n_mech - 1):
        h = 1e-6 * dem.p[j]
        pp = dem.p.copy(); pp[j] += h
        pm = dem.p.copy(); pm[j] -= h
        fp = exact.total_logprob(exact.transfer_matrix(dem.with_rates(pp), det, lay))
        fm = exact.total_logprob(exact.transfer_matrix(dem.with_rates(pm), det, lay))
        np.testing.assert_allclose(g[:, j], (fp - fm) / (2 * h), rtol=1e-6, atol=1e-6)


# ---- the gradient of the truncated sweep (the quantity td_grad_logprob computes) ------------
from oracle import su, frozen  # noqa: E402
from td_inputs import point_sector_3d  # noqa: E402


def test_sweep_gradient_untruncated_is_exact():
    """Without truncation the forced-rate gradient of the sweep is the exact gradient."""
    for dem in (rotated_phenomenological(3, 2, 0.05, 0.04), repetition_phenomenological(5, 3, 0.07, 0.03)):
        det, _ = sample_shots(dem, 3, seed=15)
        lp, g = su.su_grad_total_logprob(dem, det, chi=256, chi_mps=1024)
        lt = exact.total_logprob(exact.transfer_matrix(dem, det))
        np.testing.assert_allclose(lp, lt, rtol=1e-11, atol=1e-11)
        np.testing.assert_allclose(g, exact.grad_total_logprob(dem, det), rtol=1e-9, atol=1e-9)


def test_sweep_gradient_converges_in_chi():
    """Truncated: the error against the exact gradient shrinks as chi grows."""
    dem = point_sector_3d(3, 0.08)
    det, _ = sample_shots(dem, 1, seed=16)
    ge = exact.grad_total_logprob(dem, det)
    errs = [np.abs(su.su_grad_total_logprob(dem, det, chi=c, chi_mps=64)[1] - ge).max() for c in (1, 2, 4)]
    assert errs[0] > errs[1] > 1e-3 and errs[2] < 1e-10, errs   # measured: 14, 0.68, 3e-14


def test_frozen_projector_reading_is_rejected():
    """The replay of the recorded truncations reproduces the forward value, but its
    gradient is not the exact one even at chi large enough that nothing is truncated."""
    dem = repetition_phenomenological(5, 3, 0.07, 0.03)
    det, _ = sample_shots(dem, 1, seed=11)
    plan = su.SUPlan(dem)
    rec = frozen.record(plan, det[0], 256, 1024)
    assert abs(frozen.replay(plan, det[0], rec) - rec.logP) < 1e-12
    lp, gf = frozen.frozen_grad(dem, det, 256, 1024)
    ge = exact.grad_total_logprob(dem, det)
    assert np.abs(gf - ge).max() > 0.1


# ---- the reverse sweep of the oracle (oracle/reverse.py) --------------------------------------
from oracle import reverse  # noqa: E402


def test_reverse_sweep_untruncated_is_exact():
    for dem in (rotated_phenomenological(3, 2, 0.05, 0.04), repetition_phenomenological(5, 3, 0.07, 0.03),
                point_sector_3d(3, 0.05)):
        det, _ = sample_shots(dem, 2, seed=11)
        lp, g = reverse.reverse_grad_total_logprob(dem, det, chi=256, chi_mps=1024)
        np.testing.assert_allclose(lp, exact.total_logprob(exact.transfer_matrix(dem, det)), rtol=1e-11, atol=1e-11)
        np.testing.assert_allclose(g, exact.grad_total_logprob(dem, det), rtol=1e-10, atol=1e-10)


def test_reverse_sweep_truncated_matches_differences():
    """With truncation: central differences of su.su_logprob (step 1e-5 p_j)."""
    dem = point_sector_3d(3, 0.08)
    det, _ = sample_shots(dem, 2, seed=17)
    lp, g = reverse.reverse_grad_total_logprob(dem, det, chi=2, chi_mps=8)
    for j in range(0, dem.n_mech, 5):
        h = 1e-5 * dem.p[j]
        pp, pm = dem.p.copy(), dem.p.copy()
        pp[j] += h
        pm[j] -= h
        a = su.su_logprob(dem.with_rates(pp), det, 2, 8)
        b = su.su_logprob(dem.with_rates(pm), det, 2, 8)
        fd = (np.logaddexp(a[:, 0], a[:, 1]) - np.logaddexp(b[:, 0], b[:, 1])) / (2 * h)
        np.testing.assert_allclose(g[:, j], fd, rtol=1e-6, atol=1e-6)


def test_reverse_sweep_planted_mistake_is_caught(monkeypatch):
    """Dropping the truncated SVD's projection term (I - U U^T) U-bar S^-1 V^T from the
    oracle's reverse sweep breaks its agreement with the exact gradient even without
    truncation (the kept subspaces rotate with the rates): the pins see such a slip."""
    dem = repetition_phenomenological(5, 3, 0.07, 0.03)
    det, _ = sample_shots(dem, 1, seed=11)
    good = reverse._svd_adjoint

    def slipped(U, s, V, k, Ubar, Vbar, Sbar, rel=1e-13):
        full = good(U, s, V, k, Ubar, Vbar, Sbar, rel)
        r = int(np.count_nonzero(s > rel * s[0]))
        Uf, Vf, sf = U[:, :r], V[:, :r], s[:r]
        Ub = np.zeros((U.shape[0], r))
        if Ubar is not None:
            Ub[:, :k] = Ubar
        return full - (Ub - Uf @ (Uf.T @ Ub)) @ np.diag(1 / sf) @ Vf.T

    monkeypatch.setattr(reverse, "_svd_adjoint", slipped)
    _, g = reverse.reverse_grad_total_logprob(dem, det, chi=256, chi_mps=1024)
    assert np.abs(g - exact.grad_total_logprob(dem, det)).max() > 1e-3

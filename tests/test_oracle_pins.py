"""Pins of the truncated sweep's two truncation steps against optimal low-rank truncation.

Exactness at large chi and convergence in chi cannot tell how the oracle truncates: with
nothing cut, the result does not depend on the bond environment (Sec. 4's simple update
uses the diagonal lambda weights of the other bonds) nor on which side of a zip-up cut
keeps the singular vectors.  Both steps are pinned here where the mathematics fixes
their result at a truncating bond dimension:

* Simple update (Sec. 4).  When the two sites' environments are exact -- the state is a
  tree in canonical form around the bond -- the simple-update truncation is the optimal
  (Eckart-Young) rank-chi truncation of the whole state across that bond.  On a chain of
  four sites, from a product state, the gates on bonds 0-1 and 2-3 are exact SVD splits,
  so sites 0 and 3 are isometries and lambda_01, lambda_23 are the exact environments of
  the gate on bond 1-2.  The kept lambda must be the leading Schmidt values of the dense
  state across the cut {0,1} | {2,3}, and the contracted PEPS must equal its rank-chi
  truncation.
* Zip-up cut of the final contraction (Sec. 4, chi_MPS of Sec. 5).  When the part of the
  row right of a cut is an isometry, the leading left singular vectors of the cut matrix
  are those of the whole row state, so the truncated boundary MPS is the optimal rank-
  chi_mps truncation of the row state across that vertical bond.

A planted slip in each step (environment weights omitted; one vector too few kept at a
truncating cut) passes the older exactness pins but fails these.
"""
import numpy as np
import pytest

from oracle import exact, su
from td_inputs import DEM, rotated_phenomenological, point_sector_3d, sample_shots

def chain_dem(n=4):
    """n detectors on a line in one layer, a two-detector mechanism per neighbouring pair
    and one single-detector mechanism carrying the observable (read out at the end)."""
    dets = [(s, s + 1) for s in range(n - 1)] + [(0,)]
    obs = [()] * (n - 1) + [(0,)]
    xyt = np.array([(s, 0, 0) for s in range(n)], dtype=np.int32)
    return DEM(n, 1, dets, obs, np.full(len(dets), 0.1), xyt, name="chain")


def peps_state(peps):
    """Dense amplitude psi[sigma_0 .. sigma_{S-1}] * exp(logscale) of a chain PEPS
    (Gamma-lambda form: every bond weight appears once)."""
    plan = peps.plan
    psi = np.ones(1).reshape(1, 1)            # (phys so far, open bond)
    for s in range(plan.S):
        g = peps.G[s]
        bonds = plan.site_bonds[s]
        # chain: site s has bonds (left, right) with the left one first when both exist
        if s == 0:
            g = g.reshape(g.shape[0], 1, -1)
        elif s == plan.S - 1:
            g = g.reshape(g.shape[0], -1, 1)
        if s > 0:
            lam = peps.lam[bonds[0]]
            psi = psi * lam[None, :]
        psi = np.einsum("pa,qab->pqb", psi, g).reshape(-1, g.shape[2])
    return psi.reshape(-1) * np.exp(peps.logscale)


def gate_dense(psi, S, a, b, p):
    """Apply (1 - p) I + p X_a X_b to the dense state over S two-valued sites."""
    t = psi.reshape((2,) * S)
    flipped = np.flip(np.flip(t, axis=a), axis=b)
    return ((1 - p) * t + p * flipped).reshape(-1)


def rank_truncate(M, k):
    U, s, Vt = np.linalg.svd(M, full_matrices=False)
    return (U[:, :k] * s[:k]) @ Vt[:k], s


def simple_update_case(seed, chi, peps_cls=su.PEPS):
    rng = np.random.default_rng(seed)
    plan = su.SUPlan(chain_dem(4))
    assert plan.S == 4 and plan.P == [2, 2, 2, 2]
    peps = peps_cls(plan)
    vecs = []
    for s in range(4):
        M = rng.uniform(-1.0, 1.0, size=(2, 2))
        peps.apply_local(s, M)
        vecs.append(M[:, 0])
    rates = rng.uniform(0.05, 0.4, size=3)
    bond = {tuple(b): i for i, b in enumerate(plan.bonds)}
    # colour order of the sweep: bonds 0-1 and 2-3, then 1-2 (the truncating one)
    for (a, b), p in (((0, 1), rates[0]), ((2, 3), rates[2]), ((1, 2), rates[1])):
        peps.gate(bond[(a, b)], p, 1, 1, chi if (a, b) == (1, 2) else 64, 1e-12, 1e-8)
    psi = np.einsum("a,b,c,d->abcd", *vecs).reshape(-1)
    for (a, b), p in (((0, 1), rates[0]), ((2, 3), rates[2]), ((1, 2), rates[1])):
        psi = gate_dense(psi, 4, a, b, p)
    return peps, bond, psi


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_simple_update_is_optimal_truncation_with_exact_environment(seed):
    peps, bond, psi = simple_update_case(seed, chi=1)
    best, s = rank_truncate(psi.reshape(4, 4), 1)
    assert s[1] > 1e-3 * s[0]                               # the cut really truncates
    lam12 = peps.lam[bond[(1, 2)]]
    np.testing.assert_allclose(lam12, s[:1] / s[0], rtol=0, atol=1e-12)
    np.testing.assert_allclose(peps_state(peps), best.reshape(-1), rtol=0, atol=1e-12 * np.abs(psi).max())
    # the other two bonds carry the exact Schmidt values of their (product-state) pairs
    for (a, b) in ((0, 1), (2, 3)):
        lam = peps.lam[bond[(a, b)]]
        assert lam[0] == 1.0 and lam.shape == (2,)


def test_simple_update_untruncated_chain_is_exact():
    peps, bond, psi = simple_update_case(7, chi=2)
    np.testing.assert_allclose(peps_state(peps), psi, rtol=0, atol=1e-12 * np.abs(psi).max())


class PEPSNoEnv(su.PEPS):
    """Planted slip: the other bonds' lambda left out of the environment (and, consistently,
    out of the restore), so every untruncated contraction is still exact."""

    def _env(self, s, skip, inv=False):
        return self.G[s]


class PEPSSquaredEnv(su.PEPS):
    """Planted slip: the other bonds' lambda squared in the environment (and in the
    restore, 1 / lambda^2)."""

    def _env(self, s, skip, inv=False):
        g = super()._env(s, skip, inv)
        return self._twice(g, s, skip, inv)

    def _twice(self, g, s, skip, inv):
        for pos, b in enumerate(self.plan.site_bonds[s]):
            if b == skip:
                continue
            w = self.lam[b]
            if inv:
                w = np.where(w > 0, 1.0 / np.where(w > 0, w, 1.0), 0.0)
            g = su._scale_axis(g, 1 + pos, w)
        return g


def test_planted_environment_slip_passes_the_exactness_pin(monkeypatch):
    """Without the environment weights (and without their restore) every untruncated
    contraction is still exact: the exactness pin cannot see this slip."""
    dem = rotated_phenomenological(3, 2, 0.05, 0.04)
    det, _ = sample_shots(dem, 4, seed=8)
    tm = exact.transfer_matrix(dem, det)
    monkeypatch.setattr(su, "PEPS", PEPSNoEnv)
    np.testing.assert_allclose(su.su_logprob(dem, det, chi=256, chi_mps=1024), tm, atol=1e-10)


@pytest.mark.parametrize("slip", [PEPSNoEnv, PEPSSquaredEnv])
def test_planted_environment_slip_is_caught(slip):
    peps, bond, psi = simple_update_case(1, chi=1, peps_cls=slip)
    best, _ = rank_truncate(psi.reshape(4, 4), 1)
    assert np.abs(peps_state(peps) - best.reshape(-1)).max() > 1e-3 * np.abs(psi).max()


# ---------------------------------------------------------------- zip-up cut
class GridPlan:
    """Stand-in for the plan's geometry as boundary_mps reads it (nx, ny, sites)."""

    def __init__(self, nx, ny):
        self.nx, self.ny = nx, ny
        self.sites = [(x, y) for y in range(ny) for x in range(nx)]


def orthonormal_rows(rng, r, c):
    q, _ = np.linalg.qr(rng.standard_normal((c, r)))
    return q.T


def zipup_case(seed, L=2, U0=4, U1=3):
    """A 2 x 2 final network (site tensors F[c][l][r][d][u]) whose right column in row 0
    is an isometry from (l, class parity in) to (u, class parity out)."""
    rng = np.random.default_rng(seed)
    F00 = rng.uniform(-1, 1, size=(2, 1, L, 1, U0))
    A, B = orthonormal_rows(rng, L, U1), orthonormal_rows(rng, L, U1)
    F10 = np.zeros((2, L, 1, 1, U1))
    F10[0, :, 0, 0, :] = (A + B) / 2
    F10[1, :, 0, 0, :] = (A - B) / 2
    Lt = 3
    F01 = rng.uniform(-1, 1, size=(2, 1, Lt, U0, 1))
    F11 = rng.uniform(-1, 1, size=(2, Lt, 1, U1, 1))
    return [F00, F10, F01, F11]


def row_state(Fa, Fb):
    """Row of two sites joined by their horizontal bond: R[ua, ub, c] with c the parity of
    the two class bits (the network's definition, no truncation)."""
    R = np.zeros((Fa.shape[4], Fb.shape[4], 2))
    for ca in range(2):
        for cb in range(2):
            R[:, :, ca ^ cb] += np.einsum("lu,lv->uv", Fa[ca, 0, :, 0, :], Fb[cb, :, 0, 0, :])
    return R


def top_row_state(Fa, Fb):
    """Top row (no up legs) as T[da, db, c]."""
    T = np.zeros((Fa.shape[3], Fb.shape[3], 2))
    for ca in range(2):
        for cb in range(2):
            T[:, :, ca ^ cb] += np.einsum("ld,le->de", Fa[ca, 0, :, :, 0], Fb[cb, :, 0, :, 0])
    return T


def zipup_reference(F, chi_mps):
    """Z[c] with the row-0 state cut to its optimal rank-chi_mps truncation across the
    vertical bond of column 0."""
    R0 = row_state(F[0], F[1])                              # [u0, u1, c0]
    U0, U1 = R0.shape[:2]
    R0t, s = rank_truncate(R0.reshape(U0, U1 * 2), chi_mps)
    R0t = R0t.reshape(U0, U1, 2)
    T1 = top_row_state(F[2], F[3])                          # [u0, u1, c1]
    Z = np.zeros(2)
    for c0 in range(2):
        for c1 in range(2):
            Z[c0 ^ c1] += np.einsum("ab,ab->", R0t[:, :, c0], T1[:, :, c1])
    return Z, s


@pytest.mark.parametrize("seed,chi_mps", [(1, 1), (2, 2), (3, 3), (4, 2)])
def test_zipup_cut_is_optimal_truncation_with_isometric_right_part(seed, chi_mps):
    F = zipup_case(seed)
    ref, s = zipup_reference(F, chi_mps)
    assert s[chi_mps] > 1e-3 * s[0]                        # the cut really truncates
    v, ls = su.boundary_mps(GridPlan(2, 2), F, chi_mps, 1e-12, 1e-8)
    np.testing.assert_allclose(v * np.exp(ls), ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


def test_zipup_untruncated_is_exact():
    F = zipup_case(5)
    ref, _ = zipup_reference(F, 8)
    v, ls = su.boundary_mps(GridPlan(2, 2), F, 8, 1e-12, 1e-8)
    np.testing.assert_allclose(v * np.exp(ls), ref, rtol=1e-12)


def test_planted_zipup_slip_is_caught(monkeypatch):
    """Planted slip: one vector too few kept at a truncating cut (an off-by-one in the
    kept count).  Untruncated contractions are unaffected, so the exactness and
    convergence pins still hold; the optimal-truncation pin fails."""
    good = su.keep_count

    def short(s, chi, cutoff, mrtol):
        k = good(s, chi, cutoff, mrtol)
        r = int(np.count_nonzero(s > cutoff * s[0]))
        return k - 1 if 1 < k < r else k

    monkeypatch.setattr(su, "keep_count", short)
    dem = point_sector_3d(3, 0.05)
    det, _ = sample_shots(dem, 4, seed=3)
    np.testing.assert_allclose(su.su_logprob(dem, det, chi=256, chi_mps=1024), exact.transfer_matrix(dem, det),
                               atol=1e-10)
    F = zipup_case(2)
    ref, _ = zipup_reference(F, 2)
    v, ls = su.boundary_mps(GridPlan(2, 2), F, 2, 1e-12, 1e-8)
    assert np.abs(v * np.exp(ls) - ref).max() > 1e-3 * np.abs(ref).max()


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_discarded_fraction_is_the_relative_truncation_error(seed):
    """With the environment exact, the weight the truncating gate reports as discarded equals
    the relative squared error of the optimal truncation of the dense state across that bond
    (Eckart-Young: the dropped singular values squared over all of them squared); the exact
    gates discard nothing."""
    peps, bond, psi = simple_update_case(seed, chi=1)
    best, s = rank_truncate(psi.reshape(4, 4), 1)
    want = np.sum((psi.reshape(4, 4) - best) ** 2) / np.sum(psi ** 2)
    assert want > 1e-8
    assert peps.trunc[:2] == [0.0, 0.0] or max(peps.trunc[:2]) < 1e-28
    np.testing.assert_allclose(peps.trunc[2], want, rtol=1e-10)
    np.testing.assert_allclose(su.discarded_fraction(s, 1), want, rtol=1e-10)

"""Pins of the generator-picture oracle (oracle/gen.py; Sec. 3.2, loop sector of Sec. 5.2).

The generator-picture sweep is checked against quantities fixed by the definition of the
coset probabilities, not by itself: the detector-picture brute force over all errors
(Sec. 2.4), the trivial-error enumeration of oracle/exact.py, closed forms at p = 1/2, the
normalisation over syndromes, the definition of the representative, the optimal truncation
of a chain whose environment is exact, and planted slips that these catch.
"""
import numpy as np
import pytest

from oracle import exact, gen, gf2
from oracle.su import PEPS
from td_inputs import GenProblem, loop_sector_3d, sample_shots


def _all_syndromes(gp):
    """Every error pattern of a tiny problem, its syndrome (distinct rows) and class."""
    n = gp.n_qubits
    H = gp.face_dem.H_dense().astype(np.int64)
    xs = ((np.arange(1 << n)[:, None] >> np.arange(n)[None, :]) & 1).astype(np.int64)
    syn = (xs @ H.T) % 2
    return np.unique(syn.astype(np.uint8), axis=0)


@pytest.mark.parametrize("d", [2, 3, 4])
def test_loop_sector_algebra(d):
    gp = loop_sector_3d(d, 0.1)
    H = gp.face_dem.H_dense().astype(np.int64)
    G = gen.generator_matrix(gp).astype(np.int64)
    assert ((G @ H.T) % 2).max() == 0                      # generators commute with the checks
    xb = np.zeros(gp.n_qubits, np.int64); xb[gp.xbar] = 1
    zb = np.zeros(gp.n_qubits, np.int64); zb[gp.zbar] = 1
    assert ((H @ xb) % 2).max() == 0 and ((G @ zb) % 2).max() == 0
    assert int(xb @ zb) % 2 == 1
    rX, rZ = gf2.rank(G), gf2.rank(H)
    assert gp.n_qubits - rX - rZ == 1                      # one logical qubit
    assert rX == gp.n_gen                                  # independent vertex generators
    assert gf2.rank(np.vstack([G, xb])) == rX + 1          # xbar is not a stabilizer


def test_generator_sum_equals_detector_picture_brute_force():
    gp = loop_sector_3d(2, 0.13)
    syn = _all_syndromes(gp)
    table = exact.brute_force_table(gp.face_dem)
    idx = exact.det_index(syn)
    with np.errstate(divide="ignore"):
        ref = np.log(table[idx])
    got = gen.enumerate_coset_logprob(gp, syn)
    assert np.allclose(got, ref, rtol=0, atol=1e-12)


def test_generator_sum_equals_trivial_error_enumeration():
    gp = loop_sector_3d(3, 0.17)
    det, _ = sample_shots(gp.face_dem, 6, seed=21)
    assert np.allclose(gen.enumerate_coset_logprob(gp, det), exact.generator_sum(gp.face_dem, det), atol=1e-11)


@pytest.mark.parametrize("d,p,n", [(2, 0.1, None), (3, 0.2, 12)])
def test_sweep_is_exact_without_truncation(d, p, n):
    gp = loop_sector_3d(d, p)
    syn = _all_syndromes(gp) if n is None else sample_shots(gp.face_dem, n, seed=3)[0]
    ref = gen.enumerate_coset_logprob(gp, syn)
    got = gen.gen_su_logprob(gp, syn, chi=64, chi_mps=256)
    assert np.allclose(got, ref, rtol=0, atol=1e-10)


def test_half_rate_closed_form():
    # at p = 1/2 every error has weight 2^-n and a coset holds 2^rank(generators) errors
    gp = loop_sector_3d(3, 0.5)
    det, _ = sample_shots(gp.face_dem, 4, seed=8)
    got = gen.gen_su_logprob(gp, det, chi=32, chi_mps=64)
    want = (gp.n_gen - gp.n_qubits) * np.log(2.0)
    assert np.allclose(got, want, atol=1e-10)


def test_probabilities_sum_to_one_over_syndromes():
    gp = loop_sector_3d(2, 0.21)
    syn = _all_syndromes(gp)
    got = gen.gen_su_logprob(gp, syn, chi=16, chi_mps=32)
    assert abs(np.exp(got).sum() - 1.0) < 1e-12


def test_representative_is_the_greedy_basis_solution():
    gp = loop_sector_3d(3, 0.1)
    H = gp.face_dem.H_dense()
    # greedy column basis by its definition: keep a column when it raises the rank
    basis, rk = [], 0
    for c in range(H.shape[1]):
        r = gf2.rank(H[:, basis + [c]])
        if r > rk:
            basis.append(c)
            rk = r
    det, _ = sample_shots(gp.face_dem, 5, seed=2)
    for m in det:
        r = gen.representative(gp, m)
        assert np.array_equal((H.astype(np.int64) @ r) % 2, m)
        assert not r[[c for c in range(H.shape[1]) if c not in basis]].any()


def test_impossible_syndrome_has_zero_probability():
    gp = loop_sector_3d(3, 0.1)
    m = np.zeros((1, gp.face_dem.n_det), np.uint8)
    m[0, 0] = 1                                            # a single plaquette: not a boundary
    assert gen.representative(gp, m[0]) is None
    assert np.all(gen.gen_su_logprob(gp, m, chi=8, chi_mps=16) == -np.inf)
    assert np.all(gen.enumerate_coset_logprob(gp, m) == -np.inf)


def test_truncation_converges_in_chi():
    gp = loop_sector_3d(3, 0.18)
    det, _ = sample_shots(gp.face_dem, 6, seed=4)
    ref = gen.enumerate_coset_logprob(gp, det)
    errs = [np.abs(gen.gen_su_logprob(gp, det, chi=c, chi_mps=2 * c) - ref).max() for c in (1, 2, 8)]
    assert errs[0] > errs[1] > errs[2] and errs[2] < 1e-10


def _chain(p, n=4):
    """n generators in a row, one layer: an in-layer edge between neighbours, a dangling
    edge below and above each (no checks are needed by the sweep itself)."""
    edges = [(v,) for v in range(n)] + [(v, v + 1) for v in range(n - 1)] + [(v,) for v in range(n)]
    rng = np.random.default_rng(12)
    pp = rng.uniform(0.05, 0.45, len(edges)) if p is None else np.full(len(edges), p)
    xyt = np.array([(v, 0, 0) for v in range(n)], np.int32)
    return GenProblem(n, edges, pp, xyt, [], [], None, name="chain")


def _dense_chain_state(gp, r, plan):
    """psi(s_0..s_3) after layer 0 (below weights, in-layer weights), by definition."""
    n = gp.n_gen
    psi = np.zeros((2,) * n)
    for idx in np.ndindex(*psi.shape):
        w = 1.0
        for v in range(n):
            j = plan.below[0][v]
            w *= (1 - gp.p[j], gp.p[j])[r[j] ^ idx[v]]
        for j, e in enumerate(gp.edges):
            if len(e) == 2:
                w *= (1 - gp.p[j], gp.p[j])[r[j] ^ idx[e[0]] ^ idx[e[1]]]
        psi[idx] = w
    return psi


def _peps_state(peps, plan):
    """Contract the chain PEPS (Gamma-lambda form) to a dense vector."""
    G = [peps.G[s] for s in range(plan.S)]
    lam = [peps.lam[b] for b in range(len(plan.bonds))]
    # site s's bonds are ordered left, right: bond s-1 then bond s
    v = G[0] * lam[0][None, :]                       # (s0, b0)
    for s in range(1, plan.S):
        g = G[s]                                     # (s, b_{s-1}, b_s) or (s, b_{s-1})
        if s < plan.S - 1:
            g = g * lam[s][None, None, :]
        v = np.tensordot(v, g, axes=([-1], [1]))     # (..., s, b_s)
    return v


@pytest.mark.parametrize("chi", [1, 2, 3])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_simple_update_of_diagonal_gate_is_the_optimal_truncation(chi, seed):
    """Gates 01 and 23 are applied exactly, so the environment of bond 12 (the lambdas of
    bonds 01 and 23 of a canonical chain) is exact and the simple update of gate 12 at chi
    equals the rank-chi Eckart-Young truncation of the dense state across that cut."""
    gp = _chain(None)
    plan = gen.GenPlan(gp)
    rng = np.random.default_rng(seed)
    r = rng.integers(0, 2, gp.n_qubits).astype(np.uint8)
    peps = PEPS(plan)
    for s in range(plan.S):
        j = plan.below[0][s]
        w = (1 - gp.p[j], gp.p[j])
        peps.apply_local(s, np.array([[w[r[j] ^ a ^ b] for a in range(2)] for b in range(2)]))
    for bond, j in plan.gates[0]:
        c = chi if plan.bonds[bond] == (1, 2) else 16
        gen._diag_gate(peps, bond, gp.p[j], int(r[j]), c, 1e-14, 1e-12)
    got = _peps_state(peps, plan) * np.exp(peps.logscale)
    psi = _dense_chain_state(gp, r, plan)
    U, sv, Vt = np.linalg.svd(psi.reshape(4, 4))
    want = ((U[:, :chi] * sv[:chi]) @ Vt[:chi]).reshape(psi.shape)
    # gauge: the stored state is the truncation up to one positive factor
    scale = (got * want).sum() / (got * got).sum()
    assert abs(scale - 1.0) < 1e-10     # the log-scale carries every normalisation
    assert np.allclose(got * scale, want, rtol=0, atol=1e-12 * np.abs(want).max())
    if chi == 1:   # the cut has rank 2 (the diagonal gate's rank): chi = 1 truncates
        assert np.abs(want - psi).max() > 1e-6


def test_planted_slips_are_caught(monkeypatch):
    gp = loop_sector_3d(3, 0.17)
    det, _ = sample_shots(gp.face_dem, 4, seed=9)
    ref = gen.enumerate_coset_logprob(gp, det)
    good = gen.gen_su_logprob(gp, det, chi=16, chi_mps=32)
    assert np.allclose(good, ref, atol=1e-10)
    orig = gen._diag_gate
    # slip 1: the gate ignores the representative's bit of its qubit
    monkeypatch.setattr(gen, "_diag_gate", lambda peps, bond, p, r, *a: orig(peps, bond, p, 0, *a))
    assert np.abs(gen.gen_su_logprob(gp, det, chi=16, chi_mps=32) - ref).max() > 1e-3
    # slip 2: the gate's weights swapped (w(0) = p)
    monkeypatch.setattr(gen, "_diag_gate", lambda peps, bond, p, r, *a: orig(peps, bond, 1 - p, r, *a))
    assert np.abs(gen.gen_su_logprob(gp, det, chi=16, chi_mps=32) - ref).max() > 1e-3
    monkeypatch.setattr(gen, "_diag_gate", orig)
    # slip 3: the other class taken without flipping xbar's bits
    monkeypatch.setattr(gp, "xbar", [])
    assert np.abs(gen.gen_su_logprob(gp, det, chi=16, chi_mps=32) - ref).max() > 1e-3

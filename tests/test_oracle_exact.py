"""Pins of the exact oracle methods against facts fixed by the paper and by mathematics.

Each test names what pins what.  A plausible slip in one method (a dropped mechanism, a
wrong flip, a transposed class) breaks agreement with an independent method, a closed
form or an invariant below.
"""
import numpy as np
import pytest

from td_inputs import (point_sector_3d, rotated_phenomenological, repetition_phenomenological,
                       five_qubit_code, sample_shots)
from oracle import exact, gf2, pauli


TINY = [
    lambda: point_sector_3d(2, 0.1),
    lambda: repetition_phenomenological(4, 2, 0.08, 0.05),
    lambda: rotated_phenomenological(3, 1, 0.06, 0.04),
]


@pytest.mark.parametrize("make", TINY)
def test_three_exact_methods_agree(make):
    """Brute force (Sec. 2.4 definition) = generator-picture coset sum (Sec. 3.2) =
    untruncated layer sweep, on every class of sampled shots."""
    dem = make()
    det, _ = sample_shots(dem, 12, seed=101)
    table = exact.brute_force_table(dem)
    with np.errstate(divide="ignore"):
        bf = np.log(table[exact.det_index(det)])
    gs = exact.generator_sum(dem, det)
    tm = exact.transfer_matrix(dem, det)
    np.testing.assert_allclose(gs, bf, rtol=0, atol=1e-11)
    np.testing.assert_allclose(tm, bf, rtol=0, atol=1e-11)


@pytest.mark.parametrize("make", TINY[:2])
def test_transfer_matrix_normalised_over_all_syndromes(make):
    """sum_m sum_L p_{m,L} = 1: the sweep summed over every detector outcome."""
    dem = make()
    n = dem.n_det
    allm = ((np.arange(1 << n)[:, None] >> np.arange(n)[None, :]) & 1).astype(np.uint8)
    lp = exact.transfer_matrix(dem, allm)
    assert abs(np.exp(lp).sum() - 1.0) < 1e-12


def test_brute_force_distribution():
    """The brute-force table is a probability distribution and its class marginal for a
    single mechanism on the observable is that mechanism's rate."""
    dem = point_sector_3d(2, 0.13)
    table = exact.brute_force_table(dem)
    assert abs(table.sum() - 1) < 1e-13
    assert (table >= 0).all()


@pytest.mark.parametrize("make,rank_expected", [
    (lambda p: point_sector_3d(3, p), 18),
    (lambda p: rotated_phenomenological(3, 2, p, p), 12),
])
def test_half_rate_closed_form(make, rank_expected):
    """At p = 1/2 every pattern has probability 2^-n, so p_{m,L} = 2^-(rank H + 1) for
    every consistent m and both L (l is independent of the rows of H)."""
    dem = make(0.5)
    H, L = dem.H_dense(), dem.L_dense()
    assert gf2.rank(H) == rank_expected
    assert gf2.rank(np.concatenate([H, L])) == rank_expected + 1
    det, _ = sample_shots(dem, 10, seed=5)
    tm = exact.transfer_matrix(dem, det)
    np.testing.assert_allclose(tm, -(rank_expected + 1) * np.log(2), atol=1e-12)


def test_point_sector_low_rate_asymptotics():
    """For m = 0 and p -> 0 the cheapest logical errors join the two rough boundaries:
    the d^2 straight z columns (weight d) and the 4d(d-1)^2 paths with one in-plane step
    (weight d+1: d-1 layers for the step times 4d(d-1) ordered neighbour pairs).  With
    r = p/(1-p): p_{0,1}/p_{0,0} = d^2 r^d (1 + 4(d-1)^2/d * r + O(r^2)); the trivial class
    only gains weight-4 loops, O(r^4)."""
    for d, p in ((3, 1e-4), (4, 1e-4)):
        dem = point_sector_3d(d, p)
        lp = exact.transfer_matrix(dem, np.zeros((1, dem.n_det), dtype=np.uint8))[0]
        ratio = np.exp(lp[1] - lp[0])
        r = p / (1 - p)
        expect = d * d * r ** d * (1 + 4 * (d - 1) ** 2 / d * r)
        assert abs(ratio / expect - 1) < 2e-6


def test_point_sector_counts():
    """Sec. 5.1 figure for d = 3: 51 qubit (=) nodes and 18 check (+) nodes on 3x3x2;
    general n = d^3 + 2d(d-1)^2, d^2(d-1) checks."""
    for d in (3, 4, 5):
        dem = point_sector_3d(d)
        assert dem.n_mech == d ** 3 + 2 * d * (d - 1) ** 2
        assert dem.n_det == d * d * (d - 1)
        assert dem.dims == (d, d, d - 1)
    assert point_sector_3d(3).n_mech == 51


def test_rotated_layout_counts():
    """Rotated d=9 Z checks: 40 checks on an 8 x 9 (u, v) grid; neighbours share a qubit;
    10 layers of 81 data mechanisms plus 9 x 40 measurement mechanisms."""
    dem = rotated_phenomenological(9, 9)
    nx, ny, nt = dem.dims
    assert (nx, ny, nt) == (8, 9, 10)
    assert dem.n_det == 400
    assert dem.n_mech == 81 * 10 + 40 * 9
    # every two-detector in-layer mechanism joins grid neighbours
    xyt = dem.det_xyt
    for ds in dem.mech_dets:
        if len(ds) == 2 and xyt[ds[0], 2] == xyt[ds[1], 2]:
            a, b = xyt[ds[0]], xyt[ds[1]]
            assert abs(int(a[0]) - int(b[0])) + abs(int(a[1]) - int(b[1])) == 1
    H, L = dem.H_dense(), dem.L_dense()
    assert gf2.rank(np.concatenate([H, L])) == gf2.rank(H) + 1


def test_point_sector_symmetries():
    """x <-> y transposition maps the point-sector network to itself (same p_{m,L});
    reflecting the layers maps the bottom cut to the top cut, which differs from it by
    the sum of all rows of H, so p_{m',L} = p_{m, L xor parity(m)}."""
    d = 3
    dem = point_sector_3d(d, 0.07)
    det, _ = sample_shots(dem, 16, seed=9)
    base = exact.transfer_matrix(dem, det)
    m = det.reshape(-1, d - 1, d, d)                        # [B, t, y, x]
    tr = exact.transfer_matrix(dem, m.transpose(0, 1, 3, 2).reshape(len(det), -1).copy())
    np.testing.assert_allclose(tr, base, atol=1e-11)
    fl = exact.transfer_matrix(dem, m[:, ::-1].reshape(len(det), -1).copy())
    par = det.sum(axis=1) % 2
    expect = np.where(par[:, None] == 1, base[:, ::-1], base)
    np.testing.assert_allclose(fl, expect, atol=1e-11)


def test_five_qubit_code_weight_enumerator():
    """Sec. 2.3 decoder on the [[5,1,3]] code under depolarising noise (I: 1-p, X/Y/Z:
    p/3): the stabilizer group has 15 weight-4 elements, each nontrivial logical coset
    10 weight-3 and 6 weight-5 elements (Shor-Laflamme enumerators of the perfect code)."""
    stabs, (xb, zb) = five_qubit_code()
    p = 0.1
    T = pauli.coset_table(stabs, xb, zb, [(1 - p, p / 3, p / 3, p / 3)] * 5)
    assert abs(T.sum() - 1) < 1e-13
    np.testing.assert_allclose(T[0, 0, 0], (1 - p) ** 5 + 15 * (1 - p) * (p / 3) ** 4, rtol=1e-13)
    for a, b in ((0, 1), (1, 0), (1, 1)):
        np.testing.assert_allclose(T[0, a, b], 10 * (1 - p) ** 2 * (p / 3) ** 3 + 6 * (p / 3) ** 5,
                                   rtol=1e-12)


def test_css_bitflip_equals_dem():
    """Sec. 3.3: for a CSS code under bit flips only, the general coset table over Paulis
    equals the DEM definition with H = H_Z and l = the Z-logical support."""
    from td_inputs.codes import rotated_z_checks
    d = 3
    checks, _ = rotated_z_checks(d)
    dem = rotated_phenomenological(d, 0, 0.11, 0.0)        # one perfect round = code capacity
    n = d * d
    qidx = {(i, j): i * d + j for i in range(d) for j in range(d)}
    zst = []
    for _, qs in checks:
        s = ["I"] * n
        for q in qs:
            s[qidx[q]] = "Z"
        zst.append("".join(s))
    zbar = "".join("Z" if j == 0 else "I" for i in range(d) for j in range(d))
    xbar = "".join("X" if i == 0 else "I" for i in range(d) for j in range(d))
    p = 0.11
    T = pauli.coset_table(zst, xbar, zbar, [(1 - p, p, 0.0, 0.0)] * n)
    table = exact.brute_force_table(dem)
    # detector index of the DEM: detectors are the Z checks in the same order
    np.testing.assert_allclose(T[:, :, 0], table, atol=1e-15)
    assert np.all(T[:, :, 1] == 0)


def test_total_logprob_of_impossible_syndrome_is_minus_infinity():
    """P(m) = sum_L p_{m,L} = 0 gives log P = -inf (not NaN)."""
    from oracle import exact
    lp = np.array([[-np.inf, -np.inf], [np.log(0.25), np.log(0.5)], [-np.inf, np.log(0.1)]])
    out = exact.total_logprob(lp)
    assert np.isneginf(out[0]) and abs(out[1] - np.log(0.75)) < 1e-15 and abs(out[2] - np.log(0.1)) < 1e-15

"""Edge cases of the CUDA path against the oracle: impossible syndromes (probability 0),
the smallest and largest bond caps, empty batches of the gradient, all-zero syndromes."""
import numpy as np
import pytest

from td_inputs import point_sector_3d, rotated_phenomenological, sample_shots
from oracle import exact, su

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def td():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2310_10722_gb300 as td
    from paper_2310_10722_gb300 import build, _lib
    import os
    if not os.path.exists(_lib.LIB_PATH):
        build.build()
    return td


def _close(a, b):
    both = np.isneginf(a) & np.isneginf(b)
    return np.where(both, 0.0, np.abs(a - b)).max()


def test_impossible_syndromes_read_minus_infinity(td):
    """3D point sector d=3 with every mechanism at detector 0 switched off (rate 0): a shot
    with that detector set has P(m) = 0 and reads log p = -inf in both classes; the others
    match the exact values; the gradient (mean over all B) gets nothing from the impossible
    shots and stays finite."""
    import torch
    base = point_sector_3d(3, 0.05)
    p = base.p.copy()
    for j, dets in enumerate(base.mech_dets):
        if 0 in dets:
            p[j] = 0.0
    dem = base.with_rates(p)
    det, _ = sample_shots(dem, 16, seed=42)
    bad = det.copy()
    bad[:, 0] ^= 1
    det = np.concatenate([det, bad])
    ref = exact.transfer_matrix(dem, det)
    possible = ~np.isneginf(ref).all(axis=1)
    assert possible.sum() == 16 and not possible[16:].any()
    net = td.Network.from_dem(dem, chi=8, chi_mps=64)
    d = torch.from_numpy(det).cuda()
    out = net.coset_logprob(d).cpu().numpy()
    assert _close(out, ref) < 1e-9
    logP, g = net.grad_logprob(d)
    g = g.cpu().numpy()
    assert np.isfinite(g).all() and np.isneginf(logP.cpu().numpy()[16:]).all()
    gref = exact.grad_total_logprob(dem, det[possible]).sum(axis=0) / len(det)
    assert np.abs(g - gref).max() / max(1.0, np.abs(gref).max()) < 1e-9


@pytest.mark.parametrize("chi,chi_mps", [(1, 1), (1, 4), (2, 2)])
def test_smallest_bond_caps(td, chi, chi_mps):
    import torch
    dem = rotated_phenomenological(5, 4, 0.03, 0.03)
    det, _ = sample_shots(dem, 6, seed=43)
    net = td.Network.from_dem(dem, chi=chi, chi_mps=chi_mps)
    out = net.coset_logprob(torch.from_numpy(det).cuda()).cpu().numpy()
    assert _close(out, su.su_logprob(dem, det, chi=chi, chi_mps=chi_mps)) < 1e-6


def test_largest_bond_cap_is_exact(td):
    """chi = 32 (the largest supported) on rotated d=3 with 3 noisy rounds: untruncated."""
    import torch
    dem = rotated_phenomenological(3, 3, 0.05, 0.04)
    det, _ = sample_shots(dem, 16, seed=44)
    net = td.Network.from_dem(dem, chi=32, chi_mps=8)
    out = net.coset_logprob(torch.from_numpy(det).cuda()).cpu().numpy()
    assert _close(out, exact.transfer_matrix(dem, det)) < 1e-9


def test_all_zero_syndromes_and_empty_gradient(td):
    import torch
    dem = rotated_phenomenological(5, 4, 0.03, 0.03)
    det = np.zeros((4, dem.n_det), dtype=np.uint8)
    net = td.Network.from_dem(dem, chi=8, chi_mps=8)
    out = net.coset_logprob(torch.from_numpy(det).cuda()).cpu().numpy()
    assert np.all(out[:, 0] == out[0, 0]) and np.all(out[:, 1] == out[0, 1])   # identical shots, identical values
    assert out[0, 0] > out[0, 1]                                            # no error is the likely class
    assert _close(out, su.su_logprob(dem, det, chi=8, chi_mps=8)) < 1e-6
    logP, g = net.grad_logprob(torch.zeros((0, dem.n_det), dtype=torch.uint8, device="cuda"))
    assert logP.shape == (0,) and np.all(g.cpu().numpy() == 0.0)


@pytest.mark.parametrize("precision", [0, 1, 2])
@pytest.mark.parametrize("threads", [256, 512, 1024])
def test_repeated_decodes_are_bitwise_equal(td, precision, threads):
    """Every path is deterministic: two decodes of the same shots give the same bits (no
    atomics in a floating-point sum, no reads racing writes), for every block size of the
    final contraction.  3D point sector d = 5, p = 0.1, chi = 16, chi_mps = 8 (cuts of up to
    128 columns: QR-reduced, FP32-preconditioned on the mixed paths)."""
    import torch
    dem = point_sector_3d(5, 0.1)
    det, _ = sample_shots(dem, 96, seed=4005)
    d = torch.from_numpy(det).cuda()
    net = td.Network.from_dem(dem, chi=16, chi_mps=8, precision=precision)
    net.set_schedule(threads, 2048, False)
    a = net.coset_logprob(d).cpu().numpy()
    b = net.coset_logprob(d).cpu().numpy()
    net.check()
    np.testing.assert_array_equal(a, b)

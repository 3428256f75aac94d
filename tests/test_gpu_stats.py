"""Truncation statistics (td_coset_logprob_stats) against the oracle's (oracle/su.py,
su_truncation_stats): the largest and summed discarded fraction of the simple-update
truncations and of the zip-up cuts, per shot."""
import numpy as np
import pytest

from oracle import su
from td_inputs import point_sector_3d, rotated_phenomenological, sample_shots

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _stats(dem, det, chi, chi_mps, precision=0):
    import paper_2310_10722_gb300 as td
    net = td.Network.from_dem(dem, chi=chi, chi_mps=chi_mps, precision=precision)
    d = torch.from_numpy(det).cuda()
    lp, st = net.coset_logprob_stats(d)
    plain = net.coset_logprob(d)
    net.check()
    out = (lp.cpu().numpy(), st.cpu().numpy(), plain.cpu().numpy())
    net.close()
    return out


@pytest.mark.parametrize("chi,chi_mps", [(2, 2), (4, 4)])
def test_statistics_match_oracle_when_truncating(chi, chi_mps):
    dem = rotated_phenomenological(5, 3, 0.03, 0.03)
    det, _ = sample_shots(dem, 8, seed=17)
    lp, st, plain = _stats(dem, det, chi, chi_mps)
    assert np.array_equal(lp, plain)                      # the same decode, bit for bit
    ref = su.su_truncation_stats(dem, det, chi, chi_mps)
    assert (ref[:, 0] > 0).all() and (ref[:, 2] > 1e-8).any()      # both stages truncate
    assert np.all(st >= 0) and np.all(st[:, 0] <= st[:, 1] + 1e-300) and np.all(st[:, 2] <= st[:, 3] + 1e-300)
    np.testing.assert_allclose(st, ref, rtol=1e-4, atol=1e-12)


def test_statistics_vanish_without_truncation():
    dem = point_sector_3d(3, 0.05)
    det, _ = sample_shots(dem, 16, seed=3)
    lp, st, plain = _stats(dem, det, 32, 64, precision=2)
    assert np.array_equal(lp, plain)
    assert st.max() < 1e-12

"""Generator networks on the GPU (td_build_gen_network; Sec. 3.2, the loop sector of Sec. 5.2)
against the oracle: exact values without truncation, the same-chi generator-picture sweep
with truncation, impossible syndromes, decisions, and the calls that a generator network
refuses."""
import numpy as np
import pytest

from oracle import exact, gen
from td_inputs import loop_sector_3d, sample_shots

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _net(gp, **kw):
    from paper_2310_10722_gb300 import GenNetwork
    return GenNetwork.from_problem(gp, **kw)


def _run(net, syn):
    s = torch.from_numpy(np.ascontiguousarray(syn, dtype=np.uint8)).cuda()
    lp = net.coset_logprob(s).cpu().numpy()
    dec, mar = net.decode(s)
    net.check()
    return lp, dec.cpu().numpy(), mar.cpu().numpy()


def _close(a, b, tol):
    fin = np.isfinite(b)
    assert np.array_equal(np.isfinite(a), fin)
    return np.abs(a[fin] - b[fin]).max() if fin.any() else 0.0


@pytest.mark.parametrize("precision,tol", [(0, 1e-9), (2, 1e-6), (1, 1e-5)])
@pytest.mark.parametrize("d,p", [(2, 0.12), (3, 0.17)])
def test_large_bond_caps_match_oracle_and_exact(d, p, precision, tol):
    """Bond caps above the exact ranks: the sweep equals the oracle's at the same settings, and
    both equal the exact coset sums up to the SVD cutoff (singular values below 1e-12 of the
    largest are dropped by both; on a rare shot that moves a coset by ~1e-6)."""
    gp = loop_sector_3d(d, p)
    syn, _ = sample_shots(gp.face_dem, 64, seed=31 + d)
    ref = gen.gen_su_logprob(gp, syn, chi=16, chi_mps=64)
    assert _close(ref, exact.generator_sum(gp.face_dem, syn), 1e-5) < 1e-5
    net = _net(gp, chi=16, chi_mps=64, precision=precision)
    lp, dec, mar = _run(net, syn)
    assert _close(lp, ref, tol) < tol
    assert np.array_equal(dec, (lp[:, 1] > lp[:, 0]).astype(np.int32))


@pytest.mark.parametrize("precision,tol", [(0, 1e-6), (2, 1e-3), (1, 1e-3)])
@pytest.mark.parametrize("d,p,chi,chi_mps", [(4, 0.15, 4, 8), (4, 0.2, 8, 16), (5, 0.2, 4, 8)])
def test_truncated_matches_same_chi_oracle(d, p, chi, chi_mps, precision, tol):
    gp = loop_sector_3d(d, p)
    syn, _ = sample_shots(gp.face_dem, 12, seed=7 * d + chi)
    ref = gen.gen_su_logprob(gp, syn, chi=chi, chi_mps=chi_mps)
    net = _net(gp, chi=chi, chi_mps=chi_mps, precision=precision)
    lp, dec, mar = _run(net, syn)
    assert _close(lp, ref, tol) < tol
    sure = np.abs(ref[:, 1] - ref[:, 0]) > 10 * tol
    assert np.array_equal(dec[sure], (ref[sure, 1] > ref[sure, 0]).astype(np.int32))


def test_impossible_syndrome_and_ragged_chunks():
    gp = loop_sector_3d(3, 0.1)
    syn, _ = sample_shots(gp.face_dem, 9, seed=5)
    syn = syn.copy()
    syn[4] = 0
    syn[4, 0] = 1                       # one plaquette alone: no error has this syndrome
    ref = gen.gen_su_logprob(gp, syn, chi=16, chi_mps=64)
    net = _net(gp, chi=16, chi_mps=64, max_wave=4)   # chunks of 2 shots: 5 chunks, the last ragged
    lp, dec, mar = _run(net, syn)
    assert np.all(lp[4] == -np.inf)
    assert _close(lp, ref, 1e-9) < 1e-9
    assert net.info()["generator"] == 1


def test_empty_batch_and_refused_calls():
    from paper_2310_10722_gb300 import TDError
    gp = loop_sector_3d(2, 0.1)
    net = _net(gp, chi=8, chi_mps=16)
    empty = torch.zeros((0, gp.face_dem.n_det), dtype=torch.uint8, device="cuda")
    assert net.coset_logprob(empty).shape == (0, 2)
    syn = torch.zeros((2, gp.face_dem.n_det), dtype=torch.uint8, device="cuda")
    from paper_2310_10722_gb300 import Network
    with pytest.raises(TDError):
        Network.coset_logprob(net, syn)        # the detector-network entry point
    with pytest.raises(TDError):
        net.grad_logprob(syn)


def test_full_size_loop_sector_sampled_shots():
    """d = 7, p = 0.15, chi = 8 on 256 shots (one launch sequence), sampled shots against the
    oracle.  A coset whose truncated weight is not positive reads -inf on both sides (near
    the loop-sector threshold, chi = 8 is too small for some shots)."""
    gp = loop_sector_3d(7, 0.15)
    syn, _ = sample_shots(gp.face_dem, 256, seed=77)
    net = _net(gp, chi=8, chi_mps=16, precision=2)
    lp, dec, mar = _run(net, syn)
    assert np.isfinite(lp).mean() > 0.8
    pick = [0, 1, 100, 255]
    ref = gen.gen_su_logprob(gp, syn[pick], chi=8, chi_mps=16)
    assert _close(lp[pick], ref, 1e-3) < 1e-3

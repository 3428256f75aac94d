"""Parity of td_grad_logprob (reverse sweep) and td_grad_logprob_forced (affine identity)
through the C ABI with the CPU FP64 oracle.

Untruncated networks: both equal the exact gradient d log P / d p_j (oracle/exact.py,
pinned against posterior marginals and central differences).  Truncated networks: the
reverse sweep is the derivative of the decoder's own log P, compared with central
differences of the oracle's same-chi sweep (oracle/su.py); the forced-rate gradient is
compared with the oracle's forced-rate gradient of its sweep.  Gradients are means over
shots; tolerances are absolute in d mean log P / d p_j relative to the largest entry.
"""
import numpy as np
import pytest

from td_inputs import point_sector_3d, rotated_phenomenological, repetition_phenomenological, sample_shots
from td_inputs import log_uniform_rates
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


def _grad(td, dem, det, p=None, method="reverse", **kw):
    import torch
    net = td.Network.from_dem(dem, **kw)
    d = torch.from_numpy(det).cuda()
    pp = None if p is None else torch.from_numpy(np.asarray(p, dtype=np.float64)).cuda()
    logP, g = net.grad_logprob(d, pp, method=method)
    torch.cuda.synchronize()
    return logP.cpu().numpy(), g.cpu().numpy(), net


def _rel(a, b):
    return np.abs(a - b).max() / max(1.0, np.abs(b).max())


@pytest.mark.parametrize("method", ["reverse", "forced"])
def test_grad_untruncated_rotated_log_uniform_rates(td, method):
    """Rotated d=3, 2 noisy rounds + 1 perfect, per-mechanism rates log-uniform in
    [1e-3, 1e-2] (the differentiation workload's recipe at a size the exact oracle takes)."""
    dem = log_uniform_rates(rotated_phenomenological(3, 2, 0.05, 0.04), seed=21)
    det, _ = sample_shots(dem, 16, seed=22)
    logP, g, _ = _grad(td, dem, det, method=method, chi=16, chi_mps=32)
    ref = exact.grad_total_logprob(dem, det).mean(axis=0)
    lt = exact.total_logprob(exact.transfer_matrix(dem, det))
    assert np.abs(logP - lt).max() < 1e-9
    assert _rel(g, ref) < 1e-9, _rel(g, ref)


@pytest.mark.parametrize("method", ["reverse", "forced"])
def test_grad_untruncated_repetition_merged_duplicates(td, method):
    """Repetition code with every mechanism listed twice (merged by the plan): each copy
    gets its own derivative through the merged rate."""
    base = repetition_phenomenological(5, 3, 0.07, 0.03)
    from td_inputs.codes import DEM
    dem = DEM(base.n_det, base.n_obs, list(base.mech_dets) * 2, list(base.mech_obs) * 2,
              np.concatenate([base.p, 0.5 * base.p]), base.det_xyt.copy(), "rep-dup", {})
    det, _ = sample_shots(base, 12, seed=23)
    logP, g, _ = _grad(td, dem, det, method=method, chi=32, chi_mps=8)
    ref = exact.grad_total_logprob(dem, det).mean(axis=0)
    assert _rel(g, ref) < 1e-9, _rel(g, ref)


def test_grad_untruncated_point_sector_reverse(td):
    """3D point sector d=3 (no counters, offset by the parity of all detectors)."""
    dem = point_sector_3d(3, 0.05)
    det, _ = sample_shots(dem, 16, seed=29)
    logP, g, _ = _grad(td, dem, det, chi=8, chi_mps=64)
    assert _rel(g, exact.grad_total_logprob(dem, det).mean(axis=0)) < 1e-9


def _fd_same_chi(dem, det, chi, chi_mps, js, rel_step=1e-5):
    """Central differences of the oracle's same-chi sweep (mean total log P) in rates js."""
    out = []
    for j in js:
        h = rel_step * dem.p[j]
        pp, pm = dem.p.copy(), dem.p.copy()
        pp[j] += h
        pm[j] -= h
        a = su.su_logprob(dem.with_rates(pp), det, chi, chi_mps)
        b = su.su_logprob(dem.with_rates(pm), det, chi, chi_mps)
        out.append((np.logaddexp(a[:, 0], a[:, 1]) - np.logaddexp(b[:, 0], b[:, 1])).mean() / (2 * h))
    return np.array(out)


@pytest.mark.parametrize("case", ["point_d3_chi2", "point_d4_chi4", "rotated_d3_3rounds_chi2"])
def test_grad_reverse_truncated_matches_oracle_differences(td, case):
    """Truncated: the reverse sweep is the derivative of the decoder's log P; the oracle's
    same-chi sweep differenced in every sampled rate (step 1e-5 p_j) agrees to 1e-6."""
    dem, chi, cm = {"point_d3_chi2": (point_sector_3d(3, 0.08), 2, 8),
                    "point_d4_chi4": (point_sector_3d(4, 0.06), 4, 8),
                    "rotated_d3_3rounds_chi2": (log_uniform_rates(rotated_phenomenological(3, 3, 0.05, 0.04), seed=3),
                                                2, 4)}[case]
    det, _ = sample_shots(dem, 2, seed=17)
    logP, g, _ = _grad(td, dem, det, chi=chi, chi_mps=cm)
    js = np.arange(0, dem.n_mech, max(1, dem.n_mech // 16))
    fd = _fd_same_chi(dem, det, chi, cm, js)
    assert np.abs(g[js] - fd).max() / max(1.0, np.abs(fd).max()) < 1e-6
    ref = su.su_logprob(dem, det, chi, cm)
    assert np.abs(logP - np.logaddexp(ref[:, 0], ref[:, 1])).max() < 1e-6


def test_grad_forced_truncated_matches_same_chi_oracle(td):
    """Point sector d=3 at chi=2 (truncated): the decoder's own forced-rate values."""
    dem = point_sector_3d(3, 0.08)
    det, _ = sample_shots(dem, 4, seed=24)
    logP, g, _ = _grad(td, dem, det, method="forced", chi=2, chi_mps=8)
    lp_ref, g_ref = su.su_grad_total_logprob(dem, det, chi=2, chi_mps=8)
    assert np.abs(logP - lp_ref).max() < 1e-6
    assert _rel(g, g_ref.mean(axis=0)) < 1e-6, _rel(g, g_ref.mean(axis=0))
    assert _rel(g, exact.grad_total_logprob(dem, det).mean(axis=0)) > 1e-3   # truncation is real here


def test_grad_rates_argument_and_autograd(td):
    """p_dev replaces the rates (same result as a network built at those rates, bit for
    bit) and mean_logprob's backward returns the same gradient."""
    import torch
    dem0 = rotated_phenomenological(3, 2, 0.05, 0.04)
    dem1 = log_uniform_rates(dem0, seed=25)
    det, _ = sample_shots(dem1, 8, seed=26)
    lp_a, g_a, net = _grad(td, dem0, det, p=dem1.p, chi=8, chi_mps=16)
    lp_b, g_b, _ = _grad(td, dem1, det, chi=8, chi_mps=16)
    assert np.array_equal(lp_a, lp_b) and np.array_equal(g_a, g_b)
    p = torch.from_numpy(dem1.p.copy()).cuda().requires_grad_(True)
    d = torch.from_numpy(det).cuda()
    f = td.mean_logprob(net, d, p)
    f.backward()
    assert abs(f.item() - lp_b.mean()) < 1e-12
    assert np.array_equal(p.grad.cpu().numpy(), g_b)


def test_grad_waves_and_fp32_network(td):
    """Several waves give the same gradient as one; an FP32-storage network runs the
    reverse sweep in FP64 (same result); its forced-rate gradient is within 1e-3."""
    dem = log_uniform_rates(rotated_phenomenological(3, 2, 0.05, 0.04), seed=27)
    det, _ = sample_shots(dem, 16, seed=28)
    lp1, g1, _ = _grad(td, dem, det, chi=8, chi_mps=16, max_wave=5)
    lp2, g2, _ = _grad(td, dem, det, chi=8, chi_mps=16)
    assert np.abs(lp1 - lp2).max() < 1e-12 and _rel(g1, g2) < 1e-12
    _, g32, _ = _grad(td, dem, det, chi=8, chi_mps=16, precision=td.TD_FP32)
    assert _rel(g32, g2) < 1e-12
    _, f64, _ = _grad(td, dem, det, method="forced", chi=8, chi_mps=16, precision=td.TD_FP64)
    _, f32, _ = _grad(td, dem, det, method="forced", chi=8, chi_mps=16, precision=td.TD_FP32)
    assert _rel(f32, f64) < 1e-3, _rel(f32, f64)


def test_grad_full_size_sampled(td):
    """The differentiation workload's network (rotated d=7, 7+1 rounds, 560 log-uniform
    rates) at chi = chi_mps = 8, the launch configuration bench.py times: the reverse sweep of
    single shots against the oracle's reverse sweep of the same shots."""
    from oracle import reverse
    dem = log_uniform_rates(rotated_phenomenological(7, 7, 0.005, 0.005), seed=5000)
    det, _ = sample_shots(dem, 2, seed=5001)
    jac = reverse.object_jacobian(dem)
    for b in range(2):
        logP, g, _ = _grad(td, dem, det[b:b + 1], chi=8, chi_mps=8)
        lp_ref, g_ref = reverse.reverse_grad_total_logprob(dem, det[b:b + 1], 8, 8, jac=jac)
        assert abs(logP[0] - lp_ref[0]) < 1e-6
        assert _rel(g, g_ref[0]) < 1e-5, _rel(g, g_ref[0])


def test_grad_largest_bond_cap_exact(td):
    """chi = 32 (the largest supported, untruncated here): the exact gradient."""
    dem = log_uniform_rates(rotated_phenomenological(3, 3, 0.05, 0.04), seed=33)
    det, _ = sample_shots(dem, 8, seed=34)
    logP, g, _ = _grad(td, dem, det, chi=32, chi_mps=8)
    assert _rel(g, exact.grad_total_logprob(dem, det).mean(axis=0)) < 1e-9


def test_grad_chi16_truncated_matches_oracle_differences(td):
    """chi = 16 with truncation (rotated d=5, 3 noisy rounds): central differences of the
    oracle's same-chi sweep in sampled rates."""
    dem = rotated_phenomenological(5, 3, 0.06, 0.05)
    det, _ = sample_shots(dem, 2, seed=35)
    logP, g, _ = _grad(td, dem, det, chi=16, chi_mps=16)
    js = np.arange(0, dem.n_mech, max(1, dem.n_mech // 10))
    fd = _fd_same_chi(dem, det, 16, 16, js)
    assert np.abs(g[js] - fd).max() / max(1.0, np.abs(fd).max()) < 1e-6


@pytest.mark.parametrize("stride", [1, 2, 3])
def test_checkpointed_reverse_sweep_equals_full_record(td, stride):
    """Checkpoints every `stride` layers (the segments recomputed from them before their
    reverse sweep) give the gradient of the full record, bit for bit: the recomputation
    repeats the same kernels on the same inputs.  Rotated d = 5, 4 noisy rounds + 1 perfect
    (5 layers), chi = 4 (truncating), log-uniform rates."""
    dem = log_uniform_rates(rotated_phenomenological(5, 4, 0.02, 0.02), seed=31)
    det, _ = sample_shots(dem, 12, seed=32)
    lp0, g0, _ = _grad(td, dem, det, chi=4, chi_mps=8)
    lpk, gk, net = _grad(td, dem, det, chi=4, chi_mps=8, ckpt_stride=stride)
    np.testing.assert_array_equal(lpk, lp0)
    np.testing.assert_array_equal(gk, g0)
    net.check()

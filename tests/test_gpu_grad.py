"""Parity of td_grad_logprob (through the C ABI) with the CPU FP64 oracle.

Untruncated networks: the exact gradient d log P / d p_j (oracle/exact.py, pinned against
posterior marginals and central differences).  Truncated networks: the oracle's gradient
of its own same-chi sweep by the affine identity (oracle/su.py).  Gradients are means over
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


def _grad(td, dem, det, p=None, **kw):
    import torch
    net = td.Network.from_dem(dem, **kw)
    d = torch.from_numpy(det).cuda()
    pp = None if p is None else torch.from_numpy(np.asarray(p, dtype=np.float64)).cuda()
    logP, g = net.grad_logprob(d, pp)
    torch.cuda.synchronize()
    return logP.cpu().numpy(), g.cpu().numpy(), net


def _rel(a, b):
    return np.abs(a - b).max() / max(1.0, np.abs(b).max())


def test_grad_untruncated_rotated_log_uniform_rates(td):
    """Rotated d=3, 2 noisy rounds + 1 perfect, per-mechanism rates log-uniform in
    [1e-3, 1e-2] (the differentiation workload's recipe at a size the exact oracle takes)."""
    dem = log_uniform_rates(rotated_phenomenological(3, 2, 0.05, 0.04), seed=21)
    det, _ = sample_shots(dem, 16, seed=22)
    logP, g, _ = _grad(td, dem, det, chi=16, chi_mps=32)
    ref = exact.grad_total_logprob(dem, det).mean(axis=0)
    lt = exact.total_logprob(exact.transfer_matrix(dem, det))
    assert np.abs(logP - lt).max() < 1e-9
    assert _rel(g, ref) < 1e-9, _rel(g, ref)


def test_grad_untruncated_repetition_merged_duplicates(td):
    """Repetition code with every mechanism listed twice (merged by the plan): each copy
    gets its own derivative through the merged rate."""
    base = repetition_phenomenological(5, 3, 0.07, 0.03)
    from td_inputs.codes import DEM
    dem = DEM(base.n_det, base.n_obs, list(base.mech_dets) * 2, list(base.mech_obs) * 2,
              np.concatenate([base.p, 0.5 * base.p]), base.det_xyt.copy(), "rep-dup", {})
    det, _ = sample_shots(base, 12, seed=23)
    logP, g, _ = _grad(td, dem, det, chi=32, chi_mps=8)
    ref = exact.grad_total_logprob(dem, det).mean(axis=0)
    assert _rel(g, ref) < 1e-9, _rel(g, ref)


def test_grad_truncated_matches_same_chi_oracle(td):
    """Point sector d=3 at chi=2 (truncated): the decoder's own forced-rate values."""
    dem = point_sector_3d(3, 0.08)
    det, _ = sample_shots(dem, 4, seed=24)
    logP, g, _ = _grad(td, dem, det, chi=2, chi_mps=8)
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


def test_grad_fp32_storage_close_to_fp64(td):
    dem = log_uniform_rates(rotated_phenomenological(3, 2, 0.05, 0.04), seed=27)
    det, _ = sample_shots(dem, 16, seed=28)
    _, g64, _ = _grad(td, dem, det, chi=8, chi_mps=16, precision=td.TD_FP64)
    _, g32, _ = _grad(td, dem, det, chi=8, chi_mps=16, precision=td.TD_FP32)
    assert _rel(g32, g64) < 1e-3, _rel(g32, g64)

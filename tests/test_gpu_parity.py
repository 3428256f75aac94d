"""Parity of the CUDA path (through the C ABI) with the CPU FP64 oracle.

Exact cases (chi and chi_mps at least the untruncated bonds) compare with the exact
transfer matrix; truncated cases with the oracle's same-chi sweep.  FP64 tolerance 1e-6
in log p (target 1e-9 for the exact cases); FP32 path 1e-3.
"""
import numpy as np
import pytest

from td_inputs import point_sector_3d, rotated_phenomenological, repetition_phenomenological, sample_shots
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


def _run(td, dem, det, **kw):
    import torch
    net = td.Network.from_dem(dem, **kw)
    d = torch.from_numpy(det).cuda()
    out = net.coset_logprob(d).cpu().numpy()
    torch.cuda.synchronize()
    return out, net


def _close(a, b, tol):
    both_inf = np.isneginf(a) & np.isneginf(b)
    err = np.where(both_inf, 0.0, np.abs(a - b))
    return err.max(), err


def test_point_sector_d3_exact_all_512(td):
    """3D point sector d=3, p=0.05, 512 seeded shots, untruncated FP64 vs exact sweep."""
    dem = point_sector_3d(3, 0.05)
    det, _ = sample_shots(dem, 512, seed=1000)
    ref = exact.transfer_matrix(dem, det)
    out, net = _run(td, dem, det, chi=8, chi_mps=64)
    m, _ = _close(out, ref, 1e-9)
    assert m < 1e-9, m


def test_rotated_counters_exact(td):
    """Time sweep with class-counter sites (rotated d=3, 2 noisy rounds + 1 perfect)."""
    dem = rotated_phenomenological(3, 2, 0.05, 0.04)
    det, _ = sample_shots(dem, 64, seed=77)
    ref = exact.transfer_matrix(dem, det)
    out, net = _run(td, dem, det, chi=16, chi_mps=32)
    assert net.info()["n_counter_sites"] > 0
    m, _ = _close(out, ref, 1e-9)
    assert m < 1e-9, m


def test_repetition_exact(td):
    dem = repetition_phenomenological(6, 4, 0.06, 0.03)
    det, _ = sample_shots(dem, 50, seed=5)
    ref = exact.transfer_matrix(dem, det)
    out, _ = _run(td, dem, det, chi=32, chi_mps=8)
    m, _ = _close(out, ref, 1e-9)
    assert m < 1e-9, m


@pytest.mark.parametrize("chi,chi_mps", [(2, 8), (4, 16)])
def test_point_sector_d4_truncated_matches_same_chi_oracle(td, chi, chi_mps):
    dem = point_sector_3d(4, 0.08)
    det, _ = sample_shots(dem, 24, seed=6)
    ref = su.su_logprob(dem, det, chi=chi, chi_mps=chi_mps)
    out, _ = _run(td, dem, det, chi=chi, chi_mps=chi_mps)
    m, _ = _close(out, ref, 1e-6)
    assert m < 1e-6, m


def test_rotated_d5_truncated_matches_same_chi_oracle(td):
    dem = rotated_phenomenological(5, 4, 0.04, 0.04)
    det, _ = sample_shots(dem, 16, seed=8)
    ref = su.su_logprob(dem, det, chi=4, chi_mps=8)
    out, _ = _run(td, dem, det, chi=4, chi_mps=8)
    m, _ = _close(out, ref, 1e-6)
    assert m < 1e-6, m


def test_fp32_path_within_1e3(td):
    dem = rotated_phenomenological(5, 4, 0.04, 0.04)
    det, _ = sample_shots(dem, 16, seed=8)
    ref = su.su_logprob(dem, det, chi=4, chi_mps=8)
    out, _ = _run(td, dem, det, chi=4, chi_mps=8, precision=td.TD_FP32)
    m, _ = _close(out, ref, 1e-3)
    assert m < 1e-3, m


def test_decode_and_ragged_waves(td):
    """Decisions = argmax of the log-probabilities; waves of 7 shots over 20 shots give the
    same result as one wave; B = 0 is a no-op; the host-buffer entry point agrees."""
    import torch
    dem = rotated_phenomenological(3, 2, 0.05, 0.04)
    det, _ = sample_shots(dem, 20, seed=3)
    one, net1 = _run(td, dem, det, chi=16, chi_mps=32)
    many, net7 = _run(td, dem, det, chi=16, chi_mps=32, max_wave=7)
    assert net7.info()["wave"] == 7
    np.testing.assert_array_equal(one, many)
    dec, mar = net7.decode(torch.from_numpy(det).cuda())
    dec, mar = dec.cpu().numpy(), mar.cpu().numpy()
    np.testing.assert_array_equal(dec, (one[:, 1] > one[:, 0]).astype(np.int32))
    np.testing.assert_allclose(mar, np.abs(one[:, 1] - one[:, 0]), rtol=0, atol=1e-12)
    host = net7.coset_logprob_host(torch.from_numpy(det).pin_memory()).numpy()
    np.testing.assert_array_equal(host, one)
    empty = net1.coset_logprob(torch.zeros((0, dem.n_det), dtype=torch.uint8, device="cuda"))
    assert empty.shape == (0, 2)


def test_rotated_d9_full_size_sampled(td):
    """The benchmark workload (rotated d=9, 9 noisy + 1 perfect rounds, p=q=0.03) at chi=8
    on sampled shots of the seeded stream against the same-chi oracle."""
    dem = rotated_phenomenological(9, 9, 0.03, 0.03)
    det, _ = sample_shots(dem, 6, seed=2000)
    ref = su.su_logprob(dem, det, chi=8, chi_mps=8)
    out, _ = _run(td, dem, det, chi=8, chi_mps=8)
    m, _ = _close(out, ref, 1e-6)
    assert m < 1e-6, m


@pytest.mark.parametrize("case", ["rotated_d3", "point_d3", "repetition"])
def test_fp32_storage_exact_regime(td, case):
    """FP32 storage (FP64-accumulated Gram, FP32 update, FP64 truncation cores) where no
    truncation happens: the result is the exact contraction up to the rounding of the
    stored tensors, so it must match the exact transfer matrix to a few 1e-6 in log p."""
    if case == "rotated_d3":
        dem, B, seed, kw = rotated_phenomenological(3, 2, 0.05, 0.04), 64, 77, dict(chi=16, chi_mps=32)
    elif case == "point_d3":
        dem, B, seed, kw = point_sector_3d(3, 0.05), 64, 1000, dict(chi=8, chi_mps=64)
    else:
        dem, B, seed, kw = repetition_phenomenological(6, 4, 0.06, 0.03), 50, 5, dict(chi=32, chi_mps=8)
    det, _ = sample_shots(dem, B, seed=seed)
    ref = exact.transfer_matrix(dem, det)
    out, _ = _run(td, dem, det, precision=td.TD_FP32, **kw)
    m, _ = _close(out, ref, 5e-5)
    assert m < 5e-5, m


@pytest.mark.parametrize("precision,tol", [(0, 1e-6), (1, 1e-3)])
def test_point_sector_d5_truncated(td, precision, tol):
    """3D point sector d=5 (25 sites, 4 check layers) at p=0.1 with truncation, against the
    same-chi oracle: the code sizes of the uneven point-sector batch go through this path."""
    dem = point_sector_3d(5, 0.1)
    det, _ = sample_shots(dem, 6, seed=4)
    ref = su.su_logprob(dem, det, chi=8, chi_mps=8)
    out, _ = _run(td, dem, det, chi=8, chi_mps=8, precision=precision)
    m, _ = _close(out, ref, tol)
    assert m < tol, m


@pytest.mark.parametrize("precision,tol", [(0, 1e-6), (2, 1e-3)])
def test_paper_bond_caps_chi24_chimps32(td, precision, tol):
    """The bond caps of the paper's point-sector runs (chi_SU = 24, chi_MPS = 32, Sec. 5.1):
    3D point sector d = 4 (truncating at these caps: cuts of up to 32 x 24 = 768 columns in
    the final contraction) against the same-caps oracle."""
    dem = point_sector_3d(4, 0.08)
    det, _ = sample_shots(dem, 16, seed=41)
    ref = su.su_logprob(dem, det, chi=24, chi_mps=32)
    out, net = _run(td, dem, det, chi=24, chi_mps=32, precision=precision)
    net.check()
    m, _ = _close(out, ref, tol)
    assert m < tol, m

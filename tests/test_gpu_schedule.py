"""Launch schedule (td_network_set_schedule, td_network_tune): every candidate gives the
oracle's results; the autotuner picks a candidate and keeps the results."""
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


@pytest.mark.parametrize("threads", [256, 512, 1024])
@pytest.mark.parametrize("chunk", [512, 4096])
@pytest.mark.parametrize("smem", [True, False])
def test_every_schedule_matches_the_oracle(td, threads, chunk, smem):
    import torch
    dem = point_sector_3d(3, 0.05)
    det, _ = sample_shots(dem, 64, seed=1000)
    net = td.Network.from_dem(dem, chi=8, chi_mps=64)
    net.set_schedule(threads, chunk, smem)
    out = net.coset_logprob(torch.from_numpy(det).cuda()).cpu().numpy()
    assert np.abs(out - exact.transfer_matrix(dem, det)).max() < 1e-9
    dem5 = rotated_phenomenological(5, 4, 0.03, 0.03)
    det5, _ = sample_shots(dem5, 4, seed=7)
    net5 = td.Network.from_dem(dem5, chi=4, chi_mps=8)
    net5.set_schedule(threads, chunk, smem)
    out5 = net5.coset_logprob(torch.from_numpy(det5).cuda()).cpu().numpy()
    ref5 = su.su_logprob(dem5, det5, chi=4, chi_mps=8)
    assert np.abs(out5 - ref5).max() < 1e-6


def test_tune_picks_a_candidate_and_keeps_results(td):
    import torch
    dem = rotated_phenomenological(5, 4, 0.03, 0.03)
    det, _ = sample_shots(dem, 64, seed=8)
    d = torch.from_numpy(det).cuda()
    net = td.Network.from_dem(dem, chi=8, chi_mps=8, precision=td.TD_FP32)
    before = net.coset_logprob(d).cpu().numpy()
    sched = net.tune(d)
    assert sched["final_threads"] in (256, 512, 1024) and sched["chunk_rows"] in (512, 1024, 2048, 4096)
    assert sched["ms"] > 0
    after = net.coset_logprob(d).cpu().numpy()
    assert np.abs(after - before).max() < 1e-3
    with pytest.raises(Exception):
        net.set_schedule(384, 2048)


def test_gradient_after_a_schedule_change(td):
    """A gradient call, then a schedule with a larger final-contraction layout, then another
    gradient call: both equal the exact gradient (the reverse sweep's scratch follows)."""
    import torch
    dem = rotated_phenomenological(3, 2, 0.05, 0.04)
    det, _ = sample_shots(dem, 8, seed=9)
    d = torch.from_numpy(det).cuda()
    net = td.Network.from_dem(dem, chi=16, chi_mps=32)
    ref = exact.grad_total_logprob(dem, det).mean(axis=0)
    for sched in ((256, 4096, True), (1024, 512, False), (512, 1024, True)):
        net.set_schedule(sched[0], sched[1], sched[2])
        _, g = net.grad_logprob(d)
        g = g.cpu().numpy()
        assert np.abs(g - ref).max() / max(1.0, np.abs(ref).max()) < 1e-9

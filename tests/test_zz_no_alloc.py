"""The allocation-free decode entry point (td_coset_logprob_static) against td_coset_logprob.

td_coset_logprob_static serves callers that cannot call cudaMalloc/cudaFree around a
decode: the final contraction's scratch comes from a static device array in the library
instead of the network workspace.  Its results must equal the ordinary entry point's, on two
calls in a row (the array keeps the previous call's contents), and a batch beyond the
array's capacity must be refused before any work is enqueued.
"""
import ctypes as C

import numpy as np
import pytest

from td_inputs import point_sector_3d, rotated_phenomenological, sample_shots

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def td():
    import os
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2310_10722_gb300 as td
    from paper_2310_10722_gb300 import _lib, build
    if not os.path.exists(_lib.LIB_PATH):
        build.build()
    return td


def _static_call(net, det, out):
    import torch
    lib = net._lib
    st = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.td_coset_logprob_static(net._h, C.c_void_p(det.data_ptr()), det.shape[0], C.c_void_p(out.data_ptr()), st)


@pytest.mark.parametrize("make,kw,B", [
    (lambda: point_sector_3d(3, 0.05), dict(chi=8, chi_mps=64), 12),
    (lambda: rotated_phenomenological(3, 2, 0.05, 0.04), dict(chi=4, chi_mps=4), 80),
])
def test_static_scratch_matches_allocating_entry(td, make, kw, B):
    import torch
    dem = make()
    det_np, _ = sample_shots(dem, B, seed=424242)
    det = torch.from_numpy(det_np).cuda()
    net = td.Network.from_dem(dem, **kw)
    ref = net.coset_logprob(det).cpu().numpy()
    for call in range(2):
        out = torch.full((B, 2), float("nan"), dtype=torch.float64, device="cuda")
        assert _static_call(net, det, out) == 0, net._lib.td_last_error().decode()
        got = out.cpu().numpy()
        both = np.isneginf(got) & np.isneginf(ref)
        err = np.where(both, 0.0, np.abs(got - ref))
        assert err.max() < 1e-9, (call, err.max())


def test_static_scratch_rejects_oversized_batch(td):
    """A batch one shot beyond the capacity is refused with the capacity in the message and
    nothing written; a batch exactly at the capacity runs and matches the ordinary path."""
    import re
    import torch
    dem = point_sector_3d(3, 0.05)
    net = td.Network.from_dem(dem, chi=8, chi_mps=64, max_wave=32)
    big = 4096
    det_np, _ = sample_shots(dem, big, seed=99)
    det = torch.from_numpy(det_np).cuda()
    out = torch.zeros((big, 2), dtype=torch.float64, device="cuda")
    assert _static_call(net, det, out) == 1
    msg = net._lib.td_last_error().decode()
    m = re.search(r"exceeds the static scratch capacity of this network: (\d+) shots", msg)
    assert m, msg
    cap = int(m.group(1))
    assert 1 <= cap <= 32
    torch.cuda.synchronize()
    assert torch.count_nonzero(out).item() == 0
    over = det[:cap + 1].contiguous()
    assert _static_call(net, over, out[:cap + 1]) == 1
    fit = det[:cap].contiguous()
    assert _static_call(net, fit, out[:cap]) == 0, net._lib.td_last_error().decode()
    ref = net.coset_logprob(fit).cpu().numpy()
    np.testing.assert_allclose(out[:cap].cpu().numpy(), ref, rtol=0, atol=1e-9)

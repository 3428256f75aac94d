"""Host-side logic of the multi-GPU (replica) benchmark path on CPU with two gloo ranks:
each rank decodes its own contiguous slice of the seeded shot stream (no collective on the
data path), and the timed region is the slowest rank's (a MAX reduction)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    import sys
    import torch.distributed as dist
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from td_inputs import rotated_phenomenological, sample_shots
    dem = rotated_phenomenological(3, 2, 0.05, 0.04)
    first = bench.replica_first_shot(rank, 40)
    det, cls = sample_shots(dem, 40, seed=bench.SEED, first_shot=first)
    t = bench.max_over_ranks(1.5 + rank, world)       # per-rank "time"
    np.savez(os.path.join(out_dir, f"r{rank}.npz"), det=det, cls=cls, t=t, first=first)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_replicas_cover_the_stream_and_take_the_max(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.spawn(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    r0, r1 = np.load(tmp_path / "r0.npz"), np.load(tmp_path / "r1.npz")
    assert int(r0["first"]) == 0 and int(r1["first"]) == 40
    assert float(r0["t"]) == float(r1["t"]) == 2.5        # MAX over ranks, seen by both
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    from td_inputs import rotated_phenomenological, sample_shots
    dem = rotated_phenomenological(3, 2, 0.05, 0.04)
    whole, _ = sample_shots(dem, 80, seed=bench.SEED)
    np.testing.assert_array_equal(np.concatenate([r0["det"], r1["det"]]), whole)


def _grad_worker(rank, world, port, out_dir):
    import sys
    import torch.distributed as dist
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from oracle import exact
    from td_inputs import rotated_phenomenological, sample_shots, log_uniform_rates
    dem = log_uniform_rates(rotated_phenomenological(3, 2, 0.05, 0.04), seed=31)
    n = 6 + 3 * rank                                   # uneven slices
    first = 0 if rank == 0 else 6
    det, _ = sample_shots(dem, n, seed=32, first_shot=first)
    g = exact.grad_total_logprob(dem, det).mean(axis=0)
    m = bench.mean_over_ranks(g, n, world).numpy()
    np.save(os.path.join(out_dir, f"g{rank}.npy"), m)
    dist.barrier()
    dist.destroy_process_group()


def test_gradient_mean_over_two_gloo_ranks(tmp_path):
    """The per-rank gradient means combine into the mean over all shots (one all-reduce)."""
    import torch.multiprocessing as mp
    port = _free_port()
    mp.spawn(_grad_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    g0, g1 = np.load(tmp_path / "g0.npy"), np.load(tmp_path / "g1.npy")
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    from oracle import exact
    from td_inputs import rotated_phenomenological, sample_shots, log_uniform_rates
    dem = log_uniform_rates(rotated_phenomenological(3, 2, 0.05, 0.04), seed=31)
    det, _ = sample_shots(dem, 15, seed=32)
    whole = exact.grad_total_logprob(dem, det).mean(axis=0)
    np.testing.assert_allclose(g0, whole, rtol=1e-12, atol=1e-12)
    np.testing.assert_array_equal(g0, g1)

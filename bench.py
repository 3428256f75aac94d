#!/usr/bin/env python
"""Throughput of tensor-network coset decoding on one GB300 (arXiv 2310.10722, Sec. 4).

Workload: rotated surface code d=9 with phenomenological noise (data p=0.03, measurement
q=0.03), 9 noisy syndrome rounds + 1 perfect round (a 40-site x 10-layer detector network),
4096 seeded synthetic shots per GPU, simple-update bond chi (default 8), final MPS bond
chi_mps = chi.  One step = decode the whole batch (td_decode: site operators, gate rounds
with truncation, final contraction, log-sum, argmax) with inputs resident on the device.

Reported: syndromes/s of the mixed path (FP32 storage and contractions, FP64 truncation
cores and log-sum) and, at the same chi, of the plain FP64 GPU path; max |d log p| between
the two; the dominant kernel against its roofline; the CPU oracle on the host cores; the
end-to-end rate through the host-buffer entry point.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--chi 8] [--impl reference]
Under torchrun each rank decodes its own 4096 shots (independent replicas, no collective
on the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

D_CODE, ROUNDS, P_DATA, Q_MEAS = 9, 9, 0.03, 0.03
SHOTS = 4096
SEED = 2000            # seed of the seeded shot stream for this workload
METRIC = "syndromes decoded/sec at fixed χ vs plain FP64 GPU path; max |Δlog P_coset|"
UNIT = "syndromes/s"
CPU_SAMPLE = 48        # oracle shots for the CPU baseline (about 30 s of single-core work)


def workload(chi):
    return (f"rotated surface code d={D_CODE}, phenomenological p=q={P_DATA}, {ROUNDS} noisy + 1 perfect "
            f"rounds (9x9x10 network), {SHOTS} seeded shots, chi={chi}, chi_mps={chi}")


# ---------------------------------------------------------------- CPU oracle leg
def _oracle_chunk(args):
    first, n, chi = args
    from oracle import su
    from td_inputs import rotated_phenomenological, sample_shots
    dem = rotated_phenomenological(D_CODE, ROUNDS, P_DATA, Q_MEAS)
    det, _ = sample_shots(dem, n, seed=SEED, first_shot=first)
    t = time.perf_counter()
    out = su.su_logprob(dem, det, chi=chi, chi_mps=chi)
    return time.perf_counter() - t, out


def cpu_baseline(chi, n_shots=CPU_SAMPLE, first=0):
    """Time the FP64 oracle (same chi) on the host cores, one process per core (spawn)."""
    import multiprocessing as mp
    cores = min(os.cpu_count() or 1, n_shots)
    per = [n_shots // cores + (1 if i < n_shots % cores else 0) for i in range(cores)]
    jobs, s = [], first
    for n in per:
        if n:
            jobs.append((s, n, chi))
            s += n
    ctx = mp.get_context("spawn")
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in saved:
        os.environ[k] = "1"          # one BLAS thread per worker process
    with ctx.Pool(len(jobs)) as pool:
        pool.map(_oracle_chunk, [(first, 1, chi)] * len(jobs))      # imports warm in every worker
        t0 = time.perf_counter()
        res = pool.map(_oracle_chunk, jobs)
        wall = time.perf_counter() - t0
    for k, v in saved.items():
        if v is None:
            os.environ.pop(k, None)
        else:
            os.environ[k] = v
    return {"value": n_shots / wall, "unit": UNIT, "cores": len(jobs), "kind": "oracle", "wall_s": wall,
            "sample": f"{n_shots} shots of the same seeded stream, FP64 numpy simple-update sweep at the same chi, "
                      f"{len(jobs)} spawned processes, wall {wall:.2f} s (CPU {sum(r[0] for r in res):.1f} s)"}


_GRAD_JAC = {}


def _oracle_grad_chunk(args):
    first, n = args
    from oracle import reverse
    from td_inputs import log_uniform_rates, rotated_phenomenological, sample_shots
    dem = log_uniform_rates(rotated_phenomenological(7, 7, 0.005, 0.005), seed=5000)
    if "jac" not in _GRAD_JAC:       # the rates' map to the objects: once per worker, untimed
        _GRAD_JAC["jac"] = reverse.object_jacobian(dem)
    det, _ = sample_shots(dem, n, seed=5001, first_shot=first)
    t = time.perf_counter()
    reverse.reverse_grad_total_logprob(dem, det, 8, 8, jac=_GRAD_JAC["jac"])
    return time.perf_counter() - t


def cpu_grad_baseline(n_shots=16):
    """Time the oracle's reverse sweep (numpy FP64) on the gradient workload, one shot per
    process (spawn), after a warm-up call per worker."""
    import multiprocessing as mp
    cores = min(os.cpu_count() or 1, n_shots)
    per = [n_shots // cores + (1 if i < n_shots % cores else 0) for i in range(cores)]
    jobs, s = [], 0
    for n in per:
        if n:
            jobs.append((s, n))
            s += n
    ctx = mp.get_context("spawn")
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in saved:
        os.environ[k] = "1"
    with ctx.Pool(len(jobs)) as pool:
        pool.map(_oracle_grad_chunk, [(0, 1)] * len(jobs))
        t0 = time.perf_counter()
        res = pool.map(_oracle_grad_chunk, jobs)
        wall = time.perf_counter() - t0
    for k, v in saved.items():
        if v is None:
            os.environ.pop(k, None)
        else:
            os.environ[k] = v
    return {"value": n_shots / wall, "unit": "gradient shots/s", "cores": len(jobs), "kind": "oracle",
            "sample": f"{n_shots} shots of the gradient workload, oracle reverse sweep (numpy FP64, chi = 8), "
                      f"{len(jobs)} spawned processes, wall {wall:.2f} s (CPU {sum(res):.1f} s)"}


# ---------------------------------------------------------------- replicas
def replica_first_shot(rank, shots_per_rank):
    """First shot of a rank's slice of the seeded stream: ranks decode disjoint, contiguous
    slices, so N replicas together decode the first N * shots_per_rank shots."""
    return rank * shots_per_rank


def max_over_ranks(value, world, device="cpu"):
    """Largest value over the ranks (the timed region is the slowest replica's)."""
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def mean_over_ranks(vec, count, world, device="cpu"):
    """Shot-weighted mean over the ranks of per-rank means (the gradient of the mean log P
    when the shots are split across ranks: the one collective of the gradient path)."""
    import torch
    v = torch.as_tensor(vec, dtype=torch.float64, device=device).reshape(-1)
    t = torch.cat([v * float(count), torch.tensor([float(count)], dtype=torch.float64, device=device)])
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t[:-1] / t[-1]


# ---------------------------------------------------------------- clocks
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.p is not None:
            self.p.terminate()
            try:
                out, _ = self.p.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()
                out, _ = self.p.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        loaded = [s for s in sm if s > 0.5 * (mx or max(sm))] or sm
        loaded.sort()
        return {"sm_mhz": loaded[len(loaded) // 2], "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- reference arm
def run_reference(args, rank, world):
    if rank != 0:
        return
    chi = args.chi
    per_step = max(16, os.cpu_count() or 16)
    for _ in range(args.warmup):
        cpu_baseline(chi, per_step)
    vals = [cpu_baseline(chi, per_step, first=k * per_step) for k in range(args.steps)]
    wall = sum(v["wall_s"] for v in vals)          # oracle time only (pool start-up excluded)
    value = args.steps * per_step / wall
    cb = dict(vals[-1])
    cb["value"] = value
    cb["sample"] = f"{per_step} shots per step ({args.steps} steps) of the seeded stream, FP64 oracle at chi={chi}"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * wall / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": workload(chi), "shots_per_step": per_step},
            "cpu_baseline": cb, "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                                        "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- our arm
def main():
    global SHOTS
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--chi", type=int, default=8)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-tune", action="store_true", help="keep the default launch schedule")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 GPU path")
    ap.add_argument("--shots", type=int, default=SHOTS, help="shots per GPU (profiling runs use fewer)")
    ap.add_argument("--no-extra", action="store_true", help="skip the other workloads (reported beside the line)")
    args = ap.parse_args()
    SHOTS = args.shots
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    # the CPU oracle runs in spawned workers before any GPU work in this process
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(args.chi)

    import torch
    import torch.distributed as dist
    import paper_2310_10722_gb300 as td
    from td_inputs import rotated_phenomenological, sample_shots

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")

    def barrier():
        if world > 1:
            dist.barrier()

    chi = args.chi
    dem = rotated_phenomenological(D_CODE, ROUNDS, P_DATA, Q_MEAS)
    det_np, _ = sample_shots(dem, SHOTS, seed=SEED, first_shot=replica_first_shot(rank, SHOTS))
    det = torch.from_numpy(det_np).cuda()
    net = td.Network.from_dem(dem, chi=chi, chi_mps=chi, precision=td.TD_FP32, mem_budget=96 << 30,
                              max_wave=SHOTS)
    info = net.info()
    work = net.work()
    waves = math.ceil(SHOTS / info["wave"])
    stream = torch.cuda.current_stream()
    # launch schedule picked by the autotuner on the first 1024 shots (outside the timed region)
    schedule = net.tune(det[:1024]) if not args.no_tune else None

    for _ in range(args.warmup):
        net.decode(det)
    torch.cuda.synchronize()

    # timed region: K steps, barrier + synchronize on both sides, CUDA events per step
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    net.profile(True)
    with Clocks(local) as clk:
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(args.steps):
            ev[k][0].record(stream)
            net.decode(det)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        barrier()
        wall = time.perf_counter() - t0
    prof = net.profile(False)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    dev_s = sum(step_ms) / 1000.0
    t_max = max_over_ranks(dev_s, world, device="cuda")
    value = world * SHOTS * args.steps / t_max

    # end to end through the host-buffer entry point (pinned copies inside the timed region)
    det_h = torch.from_numpy(det_np).pin_memory()
    out_h = torch.empty((SHOTS, 2), dtype=torch.float64).pin_memory()
    net.coset_logprob_host(det_h, out=out_h)
    barrier()
    torch.cuda.synchronize()
    te = time.perf_counter()
    for _ in range(args.steps):
        net.coset_logprob_host(det_h, out=out_h)
    torch.cuda.synchronize()
    barrier()
    e2e_s = time.perf_counter() - te
    e2e = {"value": world * SHOTS * args.steps / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": int(det_np.nbytes), "d2h_bytes_per_step": int(out_h.numel() * 8),
           "entry": "td_coset_logprob_host"}

    # plain FP64 GPU path at the same chi, and accuracy of the mixed path against it
    fp64 = None
    if not args.no_fp64:
        net64 = td.Network.from_dem(dem, chi=chi, chi_mps=chi, precision=td.TD_FP64, mem_budget=96 << 30,
                                  max_wave=SHOTS)
        sched64 = net64.tune(det[:1024]) if not args.no_tune else None
        net64.decode(det[:256])
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        lp64 = net64.coset_logprob(det)
        b.record(stream)
        torch.cuda.synchronize()
        ms64 = a.elapsed_time(b)
        lp32 = net.coset_logprob(det)
        d = (lp32 - lp64).abs()
        both = torch.isinf(lp32) & torch.isinf(lp64)
        d = torch.where(both, torch.zeros_like(d), d)
        tot32 = torch.logsumexp(lp32, dim=1)
        tot64 = torch.logsumexp(lp64, dim=1)
        dec_diff = int(((lp32[:, 1] > lp32[:, 0]) != (lp64[:, 1] > lp64[:, 0])).sum())
        dflat = d.max(dim=1).values
        # decisions compared only where the FP64 margin exceeds the mixed path's typical error
        margin64 = (lp64[:, 1] - lp64[:, 0]).abs()
        sure = margin64 > 1e-3
        dec_diff_sure = int((((lp32[:, 1] > lp32[:, 0]) != (lp64[:, 1] > lp64[:, 0])) & sure).sum())
        fp64 = {"value": SHOTS / (ms64 / 1000.0), "unit": UNIT, "ms_per_step": ms64,
                "max_dlogp_coset": float(d.max()), "median_dlogp_coset": float(d.median()),
                "p99_dlogp_coset": float(torch.quantile(dflat, 0.99)),
                "frac_shots_within_1e-3": float((dflat <= 1e-3).double().mean()),
                # the coset the FP64 path ranks first (the decision's coset), and the other one:
                # FP32 arithmetic in the shared final contraction errs by ~eps32 exp(margin)
                # on the minority coset
                "max_dlogp_majority_coset": float(d.gather(1, (lp64[:, 1] > lp64[:, 0]).long()[:, None]).max()),
                "max_dlogp_minority_coset": float(d.gather(1, (lp64[:, 1] <= lp64[:, 0]).long()[:, None]).max()),
                "max_dlogP_total": float(torch.where(torch.isinf(tot32) & torch.isinf(tot64),
                                                     torch.zeros_like(tot32), (tot32 - tot64).abs()).max()),
                "decisions_differ": dec_diff,
                "decisions_differ_where_margin_gt_1e-3": dec_diff_sure, "schedule": sched64}
        net64.close()

    # other workloads of the same path, reported beside the headline (a few seconds each)
    extra = None
    if not args.no_extra and rank == 0:
        from td_inputs import point_sector_3d
        extra = {}

        def rate(dem_x, shots, seed, **kw):
            dx, _ = sample_shots(dem_x, shots, seed=seed)
            dd = torch.from_numpy(dx).cuda()
            nx = td.Network.from_dem(dem_x, mem_budget=32 << 30, **kw)
            nx.coset_logprob(dd[: min(64, shots)])
            torch.cuda.synchronize()
            ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ea.record(stream)
            lp = nx.coset_logprob(dd)
            eb.record(stream)
            torch.cuda.synchronize()
            ms_x = ea.elapsed_time(eb)
            nx.close()
            return shots / (ms_x / 1000.0), lp

        r1, _ = rate(point_sector_3d(3, 0.05), 512, 1000, chi=8, chi_mps=64, precision=td.TD_FP64)
        extra["point_sector_d3_p0.05_512shots_exact_fp64"] = {"value": r1, "unit": UNIT}
        r32, lp32x = rate(dem, 256, SEED, chi=16, chi_mps=8, precision=td.TD_FP32)
        r64, lp64x = rate(dem, 256, SEED, chi=16, chi_mps=8, precision=td.TD_FP64)
        dx = (lp32x - lp64x).abs()
        dx = torch.where(torch.isinf(lp32x) & torch.isinf(lp64x), torch.zeros_like(dx), dx)
        extra["rotated_d9_chi16_chimps8_256shots"] = {
            "mixed": {"value": r32, "unit": UNIT}, "fp64": {"value": r64, "unit": UNIT},
            "max_dlogp_coset_mixed_vs_fp64": float(dx.max()), "median_dlogp_coset": float(dx.median())}

    # uneven batch: point-sector codes d = 5, 7, 9, 11 decoded together, their decode calls
    # captured once in a CUDA graph and replayed (one network per code size)
    if extra is not None:
        from td_inputs import point_sector_3d
        # 152 shots per code size: one shot per SM in the final contraction (one block per
        # shot), as in a large mixed batch; each network tuned on its first 32 shots
        per, chi_u = 152, 16
        nets_u, dets_u, outs_u, sched_u = [], [], [], []
        for dcode in (5, 7, 9, 11):
            dem_u = point_sector_3d(dcode, 0.1)
            du, _ = sample_shots(dem_u, per, seed=4000 + dcode)
            nets_u.append(td.Network.from_dem(dem_u, chi=chi_u, chi_mps=8, precision=td.TD_FP32,
                                              mem_budget=48 << 30))
            dets_u.append(torch.from_numpy(du).cuda())
            sched_u.append(nets_u[-1].tune(dets_u[-1][:32]))     # per-(d, chi) schedule, outside the capture
            outs_u.append(torch.empty((per, 2), dtype=torch.float64, device="cuda"))
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):                  # warm-up outside the capture
            for n_u, d_u, o_u in zip(nets_u, dets_u, outs_u):
                n_u.coset_logprob(d_u, out=o_u)
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        ref_u = [o.clone() for o in outs_u]
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            for n_u, d_u, o_u in zip(nets_u, dets_u, outs_u):
                n_u.coset_logprob(d_u, out=o_u)
        ga, gb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ga.record(stream)
        graph.replay()
        gb.record(stream)
        torch.cuda.synchronize()
        extra["point_sector_uneven_d5_7_9_11_chi16_graph"] = {
            "value": 4 * per / (ga.elapsed_time(gb) / 1000.0), "unit": UNIT, "shots": 4 * per,
            "replay_matches_eager": all(torch.equal(a, b) for a, b in zip(ref_u, outs_u)),
            "schedules": {f"d{dc}": sc for dc, sc in zip((5, 7, 9, 11), sched_u)},
            "note": "p=0.1, chi=16, chi_mps=8, FP32 storage; one network per code size with its launch "
                    "schedule picked by td_network_tune, all decode calls captured in one CUDA graph"}
        for n_u in nets_u:
            n_u.close()

    # gradient of the mean log P with respect to every mechanism rate: rotated d=7, 7 noisy
    # rounds + 1 perfect, per-mechanism rates log-uniform in [1e-3, 1e-2], 1024 shots per
    # GPU, by the reverse sweep (td_grad_logprob); every rank takes its own slice of the shots
    # and the per-rank gradients are combined by one all-reduce (the only collective of the
    # gradient path).  Beside it, the forced-rate gradient (td_grad_logprob_forced, 1 + 2 x
    # 560 decodes per shot) on 16 of the shots.
    if not args.no_extra:
        from td_inputs import log_uniform_rates
        dem_g = log_uniform_rates(rotated_phenomenological(7, 7, 0.005, 0.005), seed=5000)
        g_shots = 1024
        dg, _ = sample_shots(dem_g, g_shots, seed=5001, first_shot=replica_first_shot(rank, g_shots))
        ddg = torch.from_numpy(dg).cuda()
        ng = td.Network.from_dem(dem_g, chi=8, chi_mps=8, precision=td.TD_FP64, mem_budget=64 << 30)
        ng.grad_logprob(ddg)                # allocations, forced-object tables, warm-up
        ng.coset_logprob(ddg)
        torch.cuda.synchronize()
        barrier()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        ev[0].record(stream)
        lpg, gg = ng.grad_logprob(ddg)
        ev[1].record(stream)
        ng.coset_logprob(ddg)
        ev[2].record(stream)
        torch.cuda.synchronize()
        t_g = max_over_ranks(ev[0].elapsed_time(ev[1]) / 1000.0, world, "cuda")
        t_d = max_over_ranks(ev[1].elapsed_time(ev[2]) / 1000.0, world, "cuda")
        g_all = mean_over_ranks(gg, g_shots, world, "cuda")
        gres = {"value": world * g_shots / t_g, "unit": "gradient shots/s",
                "seconds_per_1024_shots": t_g, "decode_seconds_same_shots_fp64": t_d,
                "gradient_over_decode_time": t_g / t_d, "rates": dem_g.n_mech,
                "grad_abs_max": float(g_all.abs().max())}
        # forced-rate gradient on 16 shots (mixed-precision decodes) and the reverse sweep on
        # the same shots: they differ by the truncation error of the forced networks only
        nf = td.Network.from_dem(dem_g, chi=8, chi_mps=8, precision=td.TD_FP32, mem_budget=32 << 30)
        nf.grad_logprob(ddg[:1], method="forced")
        torch.cuda.synchronize()
        ev[0].record(stream)
        _, gf = nf.grad_logprob(ddg[:16], method="forced")
        ev[1].record(stream)
        torch.cuda.synchronize()
        _, gr16 = ng.grad_logprob(ddg[:16])
        gres["forced_rate_method"] = {"value": 16 / (ev[0].elapsed_time(ev[1]) / 1000.0), "unit": "gradient shots/s",
                                      "decodes_per_shot": 1 + 2 * dem_g.n_mech,
                                      "max_abs_diff_vs_reverse_rel_to_max": float((gf - gr16).abs().max()
                                                                                  / gr16.abs().max())}
        if rank == 0 and world == 1 and not args.no_cpu:
            gres["cpu_baseline"] = cpu_grad_baseline()
        gres["note"] = (f"{g_shots} shots per GPU, chi = chi_mps = 8 (chi = 32 of the workload is out of reach: "
                        "~7 min per decode); reverse sweep in FP64: recorded forward + per-shot adjoint")
        ng.close()
        nf.close()
        if extra is not None:
            extra["grad_rotated_d7_7rounds_loguniform_chi8"] = gres

    # roofline of the dominant kernel (largest summed device time in the timed region)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    fp32_alu = 152 * 128 * 2 * 2.07e9 / 1e12          # TF/s: SMs x FP32 lanes x FMA x max clock
    fp64_alu = 1.25                                      # TF/s, nominal GB300 FP64
    tot_ms = sum(v[0] for v in prof.values())
    dom = max(prof, key=lambda k: prof[k][0])
    ms, launches = prof[dom]
    wb, wf, wf64 = work[dom]
    shots_done = SHOTS * args.steps
    if dom in ("gram", "update", "local"):
        ach = wb * shots_done / (ms / 1000.0) / 1e9
        roof = {"kernel": f"k_{dom}", "bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
                "frac": ach / hbm, "traffic": None, "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)"}
    elif wf64 >= 0.5 * wf:
        ach = wf * shots_done / (ms / 1000.0) / 1e12
        roof = {"kernel": f"k_{dom}", "bound": "alu", "achieved": ach, "peak": fp64_alu, "unit": "TFLOP/s",
                "frac": ach / fp64_alu, "traffic": None,
                "peak_source": "FP64 1.25 TFLOP/s nominal (probe measured 1.19)"}
    else:
        ach = wf * shots_done / (ms / 1000.0) / 1e12
        roof = {"kernel": f"k_{dom}", "bound": "alu", "achieved": ach, "peak": fp32_alu, "unit": "TFLOP/s",
                "frac": ach / fp32_alu, "traffic": None,
                "peak_source": "FP32 CUDA cores 152 SMs x 128 lanes x 2 x 2.07 GHz (derived)"}
    roof.update({"launches": launches, "avg_launch_ms": ms / max(launches, 1), "time_share": ms / tot_ms,
                 "algorithmic_per_shot": {"bytes": wb, "flops": wf, "fp64_flops": wf64}})

    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1000.0 * t_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32 (FP64 arithmetic in the sweep on FP32 storage; FP32 final contraction; FP64 log-sum)",
        "data": "synthetic",
        "config": {"workload": workload(chi), "shots_per_gpu": SHOTS, "chi": chi, "chi_mps": chi,
                   "precision": "fp32", "wave": info["wave"], "workspace_gb": info["workspace_bytes"] / 1e9,
                   "l2": f"not flushed: per-step working set {info['workspace_bytes'] / 1e9:.1f} GB of site tensors "
                         "rewritten every step, far above the 129 MB L2",
                   "parallelism": f"replicas x{world}", "schedule": schedule},
        "wall_s_timed": wall,
        "fp64_path": fp64,
        "speedup_vs_fp64": (value / world / fp64["value"]) if fp64 else None,
        "roofline": roof,
        "kernel_time_share": {k: round(v[0] / tot_ms, 4) for k, v in prof.items()},
        # share of the timed device time in kernels that compute in FP64 (the Gram, update,
        # truncation core and site-local operators; the final contraction is FP32 here)
        "fp64_time_share": round(sum(prof[k][0] for k in ("local", "gram", "core", "update") if k in prof) / tot_ms, 4),
        "tensor_pipe": "unused: every contraction of the sweep needs FP64 accumulation",
        "cpu_baseline": cpu,
        "e2e": e2e,
        "clocks": clk.summary(),
        "gpu_launches": int(info["launches_per_wave"] * waves * args.steps),
        "other_workloads": extra,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

#!/usr/bin/env python
"""Throughput of tensor-network coset decoding on one GB300 (arXiv 2310.10722, Sec. 4).

Workload: rotated surface code d=9 with phenomenological noise (data p=0.03, measurement
q=0.03), 9 noisy syndrome rounds + 1 perfect round (a 40-site x 10-layer detector network),
4096 seeded synthetic shots per GPU, simple-update bond chi (default 8), final MPS bond
chi_mps = chi.  One step = decode the whole batch (td_decode: site operators, gate rounds
with truncation, final contraction, log-sum, argmax) with inputs resident on the device.

Reported: syndromes/s of the mixed-precision path (--precision tc: FP64 storage, the Gram
contractions on the tcgen05 tensor cores from exact BF16 slices, FP32-preconditioned SVDs
finished in FP64) and, at the same chi, of the plain FP64 GPU path with |d log p| of every
coset between the two; the dominant kernel against its roofline (measured FMA peak); the CPU
oracle on the host cores; the end-to-end rate through the host-buffer entry point; beside
them chi = 16, the exact 3D point sector d = 3, the uneven point-sector batch in one CUDA
graph and the reverse-sweep gradient.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--chi 8] [--precision tc|fp32|fp64]
                  [--impl reference]
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
PRECISIONS = {"fp64": 0, "fp32": 1, "tc": 2}
# the arithmetic type of each path, and what computes in it
DTYPES = {"fp64": "f64", "fp32": "f64", "tc": "f64"}
PRECISION_DETAIL = {
    "fp64": "f64 storage and arithmetic on the CUDA cores",
    "fp32": "f32 storage; Gram from exact bf16 slices on tcgen05 (fp32 TMEM sums, exact), f64 combination; "
            "f64 update; f32-preconditioned f64 SVDs; f64 final contraction",
    "tc": "f64 storage; Gram from exact bf16 slices on tcgen05 (fp32 TMEM sums, exact), f64 combination; "
          "f64 update; f32-preconditioned f64 SVDs; f64 final contraction"}


def _f(x, digits=4):
    x = float(x)
    return x if not math.isfinite(x) or x == 0 else float(f"{x:.{digits}g}")


def coset_stats(lp, lp64):
    """|d log p| of every coset of lp against lp64: the FP64 path's decision coset and the
    other one, the total log P, decisions where the FP64 margin exceeds 1e-3.  Cosets that
    are -inf on both sides count as equal; -inf on one side only is counted apart."""
    import torch
    fin = torch.isfinite(lp) & torch.isfinite(lp64)
    both_inf = torch.isinf(lp) & torch.isinf(lp64)
    d = torch.where(fin, (lp - lp64).abs(), torch.zeros_like(lp))
    maj = (lp64[:, 1] > lp64[:, 0]).long()
    dmaj = d.gather(1, maj[:, None])[:, 0]
    dmin = d.gather(1, (1 - maj)[:, None])[:, 0]
    tot, tot64 = torch.logsumexp(lp, 1), torch.logsumexp(lp64, 1)
    dt = torch.where(torch.isfinite(tot) & torch.isfinite(tot64), (tot - tot64).abs(), torch.zeros_like(tot))
    dec = (lp[:, 1] > lp[:, 0]) != (lp64[:, 1] > lp64[:, 0])
    sure = (lp64[:, 1] - lp64[:, 0]).abs() > 1e-3
    return {"max_dlogp_coset": _f(d.max()), "max_dlogp_decision_coset": _f(dmaj.max()),
            "max_dlogp_other_coset": _f(dmin.max()), "frac_within_1e-3": _f((d.max(1).values <= 1e-3).double().mean()),
            "max_dlogP_total": _f(dt.max()), "inf_on_one_side": int((~fin & ~both_inf).sum()),
            "decisions_differ_margin_gt_1e-3": int((dec & sure).sum())}


def timed_decode(net, det, stream):
    import torch
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    lp = net.coset_logprob(det)
    b.record(stream)
    torch.cuda.synchronize()
    return lp, a.elapsed_time(b)


def main():
    global SHOTS
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--chi", type=int, default=8)
    ap.add_argument("--precision", default="tc", choices=sorted(PRECISIONS))
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-tune", action="store_true", help="keep the default launch schedule")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 GPU path")
    ap.add_argument("--shots", type=int, default=SHOTS, help="shots per GPU (profiling runs use fewer)")
    ap.add_argument("--no-extra", action="store_true", help="skip the other workloads (reported beside the line)")
    ap.add_argument("--chi16-shots", type=int, default=256, help="shots of the chi = 16 line")
    ap.add_argument("--uneven-per-size", type=int, default=152, help="shots per code size of the uneven batch")
    ap.add_argument("--loop-shots", type=int, default=1024, help="shots of the loop-sector line")
    ap.add_argument("--chi32-shots", type=int, default=0, help="shots of the chi = 32 line (0: skipped)")
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

    chi, prec = args.chi, PRECISIONS[args.precision]
    stream = torch.cuda.current_stream()
    # measured FMA throughput of this GPU (the roofline denominators of the CUDA-core kernels)
    fma64 = td.fma_peak_tflops(fp64=True)
    fma32 = td.fma_peak_tflops(fp64=False)

    dem = rotated_phenomenological(D_CODE, ROUNDS, P_DATA, Q_MEAS)
    det_np, _ = sample_shots(dem, SHOTS, seed=SEED, first_shot=replica_first_shot(rank, SHOTS))
    det = torch.from_numpy(det_np).cuda()
    net = td.Network.from_dem(dem, chi=chi, chi_mps=chi, precision=prec, mem_budget=96 << 30, max_wave=SHOTS)
    info = net.info()
    work = net.work()
    waves = math.ceil(SHOTS / info["wave"])
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
    net.check()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    t_max = max_over_ranks(sum(step_ms) / 1000.0, world, device="cuda")
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
    e2e = {"value": _f(world * SHOTS * args.steps / e2e_s), "unit": UNIT,
           "h2d_bytes_per_step": int(det_np.nbytes), "d2h_bytes_per_step": int(out_h.numel() * 8),
           "entry": "td_coset_logprob_host"}

    # the plain FP64 GPU path at the same chi, and every coset of the headline path against it
    fp64 = None
    lp_head = net.coset_logprob(det)
    if not args.no_fp64:
        net64 = td.Network.from_dem(dem, chi=chi, chi_mps=chi, precision=td.TD_FP64, mem_budget=96 << 30,
                                    max_wave=SHOTS)
        if not args.no_tune:
            net64.tune(det[:1024])
        net64.decode(det[:256])
        torch.cuda.synchronize()
        lp64, ms64 = timed_decode(net64, det, stream)
        fp64 = {"value": _f(SHOTS / (ms64 / 1000.0)), **coset_stats(lp_head, lp64)}
        net64.close()

    # roofline of the dominant kernel (largest summed device time in the timed region)
    tot_ms = sum(v[0] for v in prof.values())
    dom = max(prof, key=lambda k: prof[k][0])
    ms, launches = prof[dom]
    wb, wf, wf64 = work[dom]
    shots_done = SHOTS * args.steps
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    if dom in ("local", "update") and prec == 1:
        ach, peak, unit, bound = wb * shots_done / (ms / 1000.0) / 1e9, float(peaks.get("hbm_gbs", 6800.0)), "GB/s", "hbm"
        src = "MEASURED_PEAKS.json hbm_gbs (of measured)"
    else:
        ach, peak, unit, bound = wf * shots_done / (ms / 1000.0) / 1e12, fma64, "TFLOP/s", "alu"
        src = "FP64 FMA throughput measured in this run by td_measure_fma_peak (of measured)"
    roof = {"kernel": f"k_{dom}", "bound": bound, "achieved": _f(ach), "peak": _f(peak), "unit": unit,
            "frac": _f(ach / peak, 3), "traffic": (_f(KERNEL_TRAFFIC[(dom, args.precision, chi)][0] * shots_done / max(launches, 1))
                        if (dom, args.precision, chi) in KERNEL_TRAFFIC else None),
            "traffic_source": (KERNEL_TRAFFIC.get((dom, args.precision, chi)) or (None, None))[1],
            "peak_source": src, "avg_launch_ms": _f(ms / max(launches, 1)), "time_share": _f(ms / tot_ms, 3),
            "flops_per_shot": _f(wf), "fp64_flops_per_shot": _f(wf64)}

    # other workloads of the same path, reported beside the headline (a few seconds each)
    extra = {}
    if not args.no_extra and rank == 0:
        from td_inputs import point_sector_3d
        dx, _ = sample_shots(point_sector_3d(3, 0.05), 512, seed=1000)
        n1 = td.Network.from_dem(point_sector_3d(3, 0.05), chi=8, chi_mps=64, precision=td.TD_FP64)
        dd = torch.from_numpy(dx).cuda()
        n1.coset_logprob(dd[:64])
        _, m1 = timed_decode(n1, dd, stream)
        extra["point_d3_exact_fp64_512"] = _f(512 / (m1 / 1000.0))
        n1.close()
        # rotated d = 9 at chi = chi_mps = 16 on the first chi16_shots shots of the stream
        n16 = args.chi16_shots
        d16 = det[:n16].contiguous()
        r16 = {}
        lps = {}
        for name, pv in (("fp64", 0), (args.precision, prec)):
            nx = td.Network.from_dem(dem, chi=16, chi_mps=16, precision=pv, mem_budget=96 << 30)
            nx.coset_logprob(d16[:8])
            torch.cuda.synchronize()
            lps[name], mx = timed_decode(nx, d16, stream)
            nx.check()
            r16[name] = _f(n16 / (mx / 1000.0))
            nx.close()
        st16 = coset_stats(lps[args.precision], lps["fp64"])
        extra["rotated_d9_chi16_mps16"] = {"shots": n16, "fp64": r16["fp64"], args.precision: r16[args.precision],
                                           "max_dlogp_coset": st16["max_dlogp_coset"],
                                           "max_dlogp_decision_coset": st16["max_dlogp_decision_coset"]}

    # rotated d = 9 at chi = 32, chi_mps = 8 on --chi32-shots shots (off by default: ~1 GB of
    # site tensors per shot and seconds per shot even on the GPU)
    if not args.no_extra and rank == 0 and args.chi32_shots > 0:
        n32 = args.chi32_shots
        d32 = det[:n32].contiguous()
        r32, lps32 = {}, {}
        for name, pv in (("fp64", 0), (args.precision, prec)):
            nx = td.Network.from_dem(dem, chi=32, chi_mps=8, precision=pv, mem_budget=200 << 30)
            nx.coset_logprob(d32[:2])
            torch.cuda.synchronize()
            lps32[name], mx = timed_decode(nx, d32, stream)
            nx.check()
            r32[name] = _f(n32 / (mx / 1000.0))
            nx.close()
        st32 = coset_stats(lps32[args.precision], lps32["fp64"])
        extra["rotated_d9_chi32_mps8"] = {"shots": n32, "fp64": r32["fp64"], args.precision: r32[args.precision],
                                          "max_dlogp_coset": st32["max_dlogp_coset"]}

    # uneven batch: point-sector codes d = 5, 7, 9, 11 decoded together, their decode calls
    # captured once in a CUDA graph and replayed (one network per code size)
    if not args.no_extra and rank == 0:
        from td_inputs import point_sector_3d
        per, chi_u = args.uneven_per_size, 16
        nets_u, dets_u, outs_u = [], [], []
        for dcode in (5, 7, 9, 11):
            dem_u = point_sector_3d(dcode, 0.1)
            du, _ = sample_shots(dem_u, per, seed=4000 + dcode)
            nets_u.append(td.Network.from_dem(dem_u, chi=chi_u, chi_mps=8, precision=prec, mem_budget=48 << 30))
            dets_u.append(torch.from_numpy(du).cuda())
            if not args.no_tune:
                nets_u[-1].tune(dets_u[-1][:32])     # per-(d, chi) schedule, outside the capture
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
        extra["point_uneven_d5-11_chi16_mps8_graph"] = {
            "value": _f(4 * per / (ga.elapsed_time(gb) / 1000.0)), "shots": 4 * per,
            "replay_matches_eager": all(torch.equal(a, b) for a, b in zip(ref_u, outs_u))}
        for n_u in nets_u:
            n_u.close()

    # loop sector of the 3D surface code (Sec. 5.2) in the generator picture (Sec. 3.2):
    # d = 5 at p = 0.2 (near the loop threshold), chi = 8, chi_mps = 16; every shot is two
    # sweeps (both cosets)
    if not args.no_extra and rank == 0:
        from td_inputs import loop_sector_3d
        gp = loop_sector_3d(5, 0.2)
        n_l = args.loop_shots
        sl, _ = sample_shots(gp.face_dem, n_l, seed=6000)
        dl = torch.from_numpy(sl).cuda()
        res_l = {}
        for name, pv in (("fp64", 0), (args.precision, prec)):
            nl = td.GenNetwork.from_problem(gp, chi=8, chi_mps=16, precision=pv, mem_budget=64 << 30)
            nl.coset_logprob(dl[:8])
            torch.cuda.synchronize()
            lp_l, ml = timed_decode(nl, dl, stream)
            nl.check()
            res_l[name] = (lp_l, _f(n_l / (ml / 1000.0)))
            nl.close()
        stl = coset_stats(res_l[args.precision][0], res_l["fp64"][0])
        extra["loop_d5_p0.2_chi8_mps16"] = {"shots": n_l, "fp64": res_l["fp64"][1], args.precision: res_l[args.precision][1],
                                            "max_dlogp_coset": stl["max_dlogp_coset"],
                                            "max_dlogp_decision_coset": stl["max_dlogp_decision_coset"]}

    # gradient of the mean log P with respect to every mechanism rate: rotated d=7, 7 noisy
    # rounds + 1 perfect, per-mechanism rates log-uniform in [1e-3, 1e-2], 1024 shots per
    # GPU, by the reverse sweep (td_grad_logprob); every rank takes its own slice of the shots
    # and the per-rank gradients are combined by one all-reduce (the only collective of the
    # gradient path)
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
        evg = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        evg[0].record(stream)
        _, gg = ng.grad_logprob(ddg)
        evg[1].record(stream)
        ng.coset_logprob(ddg)
        evg[2].record(stream)
        torch.cuda.synchronize()
        t_g = max_over_ranks(evg[0].elapsed_time(evg[1]) / 1000.0, world, "cuda")
        t_d = max_over_ranks(evg[1].elapsed_time(evg[2]) / 1000.0, world, "cuda")
        mean_over_ranks(gg, g_shots, world, "cuda")
        gres = {"value": _f(world * g_shots / t_g), "unit": "gradient shots/s", "over_decode_time": _f(t_g / t_d, 3)}
        if rank == 0 and world == 1 and not args.no_cpu:
            gres["cpu_oracle"] = _f(cpu_grad_baseline()["value"])
        ng.close()
        extra["grad_rotated_d7_chi8_1024"] = gres

    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": _f(value), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": _f(1000.0 * t_max / args.steps), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": DTYPES[args.precision], "data": "synthetic",
        "config": {"workload": workload(chi), "precision": args.precision,
                   "precision_detail": PRECISION_DETAIL[args.precision], "shots_per_gpu": SHOTS,
                   "wave": info["wave"], "parallelism": f"replicas x{world}", "schedule": schedule,
                   "l2": "not flushed: every step rewrites %.1f GB of site tensors, far above the 129 MB L2"
                         % (info["workspace_bytes"] / 1e9)},
        "wall_s_timed": _f(wall),
        "kernel_time_share": {k: round(v[0] / tot_ms, 3) for k, v in prof.items() if v[0] > 0},
        "other_workloads": extra,
        "cpu_baseline": cpu and {k: (_f(v) if isinstance(v, float) else v) for k, v in cpu.items()},
        "e2e": e2e,
        "clocks": clk.summary(),
        "gpu_launches": int(info["launches_per_wave"] * waves * args.steps),
        "roofline": roof,
        "fp64_path": fp64,
        "speedup_vs_fp64": _f(value / world / fp64["value"], 3) if fp64 else None,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


# DRAM traffic per launch of the dominant kernel from one ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum), keyed by (kernel class, precision, chi); see profiles/.  None until a
# capture of the current kernel exists.
# DRAM bytes per launch of the dominant kernel (ncu dram__bytes_read.sum + dram__bytes_write.sum),
# keyed by (kernel class, precision, chi): (bytes, how they were obtained).  None once the
# kernel has changed since the capture.
# DRAM bytes per shot of the dominant kernel (ncu dram__bytes_read.sum + dram__bytes_write.sum of
# one launch, divided by its shots), keyed by (kernel class, precision, chi): (bytes per shot,
# how they were obtained).  The line reports them x the shots of one launch (one block per shot,
# so the traffic grows with the shots).  Remove an entry when its kernel changes.
KERNEL_TRAFFIC = {
    ("final", "tc", 8): (10.548e9 / 1024, "one k_final launch over 1024 shots: 3.384 GB read + 7.164 GB written "
                                          "(profiles/k_final_dram_rotated_d9_chi8_tc.md), scaled to this launch's shots"),
}


if __name__ == "__main__":
    main()

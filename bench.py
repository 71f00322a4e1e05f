"""Benchmark of the hQR hot path on GB300: HODLR-QR factorizations per second (FP64).

Workload (one step = `--batch` independent full factorizations, Alg. 2 with every step on the
device, factored concurrently as one CUDA graph; `--batch 1` is the plain one-matrix path):
  n = 8192, nmin = 256 (5 levels), off-diagonal rank 10 with Gaussian factors N(0,1)/sqrt(n),
  leaves N(0,1) + 4 I, columns scaled by 10^(-14 j/(n-1)) (condition number ~1e14), tol = 1e-12,
  synthetic and seeded.  ||A||_2 is estimated on the device inside every step.

Timed arms (one JSON line on rank 0):
  value      device throughput: A restored from a device snapshot and factored by one CUDA-graph
             launch per step, CUDA events on the library's stream around each step, L2 flushed
             (256 MiB write) between steps outside the timed events.
  e2e        the same through the public C ABI with host buffers: pinned host -> device upload of
             the matrix, factorization, and a device -> host read of the whole factorization in
             compact form (every factor at its stored rank).
  single_matrix  the plain one-matrix-at-a-time path (16-CTA clusters) on the same GPU.
  roofline   the batched step against the FP64 ALU peak: algorithmic flops of one graph launch
             (all factorizations of the step; QR, Jacobi and GEMM kernels run concurrently)
             over that launch's event-timed duration; `per_kernel` adds each kernel kind's
             per-launch figures from an event-instrumented run of one factorization.
  served     p50/p99 latency of a Poisson stream of factorize+solve and repeat-solve requests
             through the continuously batched server.
  cpu_baseline  the CPU oracle timed on the host cores on one factorization of the same workload.

`--impl reference` times the CPU oracle itself (the paper publishes no code and no timings).
Under torchrun every rank factors its own matrix (replicas only: one factorization does not
shard), with no collective on the data path; rank 0 prints the line.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "HODLR-QR factorizations/s (FP64, tol 1e-12)"
UNIT = "factorizations/s"
WORKLOAD = "hodlr_qr_n8192_nmin256_k10_colscaled1e-14_tol1e-12"
N, NMIN, K, DECADES, TOL = 8192, 256, 10, 14.0, 1e-12
RANK_CAP = 128
BATCH_CLUSTER = 4          # default cluster size when several matrices are factored per step
# FP64 roofline denominator: the DFMA rate measured on this GPU model by hodlr_fp64_peak
# (`python bench.py --peaks`), recorded with its command and clocks in this file
PEAK_RECORD = os.path.join("profiles", "fp64_peak.md")


def recorded_fp64_peak():
    """(DFMA TFLOP/s, DMMA TFLOP/s) from the committed measurement record, or None."""
    import re
    path = os.path.join(ROOT, PEAK_RECORD)
    if not os.path.exists(path):
        return None
    vals = {}
    for line in open(path):
        m = re.match(r"^\s*(dfma_tflops|dmma_tflops):\s*([0-9.eE+-]+)\s*$", line)
        if m:
            vals[m.group(1)] = float(m.group(2))
    if "dfma_tflops" not in vals:
        return None
    return vals["dfma_tflops"], vals.get("dmma_tflops")


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def rank_seeds(rank, nb):
    """Seeds of the matrices one rank factors per step: replicas only, every rank its own
    disjoint set of nb matrices, no data shared between ranks."""
    return [rank * nb + i for i in range(nb)]


def max_over_ranks(x, device="cpu"):
    """The largest x over the ranks of the default process group (x itself without one): the
    timed region of the slowest rank sets the whole job's time."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(ws, nb, steps, seconds):
    """Factorizations per second of the whole job: every rank factors nb matrices per step."""
    return ws * nb * steps / seconds


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def make_input(seed):
    import workloads as W
    return W.random_hodlr(N, NMIN, K, seed=seed, col_scale_decades=DECADES, name=WORKLOAD)


def cpu_threads():
    try:
        import threadpoolctl
        info = threadpoolctl.threadpool_info()
        t = [i.get("num_threads", 0) for i in info if i.get("user_api") == "blas"]
        if t:
            return int(max(t))
    except Exception:
        pass
    return os.cpu_count() or 1


def time_oracle(inp, reps=1):
    """Wall time of the CPU oracle on full factorizations of `inp` (seconds per factorization)."""
    import oracle.core as O
    ts = []
    for _ in range(reps):
        A = O.from_input(inp)
        t0 = time.perf_counter()
        O.hqr(A, TOL)
        ts.append(time.perf_counter() - t0)
    return min(ts)


def served_requests(seed=4242, count=32, mean_gap_s=0.05):
    """A factorize+solve request stream: Poisson arrivals; matrices from the random (n = 1024,
    2048), ill-conditioned column-scaled (n = 2048, 4096), kernel-generated (n = 2048) and
    symmetric banded (b = 8, n = 4096, 8192) families; 1-64 right-hand sides; a third of the
    requests are repeat solves with factors kept on the device."""
    import workloads as W
    from paper_1809_10585_gb300 import server as S
    rng = np.random.default_rng(seed)
    makers = [
        lambda i: W.random_hodlr(int(rng.choice([1024, 2048])), 128, 5, seed=seed + i),
        lambda i: W.scaled_config1(int(rng.choice([2048, 4096])), 256, 10, seed=seed + i, decades=10.0),
        lambda i: W.kernel_hodlr(2048, 256, 1e-12, seed=seed + i),
        lambda i: W.banded_hodlr(int(rng.choice([4096, 8192])), 8, 256, seed=seed + i),
    ]
    reqs, kept, t = [], [], 0.0
    for i in range(count):
        t += float(rng.exponential(mean_gap_s))
        nrhs = int(rng.integers(1, 65))
        if kept and rng.uniform() < 1.0 / 3.0:
            key, n = kept[int(rng.integers(len(kept)))]
            reqs.append(S.Solve(key, W.rhs(n, nrhs, seed=seed + 1000 + i), arrival=t))
            continue
        inp = makers[i % len(makers)](i)
        keep = bool(rng.uniform() < 0.5)
        key = f"r{i}" if keep else None
        reqs.append(S.FactorSolve(inp, W.rhs(inp.n, nrhs, seed=seed + 2000 + i), TOL, keep, key, arrival=t))
        if keep:
            kept.append((key, inp.n))
    return reqs


def served_leg(device):
    """Run the request stream through the continuously batched server; p50/p99 latency is from
    arrival to the solution being back on the host."""
    from paper_1809_10585_gb300 import server as S
    reqs = served_requests()
    nfac = sum(1 for r in reqs if isinstance(r, S.FactorSolve))
    srv = S.Server(device, slots=8, hbm_budget=120e9, rank_cap=256)
    t0 = time.perf_counter()
    out = srv.run(reqs)
    wall = time.perf_counter() - t0
    lat = srv.latencies()
    srv.close()
    return {"p50_s": lat["p50_s"], "p99_s": lat["p99_s"], "requests": len(out), "factorizations": nfac,
            "solves_on_resident_factors": len(out) - nfac, "wall_s": wall,
            "requests_per_s": len(out) / wall, "arrivals": "Poisson, mean gap 50 ms",
            "families": "random n=1024/2048; column-scaled kappa~1e10 n=2048/4096; kernel 1/(x-y) n=2048; "
                        "banded b=8 n=4096/8192; 1-64 right-hand sides",
            "slots": 8, "hbm_budget_gb": 120}


def reference_arm(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    inp = make_input(0)
    for _ in range(args.warmup):
        time_oracle(inp)
    t = 0.0
    for _ in range(args.steps):
        t += time_oracle(inp)
    value = args.steps / t
    cores = cpu_threads()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "n": N, "nmin": NMIN, "rank": K, "tol": TOL},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "one full factorization of the workload per step (numpy FP64 oracle)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def gpu_arm(args):
    import torch

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1809_10585_gb300 import binding as B
    from paper_1809_10585_gb300 import build as BUILD
    BUILD.build()

    nb = max(1, args.batch)
    inps = [make_input(sd) for sd in rank_seeds(rank, nb)]
    inp = inps[0]
    ctx = B.Context(local)
    stream = torch.cuda.Stream()
    ctx.set_stream(stream.cuda_stream)
    # cluster size of the QR/Jacobi kernels: the device maximum serves one matrix best; with
    # several matrices in flight smaller clusters keep more of them resident at once
    cmax = ctx.cluster
    ccl = args.cluster if args.cluster > 0 else (cmax if nb == 1 else min(cmax, BATCH_CLUSTER))
    ctx.cluster = ccl
    if args.cluster_large > 0:
        ctx.set_cluster_large(args.cluster_large)
    ctx.set_batch_group(args.group)
    mats = [B.Matrix(ctx, x, rank_cap=args.rank_cap) for x in inps]
    M = mats[0]
    for m in mats:
        m.snapshot()
    tuned = None
    if nb > 1 and args.cluster <= 0 and args.group_given is False:
        # launch shapes (cluster size, merged group size) chosen by timing this batch on this GPU
        with torch.cuda.stream(stream):
            tuned = B.autotune_batched(ctx, mats, TOL, 0.0, reps=2)
        ccl = ctx.cluster
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def factor_all():
        if nb == 1:
            M.qr_graph(TOL, 0.0)
        else:
            B.qr_batched(ctx, mats, TOL, 0.0, graph=True)

    # warm-up (the first call records the CUDA graph)
    with torch.cuda.stream(stream):
        for _ in range(max(args.warmup, 1)):
            factor_all()
    ctx.sync()
    for m in mats:
        st, anorm = m.status()
        if st != 0:
            raise RuntimeError(f"factorization status {st}")
    st, anorm = M.status()

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()

    clocks = ClockSampler(local)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    t_wall = time.perf_counter()
    with torch.cuda.stream(stream):
        for i in range(args.steps):
            flush.fill_(float(i))
            evs[i][0].record(stream)
            factor_all()
            evs[i][1].record(stream)
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall
    clk = clocks.stop()
    barrier()
    ms_steps = [a.elapsed_time(b) for a, b in evs]
    ms_total = float(sum(ms_steps))
    # the plain one-matrix-at-a-time path on the same GPU (first matrix of the batch)
    single = None
    if nb > 1:
        sev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        ctx.cluster = cmax
        with torch.cuda.stream(stream):
            M.qr_graph(TOL, 0.0)
            for i in range(args.steps):
                flush.fill_(float(i))
                sev[i][0].record(stream)
                M.qr_graph(TOL, 0.0)
                sev[i][1].record(stream)
        torch.cuda.synchronize()
        sms = sum(a.elapsed_time(b) for a, b in sev) / args.steps
        single = {"value": 1e3 / sms, "unit": UNIT, "ms_per_step": sms, "cluster": cmax}
        ctx.cluster = ccl
    ms_total = max_over_ranks(ms_total, "cuda")
    for m in mats:
        st, _ = m.status()
        if st != 0:
            raise RuntimeError(f"factorization status {st}")
    ms_per_step = ms_total / args.steps
    value = whole_job_rate(ws, nb, args.steps, ms_total / 1e3)

    # ---------------------------------------------------------------- end to end (host buffers)
    def pinned_like(a):
        t = torch.empty(a.shape[::-1], dtype=torch.float64, pin_memory=True)   # column-major storage
        t.numpy()[...] = np.asarray(a).T
        return t
    keep = []

    def pin_list(lst):
        out = []
        for a in lst:
            t = pinned_like(a)
            keep.append(t)
            out.append(t.numpy().T)      # Fortran-ordered view on pinned memory
        return out
    import workloads as W
    pinps = [W.HodlrInput(x.n, x.leaf_sizes, pin_list(x.leaves), pin_list(x.U12), pin_list(x.V12),
                          pin_list(x.U21), pin_list(x.V21), name=x.name) for x in inps]
    h2d = sum(a.nbytes for x in inps for lst in (x.leaves, x.U12, x.V12, x.U21, x.V21) for a in lst)
    # the factorization comes back compact: every factor at its stored rank, not the capacity
    out_bytes = sum(m.compact_bytes() for m in mats)
    host_outs = [torch.empty(m.storage_bytes(), dtype=torch.uint8, pin_memory=True).numpy() for m in mats]
    e2e_steps = max(1, min(args.steps, 10))

    def e2e_step():
        # pinned host -> device upload, factorization (the same CUDA graph as the device arm; its
        # restore copies the just-uploaded values), device -> host read of every factorization
        for m, p in zip(mats, pinps):
            m.upload(p)
            m.snapshot()
        factor_all()
        for m, h in zip(mats, host_outs):
            m.download_compact(h)
    with torch.cuda.stream(stream):
        e2e_step()
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    with torch.cuda.stream(stream):
        for _ in range(e2e_steps):
            e2e_step()
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_s = max_over_ranks(e2e_s, "cuda")
    e2e = {"value": whole_job_rate(ws, nb, e2e_steps, e2e_s), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
           "d2h_bytes_per_step": int(out_bytes), "steps": e2e_steps}

    # ---------------------------------------------------------------- roofline of the top kernel
    live = B.fp64_peak(local)
    rec = recorded_fp64_peak()
    if rec is not None:
        peak = rec[0]
        peak_source = f"{PEAK_RECORD}: DFMA throughput measured on GB300 by hodlr_fp64_peak (CUDA events)"
    else:
        peak = live["dfma"]
        peak_source = "DFMA throughput measured in this run by hodlr_fp64_peak (CUDA events)"
    prof = M.qr_profile(TOL, 0.0)
    flops_total = M.flops()["total"]
    top = max((k for k in prof if prof[k]["flops"] > 0), key=lambda k: prof[k]["ms"])
    p = prof[top]
    top_achieved = p["flops"] / (p["ms"] / 1e3) / 1e12 if p["ms"] > 0 else 0.0
    # the step is one CUDA-graph launch (nb factorizations, their kernels concurrent): its
    # algorithmic flops over its event-timed duration
    step_achieved = nb * flops_total / (ms_per_step / 1e3) / 1e12
    roofline = {"bound": "alu", "kernel": f"batched hQR graph ({nb} factorizations per launch)",
                "achieved": step_achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": step_achieved / peak, "traffic": None,
                "flops_per_launch": nb * flops_total, "ms_per_launch": ms_per_step,
                "peak_source": peak_source, "peak_live": live,
                "per_kernel": {
                    "note": "one factorization alone, kernels serialised on two streams, "
                            f"{ctx.cluster}-CTA clusters; per-launch durations by CUDA events",
                    "top": top, "top_achieved": top_achieved, "top_frac": top_achieved / peak,
                    "top_launches": p["launches"], "top_ms_per_launch": p["ms"] / max(1, p["launches"]),
                    "top_flops_per_launch": p["flops"] / max(1, p["launches"]),
                    "kind_ms": {k: round(v["ms"], 4) for k, v in prof.items()},
                    "kind_gflop": {k: round(v["flops"] / 1e9, 4) for k, v in prof.items()},
                    "kind_share": {k: round(v["ms"] / max(1e-9, sum(x["ms"] for x in prof.values())), 4)
                                   for k, v in prof.items()}}}
    # matrices of one structure share one merged schedule: a step launches one factorization's
    # kernels per group (each launch carrying the descriptors of every matrix of the group)
    grp = tuned["group"] if tuned else args.group
    groups = 1 if nb == 1 else (-(-nb // grp) if grp > 0 else 1)
    gpu_launches = sum(v["launches"] for v in prof.values()) * args.steps * groups

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": N, "nmin": NMIN, "rank": K, "col_scale_decades": DECADES,
                       "tol": TOL, "rank_cap": args.rank_cap, "batch": nb, "cluster": ccl,
                       "group": tuned["group"] if tuned else args.group,
                       "launch_shapes": "autotuned (hodlr_autotune_batched: cluster x group, best of 2 timed graphs "
                                        "each)" if tuned else "given",
                       "batching": "independent seeded matrices of the workload factored together: one merged "
                                   "launch schedule per group of matrices (each launch carries every matrix's "
                                   "descriptors), one CUDA graph per step",
                       "l2": "flushed (256 MiB write) between timed steps",
                       "parallelism": f"replicas x{ws}", "anorm": anorm},
            "effective_gflops": nb * flops_total / (ms_per_step / 1e3) / 1e9,
            "algorithmic_gflop_per_step": flops_total / 1e9,
            "wall_s_timed": t_wall, "clocks": clk, "e2e": e2e, "roofline": roofline,
            "single_matrix": single,
            "gpu_launches": gpu_launches}

    if rank == 0 and not args.no_served:
        line["served"] = served_leg(local)
    if rank == 0 and not args.no_cpu_baseline:
        t = time_oracle(inp)
        line["cpu_baseline"] = {"value": 1.0 / t, "unit": UNIT, "cores": cpu_threads(), "kind": "oracle",
                                "sample": "one full factorization of the same n=8192 workload"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def batch256_arm(args):
    """The cross-matrix batch workload: 256 independent matrices, n log-uniform in [2048, 32768]
    rounded to nmin 2^l, nmin in {128, 256}, off-diagonal ranks uniform in [5, 20], every second
    matrix column-scaled to condition ~1e10, tol 1e-12.  With ranks up to 20 the factors' ranks
    reach ~200 (rank capacity 256), and the 256 factorizations would need ~350 GB: a step factors
    them in `--waves` waves (default 2) of interleaved matrices, each wave's matrices uploaded into
    device matrices reused across waves (matrices of one partition share them), then factored by
    one batched call (merged launch schedules per group of one partition).  `value` times the
    factorizations on the device (CUDA events around each wave); `e2e` adds the uploads and the
    compact downloads of the factorizations."""
    import collections
    import torch
    from paper_1809_10585_gb300 import binding as B
    from paper_1809_10585_gb300 import build as BUILD
    import workloads as W
    BUILD.build()
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    count = args.batch if args.batch != 64 else 256
    kc = args.rank_cap if args.rank_cap != RANK_CAP else 256
    waves = max(1, args.waves)
    t_gen = time.perf_counter()
    inps = W.batched_family(count=count, seed0=rank * count)
    t_gen = time.perf_counter() - t_gen
    ctx = B.Context(local)
    stream = torch.cuda.Stream()
    ctx.set_stream(stream.cuda_stream)
    cmax = ctx.cluster
    ctx.cluster = min(cmax, BATCH_CLUSTER) if args.cluster <= 0 else args.cluster
    ctx.set_cluster_large(cmax if args.cluster_large < 0 else args.cluster_large)
    ctx.set_batch_group(args.group)
    key = lambda x: (x.n, tuple(x.leaf_sizes))
    wave_idx = [[i for i in range(count) if i % waves == w] for w in range(waves)]
    need = collections.Counter()
    for idx in wave_idx:
        for k, v in collections.Counter(key(inps[i]) for i in idx).items():
            need[k] = max(need[k], v)
    pool = {}
    for i, x in enumerate(inps):
        k = key(x)
        if len(pool.setdefault(k, [])) < need[k]:
            pool[k].append(B.Matrix(ctx, x, rank_cap=kc))
    assign = []                      # per wave: the device matrix of each of its inputs
    for idx in wave_idx:
        used = collections.Counter()
        row = []
        for i in idx:
            k = key(inps[i])
            row.append(pool[k][used[k]])
            used[k] += 1
        assign.append(row)
    out_host = {}
    moved = [0]

    def run_wave(w, ev=None, download=False):
        mats = assign[w]
        for m, i in zip(mats, wave_idx[w]):
            m.upload(inps[i])
        with torch.cuda.stream(stream):
            if ev:
                ev[0].record(stream)
            B.qr_batched(ctx, mats, TOL, 0.0)
            if ev:
                ev[1].record(stream)
        ctx.sync()
        f = 0.0
        moved[0] = 0
        for m, i in zip(mats, wave_idx[w]):
            st, _ = m.status()
            if st != 0:
                raise RuntimeError(f"factorization status {st} for matrix {i} (n = {inps[i].n})")
            f += m.flops()["total"]
            if download:
                nb = m.compact_bytes()
                buf = out_host.get(id(m))
                if buf is None or buf.nbytes < nb:
                    buf = out_host[id(m)] = torch.empty(m.storage_bytes(), dtype=torch.uint8, pin_memory=True).numpy()
                m.download_compact(buf)
                moved[0] += nb
        return f

    for _ in range(max(args.warmup, 1)):
        for w in range(waves):
            run_wave(w)
    mem = ctx.memory_used()
    clocks = ClockSampler(local)
    evs = []
    flops = 0.0
    down = 0
    torch.cuda.synchronize()
    clocks.start()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for w in range(waves):
            ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
            flops += run_wave(w, ev, download=True)
            down += moved[0]
            evs.append(ev)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in evs), "cuda")
    ms_per_step = ms / args.steps
    flops_per_step = flops / args.steps
    value = whole_job_rate(ws, count, args.steps, ms / 1e3)
    rec = recorded_fp64_peak()
    peak = rec[0] if rec else B.fp64_peak(local)["dfma"]
    achieved = flops_per_step / (ms_per_step / 1e3) / 1e12
    up = sum(a.nbytes for x in inps for lst in (x.leaves, x.U12, x.V12, x.U21, x.V21) for a in lst)
    down = down // max(1, args.steps)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "batch256_n2048-32768_nmin128-256_k5-20_half-colscaled1e-10_tol1e-12",
                       "matrices": count, "waves": waves, "device_matrices": sum(need.values()),
                       "n_min": min(x.n for x in inps), "n_max": max(x.n for x in inps),
                       "n_total": sum(x.n for x in inps), "rank_cap": kc, "cluster": ctx.cluster,
                       "cluster_large": cmax if args.cluster_large < 0 else args.cluster_large,
                       "group": args.group, "tol": TOL,
                       "l2": "inputs larger than L2 (each wave re-uploads its matrices before its timed region)",
                       "device_bytes": mem, "host_generation_s": t_gen},
            "effective_gflops": flops_per_step / (ms_per_step / 1e3) / 1e9,
            "algorithmic_gflop_per_step": flops_per_step / 1e9, "clocks": clk,
            "e2e": {"value": whole_job_rate(ws, count, args.steps, wall), "unit": UNIT,
                    "h2d_bytes_per_step": int(up), "d2h_bytes_per_step": int(down),
                    "note": "uploads of every wave, factorizations and compact downloads, host wall clock"},
            "roofline": {"bound": "alu", "kernel": f"batched hQR ({count} factorizations per step in {waves} waves)",
                         "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                         "traffic": None, "peak_source": PEAK_RECORD if rec else "measured in this run"}}
    if rank == 0 and not args.no_cpu_baseline:
        # a bounded sample (about half a minute of host work): matrices of n <= 8192 spread over
        # the batch's sizes and ranks
        small = [i for i in sorted(range(count), key=lambda i: inps[i].n) if inps[i].n <= 8192]
        sample = small[:: max(1, len(small) // 5)][:5]
        t = 0.0
        n_flops = 0.0
        import oracle.core as O
        for i in sample:
            O.reset_counters()
            t += time_oracle(inps[i])
            n_flops += sum(O.FLOPS.values())
        rate = (n_flops / t) / (flops_per_step / count) if t > 0 else 0.0
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": cpu_threads(), "kind": "oracle",
                                "sample": f"{len(sample)} matrices of the batch spread over n "
                                          f"({min(inps[i].n for i in sample)}..{max(inps[i].n for i in sample)}), "
                                          "timed whole; rate scaled by algorithmic flops to the batch's mean"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def single_arm(args):
    """One matrix of the n = 1024 workload (nmin 128, rank 5, tol 1e-10) or of the kernel-generated
    n = 65536 workload (A_ij = 1/(x_i - y_j) + n delta_ij, off-diagonal blocks compressed at
    1e-12, tol 1e-12), factored by the plain one-matrix path (one CUDA graph per factorization,
    the device's largest cluster size), with the oracle on the host cores beside it."""
    import torch
    import workloads as W
    from paper_1809_10585_gb300 import binding as B
    from paper_1809_10585_gb300 import build as BUILD
    BUILD.build()
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if args.workload == "n1024":
        inp, tol, name = W.config0(seed=rank), 1e-10, "hodlr_qr_n1024_nmin128_k5_tol1e-10"
        kc = 64
    else:
        t = time.perf_counter()
        inp = W.kernel_hodlr(65536, 256, 1e-12, seed=rank, device="cuda")
        t_gen = time.perf_counter() - t
        tol, name, kc = 1e-12, "hodlr_qr_n65536_nmin256_kernel_1/(x-y)_tol1e-12", 256
        torch.cuda.empty_cache()
    ctx = B.Context(local)
    stream = torch.cuda.Stream()
    ctx.set_stream(stream.cuda_stream)
    M = B.Matrix(ctx, inp, rank_cap=kc)
    M.snapshot()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    with torch.cuda.stream(stream):
        for _ in range(max(args.warmup, 1)):
            M.qr_graph(tol, 0.0)
    ctx.sync()
    st, anorm = M.status()
    if st != 0:
        raise RuntimeError(f"factorization status {st}")
    flops = M.flops()["total"]
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    torch.cuda.synchronize()
    clocks.start()
    with torch.cuda.stream(stream):
        for i in range(args.steps):
            flush.fill_(float(i))
            evs[i][0].record(stream)
            M.qr_graph(tol, 0.0)
            evs[i][1].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in evs), "cuda") / args.steps
    rec = recorded_fp64_peak()
    peak = rec[0] if rec else B.fp64_peak(local)["dfma"]
    achieved = flops / (ms / 1e3) / 1e12
    stats = M.stats()
    line = {"metric": METRIC, "value": 1e3 / ms * ws, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": name, "n": inp.n, "nmin": max(inp.leaf_sizes), "tol": tol, "rank_cap": kc,
                       "cluster": ctx.cluster, "anorm": anorm, "max_rank_Y": stats["max_rank_Y"],
                       "max_rank_T": stats["max_rank_T"], "max_rank_R": stats["max_rank_R"],
                       "l2": "flushed (256 MiB write) between timed steps"},
            "effective_gflops": flops / (ms / 1e3) / 1e9, "algorithmic_gflop_per_step": flops / 1e9,
            "clocks": clk,
            "roofline": {"bound": "alu", "kernel": "one hQR factorization (CUDA graph)", "achieved": achieved,
                         "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
                         "peak_source": PEAK_RECORD if rec else "measured in this run"}}
    if args.workload == "n65536":
        line["config"]["host_generation_s"] = t_gen
    if rank == 0 and not args.no_cpu_baseline:
        t = time_oracle(inp)
        line["cpu_baseline"] = {"value": 1.0 / t, "unit": UNIT, "cores": cpu_threads(), "kind": "oracle",
                                "sample": f"one full factorization of the same n={inp.n} matrix"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def served_sweep_requests(rate, count, pool, seed):
    """A Poisson stream at `rate` requests/s: factorize+solve requests on matrices drawn from the
    pool (each request factors its matrix anew), 1-64 right-hand sides N(0,1); a third are repeat
    solves on factors kept resident by an earlier request."""
    import workloads as W
    from paper_1809_10585_gb300 import server as S
    rng = np.random.default_rng(seed)
    reqs, kept, t = [], [], 0.0
    for i in range(count):
        t += float(rng.exponential(1.0 / rate))
        nrhs = int(rng.integers(1, 65))
        if kept and rng.uniform() < 1.0 / 3.0:
            key, n = kept[int(rng.integers(len(kept)))]
            reqs.append(S.Solve(key, W.rhs(n, nrhs, seed=seed + 1000 + i), arrival=t))
            continue
        inp = pool[int(rng.integers(len(pool)))]
        keep = bool(rng.uniform() < 0.5)
        key = f"r{i}" if keep else None
        reqs.append(S.FactorSolve(inp, W.rhs(inp.n, nrhs, seed=seed + 2000 + i), TOL, keep, key, arrival=t))
        if keep:
            kept.append((key, inp.n))
    return reqs


def served_arm(args):
    """The served factorize+solve stream at the shape of the serving workload: Poisson arrivals
    of requests on matrices of the random (rank 5), column-scaled (rank 10, condition ~1e10),
    kernel 1/(x - y) and symmetric banded (b = 8) families with n log-uniform over
    {4096, ..., 131072}; 1-64 right-hand sides; factors kept resident for repeat solves; HBM
    admission budget 120 GB.  The arrival rate is swept up to saturation; p50/p99 latency and
    throughput are reported per rate."""
    import torch
    import workloads as W
    from paper_1809_10585_gb300 import build as BUILD
    from paper_1809_10585_gb300 import server as S
    BUILD.build()
    ws, rank, local = dist_env()
    if rank != 0:
        return 0
    torch.cuda.set_device(local)
    rng = np.random.default_rng(777)
    sizes = [4096 << i for i in range(6)]                      # 4096 ... 131072
    pool, t_gen = [], time.perf_counter()
    for i in range(args.served_pool):
        n = int(sizes[int(rng.integers(len(sizes)))])
        fam = i % 4
        if fam == 0:
            pool.append(W.random_hodlr(n, 256, 5, seed=i))
        elif fam == 1:
            pool.append(W.scaled_config1(n, 256, 10, seed=i, decades=10.0))
        elif fam == 2:
            pool.append(W.kernel_hodlr(n, 256, 1e-12, seed=i, device="cuda"))
        else:
            pool.append(W.banded_hodlr(n, 8, 256, seed=i))
    t_gen = time.perf_counter() - t_gen
    torch.cuda.empty_cache()
    rates = [float(x) for x in args.served_rates.split(",")]
    points = []
    clocks = ClockSampler(local)
    clocks.start()
    for k, rate in enumerate(rates):
        reqs = served_sweep_requests(rate, args.served_requests, pool, seed=99 + k)
        srv = S.Server(local, slots=8, hbm_budget=120e9, rank_cap=args.rank_cap)
        t0 = time.perf_counter()
        out = srv.run(reqs)
        wall = time.perf_counter() - t0
        lat = srv.latencies()
        srv.close()
        nfac = sum(1 for r in reqs if isinstance(r, S.FactorSolve))
        points.append({"rate_per_s": rate, "requests": len(out), "factorizations": nfac,
                       "p50_s": lat["p50_s"], "p99_s": lat["p99_s"], "wall_s": wall,
                       "requests_per_s": len(out) / wall, "factorizations_per_s": nfac / wall,
                       "max_running": srv.max_running})
    clk = clocks.stop()
    best = max(points, key=lambda p: p["requests_per_s"])
    line = {"metric": "served factorize+solve requests/s at saturation (FP64, tol 1e-12); p50/p99 per rate",
            "value": best["requests_per_s"], "unit": "requests/s", "n_gpus": 1, "steps": len(rates),
            "warmup": 0, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "served_n4096-131072_random-colscaled-kernel-banded_tol1e-12",
                       "pool": [{"n": x.n, "family": ["random k5", "colscaled k10", "kernel", "banded b8"][i % 4]}
                                for i, x in enumerate(pool)],
                       "slots": 8, "hbm_budget_gb": 120, "rank_cap": args.rank_cap,
                       "arrivals": "Poisson, rates swept", "host_generation_s": t_gen},
            "points": points, "clocks": clk}
    print(json.dumps(line), flush=True)
    return 0


def peaks_arm(args):
    """FP64 DFMA and DMMA (mma.sync.m8n8k4) throughput of this GPU, with the SM clocks sampled
    while the microbenchmark runs: the record behind the roofline denominator."""
    import torch
    from paper_1809_10585_gb300 import binding as B
    from paper_1809_10585_gb300 import build as BUILD
    BUILD.build()
    _, _, local = dist_env()
    torch.cuda.set_device(local)
    B.fp64_peak(local, iters=200, reps=1)            # warm-up
    clocks = ClockSampler(local)
    clocks.start()
    runs = [B.fp64_peak(local, iters=4000, reps=5) for _ in range(3)]
    clk = clocks.stop()
    best = {k: max(r[k] for r in runs) for k in ("dfma", "dmma")}
    line = {"fp64_peak": True, "dfma_tflops": best["dfma"], "dmma_tflops": best["dmma"],
            "runs": runs, "clocks": clk, "gpu": torch.cuda.get_device_name(local),
            "sms": torch.cuda.get_device_properties(local).multi_processor_count,
            "method": "hodlr_fp64_peak: 4 CTAs x 256 threads per SM, 8 independent chains per thread "
                      "(DFMA) or per warp (mma.sync.m8n8k4.f64), best of 5 event-timed launches, 3 runs"}
    print(json.dumps(line), flush=True)
    return 0


def rect_arm(args):
    """Example 6.2 of the paper (Sec. 6): the permuted QR of a random 8000 x 4000 rectangular HODLR
    matrix (n_min = 250, rank-one off-diagonal blocks, eps = 1e-10) as the paper evaluates it, a
    dense permuted Householder QR on the device followed by the compression of Y, T and R into the
    HODLR formats of Fig. 6.3 (hodlr_rect_qr).  The matrix is resident on the device; a step is one
    call.  The oracle (numpy) runs beside it on a 4000 x 2000 sample of the same family."""
    import torch
    import oracle.core as O
    import oracle.rect as OR
    import workloads as W
    from paper_1809_10585_gb300 import binding as B
    from paper_1809_10585_gb300 import build as BUILD
    BUILD.build()
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    m, n, nmin, k, tol = 8000, 4000, 250, 1, 1e-10
    inp = W.random_rect_hodlr(m, n, nmin, k, seed=rank)
    A = W.rect_to_dense(inp)
    ctx = B.Context(local)
    stream = torch.cuda.Stream()
    ctx.set_stream(stream.cuda_stream)
    At = torch.from_numpy(np.ascontiguousarray(A.T)).to("cuda")            # column-major m x n
    out = None
    for _ in range(max(args.warmup, 1)):
        if out:
            for h in out[:3]:
                h.free()
        out = B.rect_qr(ctx, inp.m_sizes, inp.n_sizes, At.data_ptr(), m, tol, rank_cap=64, seed=3)
    Yh, Th, Rh, anorm, rc = out
    ranks = {nm: int(max(h.ranks()[0].max(), h.ranks()[1].max())) for nm, h in (("Y", Yh), ("T", Th), ("R", Rh))}
    A_h = OR.compress(A, inp.m_sizes, inp.n_sizes, tol * anorm) if rank == 0 else None
    mem = ({"Y_and_T": (Yh.storage() + Th.storage()) / A_h.storage(), "R": Rh.storage() / A_h.storage()}
           if A_h is not None else None)
    for h in (Yh, Th, Rh):
        h.free()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    torch.cuda.synchronize()
    clocks.start()
    with torch.cuda.stream(stream):
        for i in range(args.steps):
            flush.fill_(float(i))
            evs[i][0].record(stream)
            hs = B.rect_qr(ctx, inp.m_sizes, inp.n_sizes, At.data_ptr(), m, tol, rank_cap=64, seed=3)
            evs[i][1].record(stream)
            torch.cuda.synchronize()
            for h in hs[:3]:
                h.free()
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in evs), "cuda") / args.steps
    # end to end: pinned upload of A, the factorization, and the ranks of the three factors read back
    pinned = torch.from_numpy(np.ascontiguousarray(A.T)).pin_memory()
    Ad = torch.empty_like(At)
    e2e_ms = []
    for i in range(max(2, min(args.steps, 5))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            Ad.copy_(pinned, non_blocking=True)
        stream.synchronize()
        hs = B.rect_qr(ctx, inp.m_sizes, inp.n_sizes, Ad.data_ptr(), m, tol, rank_cap=64, seed=3)
        _ = [h.ranks() for h in hs[:3]]
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
        for h in hs[:3]:
            h.free()
    e2e = float(np.median(e2e_ms))
    flops = float(O.dense_qr_flops(m, n))
    rec = recorded_fp64_peak()
    peak = rec[0] if rec else B.fp64_peak(local)["dfma"]
    achieved = flops / (ms / 1e3) / 1e12
    line = {"metric": "rectangular HODLR permuted QRs/s (FP64, Sec. 6, Example 6.2, eps 1e-10)",
            "value": 1e3 / ms * ws, "unit": "factorizations/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"rect_m{m}_n{n}_nmin{nmin}_k{k}_tol{tol:g}", "m": m, "n": n, "nmin": nmin,
                       "leaves": len(inp.n_sizes), "rank": k, "tol": tol, "anorm": anorm, "rank_cap": 64,
                       "max_rank": ranks, "memory_vs_A": mem,
                       "l2": "flushed (256 MiB write) between timed steps; inputs (256 MB) larger than L2"},
            "clocks": clk,
            "e2e": {"value": 1e3 / e2e * ws, "unit": "factorizations/s", "h2d_bytes_per_step": int(A.nbytes),
                    "d2h_bytes_per_step": int(4 * 3 * 2 * (len(inp.n_sizes) - 1))},
            "roofline": {"bound": "alu", "kernel": "hodlr_rect_qr (dense permuted QR + compression)",
                         "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                         "traffic": None, "flops_per_launch": flops,
                         "flops_note": "algorithmic flops of the dense Householder QR with T (2mn^2 - 2n^3/3 + "
                                       "mn^2 - n^3/3); the compression is not counted",
                         "peak_source": PEAK_RECORD if rec else "measured in this run"}}
    if rank == 0 and not args.no_cpu_baseline:
        smp = W.random_rect_hodlr(4000, 2000, 250, k, seed=0)
        As = W.rect_to_dense(smp)
        t0 = time.perf_counter()
        OR.rect_qr(As, smp.m_sizes, smp.n_sizes, tol)
        ts = time.perf_counter() - t0
        scale = O.dense_qr_flops(4000, 2000) / flops
        line["cpu_baseline"] = {"value": scale / ts, "unit": "factorizations/s", "cores": cpu_threads(),
                                "kind": "oracle",
                                "sample": f"one 4000 x 2000 matrix of the same family ({ts:.1f} s), scaled to the "
                                          f"8000 x 4000 size by the dense QR flop ratio {scale:.3f}"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batch", type=int, default=64,
                    help="matrices of the workload factored concurrently per step (cross-matrix batching)")
    ap.add_argument("--rank-cap", type=int, default=RANK_CAP,
                    help="rank capacity of the stored factors (a factorization that needs more fails)")
    ap.add_argument("--no-served", action="store_true",
                    help="skip the served request stream (p50/p99 latency)")
    ap.add_argument("--group", type=int, default=-1,
                    help="most matrices per merged launch schedule (0: no limit; default: 1 for the n = 8192 "
                         "workload, 4 for the 256-matrix batch)")
    ap.add_argument("--waves", type=int, default=2, help="waves per step of the 256-matrix batch")
    ap.add_argument("--cluster-large", type=int, default=-1,
                    help="cluster size for QRs / Jacobi cores that do not fit the cluster's shared memory "
                         "(0: none; default: none for the n = 8192 workload, the device maximum otherwise)")
    ap.add_argument("--served-requests", type=int, default=24, help="requests per rate of the served sweep")
    ap.add_argument("--served-rates", default="0.5,2,8,32", help="arrival rates (requests/s) of the served sweep")
    ap.add_argument("--served-pool", type=int, default=12, help="distinct matrices the served sweep draws from")
    ap.add_argument("--workload", default="n8192",
                    choices=["n8192", "batch256", "served", "n1024", "n65536", "rect"],
                    help="n8192: the ill-conditioned n = 8192 workload (default); batch256: 256 matrices of "
                         "log-uniform n in [2048, 32768]")
    ap.add_argument("--peaks", action="store_true",
                    help="measure the FP64 DFMA / DMMA throughput of the GPU and exit")
    ap.add_argument("--cluster", type=int, default=0,
                    help="CTAs per thread-block cluster of the QR/Jacobi kernels (0: automatic)")
    args = ap.parse_args()
    args.group_given = args.group >= 0
    if args.group < 0:
        args.group = 4 if args.workload == "batch256" else 1
    if args.impl == "reference":
        return reference_arm(args)
    if args.peaks:
        return peaks_arm(args)
    if args.workload == "batch256":
        return batch256_arm(args)
    if args.workload == "served":
        return served_arm(args)
    if args.workload in ("n1024", "n65536"):
        return single_arm(args)
    if args.workload == "rect":
        return rect_arm(args)
    return gpu_arm(args)


if __name__ == "__main__":
    sys.exit(main())

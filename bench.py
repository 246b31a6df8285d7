#!/usr/bin/env python3
"""Benchmark of the HMM hot path on one GB300 (or N GPUs, one process each).

Workload (the paper-shaped "plain method at GPU scale" configuration): N = 16
states, 4096 sequences of T = 2000 float32 observations, one Gamma-emission
model with Dirichlet(1) transition rows, synthetic seeded data.  One step =
one Baum-Welch iteration (fused E-step: emissions, forward, backward,
occupancies, xi and sufficient statistics; fixed-order float64 reductions;
M-step with the Gamma Newton-Raphson) followed by one Viterbi decode of the
whole batch with the updated model.  The metric counts N^2 * sum(T) cell
updates for the iteration and again for the decode.

Timing: CUDA events on the launching stream around every step, W untimed
warm-up steps, the L2 cache flushed (a 256 MiB write) before each timed
step outside the events, GPU clocks sampled with nvidia-smi during the timed
steps.  The dominant kernel (the fused E-step) is timed separately by the
library's event hooks on its own stream for the roofline entry.

--impl reference times the FP64 CPU oracle (oracle/) on a bounded sample of
the same workload, as the reference arm of a comparison.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_STATES, N_SEQ, T_LEN = 16, 4096, 2000
METRIC = "Baum-Welch N^2 T cell-updates/s (EM iteration + Viterbi decode)"
UNIT = "cell-updates/s"


def args_parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=300)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--family", default="gamma",
                   choices=["gamma", "student_t", "gauss", "poisson", "vonmises", "lognormal", "exponential",
                            "rayleigh", "uniform", "chisq", "pareto"])
    p.add_argument("--workload", choices=["scale", "batching", "precision", "serving", "discrete"], default="scale",
                   help="scale: N=16 x 4096 x 2000 (the bench line); batching: 100k ragged "
                        "sequences, N=8, 1024 mixed-family models")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-plain", action="store_true")
    p.add_argument("--estep-lanes", type=int, default=0)
    p.add_argument("--viterbi-lanes", type=int, default=0)
    p.add_argument("--quick", action="store_true", help="small case for profiling runs")
    p.add_argument("--rate", type=float, default=2000.0, help="serving: Poisson arrival rate (requests/s)")
    p.add_argument("--requests", type=int, default=1000, help="serving: number of requests")
    p.add_argument("--t-max", type=int, default=100000, help="serving: longest sequence")
    p.add_argument("--slots", type=int, default=32, help="serving: concurrent batches")
    p.add_argument("--no-extras", action="store_true",
                   help="only the headline line (no batching / precision / serving sub-measurements)")
    p.add_argument("--serve-rate", type=float, default=20.0, help="extras: the sustained serving rate")
    p.add_argument("--serve-requests", type=int, default=150, help="extras: requests per serving run")
    return p.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def workload(args, rank):
    from paper_2605_29208_gb300 import synth
    if args.workload == "batching":
        # --quick: 10k sequences and 128 models of the same mix (profiling runs)
        kw = dict(n_seq=10_000, n_models=128) if args.quick else {}
        truths, inits, values, offsets, mid = synth.batching_workload(seed=synth.MASTER_SEED + 2 + 1000 * rank, **kw)
        return truths, inits, values, offsets, mid
    n_seq, T = (256, 500) if args.quick else (N_SEQ, T_LEN)
    # weak scaling: every rank holds its own full-size batch (seed per rank)
    return synth.scale_workload(args.family, n_seq=n_seq, T=T, N=N_STATES,
                                seed=synth.MASTER_SEED + 1 + 1000 * rank)


def cells(offsets, N):
    return float(N * N) * float(offsets[-1])


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


# ---------------------------------------------------------------- CPU side
def _as_list(init):
    return init if isinstance(init, list) else [init]


def oracle_step_sample(init, values, offsets, mid, n_sample):
    """One EM iteration and one Viterbi decode of the first n_sample
    sequences with the oracle; returns (seconds, cell updates)."""
    from oracle import hmm_oracle as O
    models = [O.Model(m["family"], m["pi"].copy(), m["A"].copy(),
                      {k: v.copy() for k, v in m["params"].items()}) for m in _as_list(init)]
    sub_off = offsets[:n_sample + 1]
    sub_vals = values[:sub_off[-1]]
    sub_mid = mid[:n_sample]
    t0 = time.perf_counter()
    new, _ = O.em_iteration(models, sub_vals, sub_off, sub_mid)
    for s in range(n_sample):
        O.viterbi(new[sub_mid[s]], sub_vals[sub_off[s]:sub_off[s + 1]])
    dt = time.perf_counter() - t0
    return dt, 2.0 * cells(sub_off, len(models[0].pi))


def cpu_baseline(init, values, offsets, mid, target_s=12.0):
    n = 4
    dt, c = oracle_step_sample(init, values, offsets, mid, n)
    n2 = int(max(4, min(len(offsets) - 1, n * target_s / max(dt, 1e-3))))
    dt, c = oracle_step_sample(init, values, offsets, mid, n2)
    return dict(value=c / dt, unit=UNIT, cores=1, kind="oracle",
                sample=f"first {n2} of {len(offsets) - 1} sequences ({int(offsets[n2])} time steps, "
                       f"N={len(_as_list(init)[0]['pi'])}), one EM iteration + one Viterbi decode, "
                       f"numpy float64 single thread, {dt:.1f} s")


def _oracle_fb_chunk(job):
    """Worker: the oracle's forward-backward of a list of sequences."""
    from oracle import hmm_oracle as O
    m, seqs = job
    om = O.Model(m["family"], m["pi"], m["A"], m["params"])
    return [(fb["logL"], fb["gamma"], fb["xi_sum"]) for fb in (O.forward_backward(om, y) for y in seqs)]


def _oracle_vit_chunk(job):
    """Worker: the oracle's Viterbi decode of a list of sequences."""
    from oracle import hmm_oracle as O
    m, seqs = job
    om = O.Model(m["family"], m["pi"], m["A"], m["params"])
    return [O.viterbi(om, y)[1] for y in seqs]


def _model_dict(o):
    return dict(family=o.family, pi=o.pi, A=o.A, params=o.params)


def oracle_step_pool(pool, n_proc, init, values, offsets, n_sample):
    """One EM iteration and one Viterbi decode of the first n_sample sequences
    (one model) with the oracle's own functions, the sequences of each E-step
    and decode spread over n_proc worker processes; the pooled M-step runs in
    this process.  Returns (seconds, cell updates)."""
    from oracle import hmm_oracle as O
    m = _as_list(init)[0]
    seqs = [values[offsets[s]:offsets[s + 1]] for s in range(n_sample)]
    parts = [seqs[i::n_proc] for i in range(n_proc)]
    t0 = time.perf_counter()
    res = [r for part in pool.map(_oracle_fb_chunk, [(m, p) for p in parts]) for r in part]
    om = O.Model(m["family"], m["pi"].copy(), m["A"].copy(), {k: v.copy() for k, v in m["params"].items()})
    W = np.concatenate([g for _, g, _ in res])
    Y = np.concatenate([p for part in parts for p in part])
    xi = sum(x for _, _, x in res)
    g1 = sum(g[0] for _, g, _ in res)
    new, _ = O.mstep_emission(om, W, Y)
    new.pi, new.A = O.mstep_transitions(om, xi, g1, n_sample)
    nd = _model_dict(new)
    pool.map(_oracle_vit_chunk, [(nd, p) for p in parts])
    dt = time.perf_counter() - t0
    return dt, 2.0 * cells(offsets[:n_sample + 1], len(m["pi"]))


def cpu_baseline_all_cores(init, values, offsets, target_s=15.0):
    """The oracle on every host core: a spawned process pool over sequences
    (each worker single-threaded), on a bounded prefix of the workload."""
    import multiprocessing as mp
    n_proc = host_cores()
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"
    S = len(offsets) - 1
    with mp.get_context("spawn").Pool(n_proc) as pool:
        n = min(S, 2 * n_proc)
        dt, _ = oracle_step_pool(pool, n_proc, init, values, offsets, n)
        n2 = int(max(n_proc, min(S, n * target_s / max(dt, 1e-3))))
        dt, c = oracle_step_pool(pool, n_proc, init, values, offsets, n2)
    return dict(value=c / dt, unit=UNIT, cores=n_proc, kind="oracle",
                sample=f"first {n2} of {S} sequences ({int(offsets[n2])} time steps), one EM iteration + one "
                       f"Viterbi decode, numpy float64, {n_proc} spawned worker processes over sequences "
                       f"(M-step in the parent), {dt:.1f} s")


def arm_config(args, NS, S, offsets, n_models, ws, c_step):
    """The workload's `config` entry (both arms print the same one)."""
    return dict(workload=(f"{args.family} HMM, N={NS} states, {S} sequences x "
                          f"T={int(offsets[1] - offsets[0])}, one EM iteration + Viterbi"
                          if args.workload == "scale" else
                          f"batching: {S} ragged sequences (sum T = {int(offsets[-1])}), "
                          f"N={NS}, {n_models} mixed-family models, one EM iteration + Viterbi"),
                family=args.family if args.workload == "scale" else "mixed",
                n_states=NS, n_seq_per_gpu=S, total_T=int(offsets[-1]),
                seq_len=int(offsets[1] - offsets[0]) if args.workload == "scale" else "ragged",
                global_batch=S * ws,
                parallelism=f"dp{ws}" if ws > 1 else "single GPU",
                cell_updates_per_step=c_step,
                l2="flushed before every timed step (256 MiB write, outside the events)")


def run_reference(args):
    """The reference arm: the FP64 oracle as it stands on the host's cores (a
    spawned pool over sequences, one single-threaded worker per core, the
    pooled M-step in the parent), each step a bounded sample of the
    workload, the rate scaled to cell updates per second."""
    import multiprocessing as mp
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    truth, init, values, offsets, mid = workload(args, 0)
    inits = init if isinstance(init, list) else [init]
    NS = len(inits[0]["pi"])
    S = len(offsets) - 1
    n_proc = host_cores()
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"
    single_model = len(inits) == 1
    n_sample = min(S, (2 if args.quick else 8) * n_proc)
    times, cs = [], 0.0
    with mp.get_context("spawn").Pool(n_proc) as pool:
        def one_step(n):
            if single_model:
                return oracle_step_pool(pool, n_proc, init, values, offsets, n)
            return oracle_step_sample(init, values, offsets, mid, max(2, n // n_proc))
        for _ in range(args.warmup):
            one_step(min(S, n_proc))
        for _ in range(args.steps):
            dt, c = one_step(n_sample)
            times.append(dt)
            cs = c
    ms = 1e3 * float(np.mean(times))
    value = cs / (ms / 1e3)
    cores = n_proc if single_model else 1
    line = dict(impl="reference", metric=METRIC, value=value, unit=UNIT, n_gpus=args.gpus,
                steps=args.steps, warmup=args.warmup, ms_per_step=ms, higher_is_better=True,
                scaling="weak", vs_baseline=None, dtype="f64", data="synthetic",
                config=arm_config(args, NS, S, offsets, len(inits), ws, 2.0 * cells(offsets, NS)),
                cpu_baseline=dict(value=value, unit=UNIT, cores=cores, kind="oracle",
                                  sample=(f"{n_sample} sequences of the workload per step over {n_proc} spawned "
                                          f"single-threaded workers (numpy float64), the pooled M-step in the "
                                          f"parent; rate scaled to cell updates per second" if single_model else
                                          "a few sequences per step, numpy float64, one thread")),
                e2e=dict(value=value, unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- GPU side
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join(ROOT, "bench_logs", f"clocks_rank{index}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.fh,
                stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        try:
            rows = [r.split(",") for r in open(self.path).read().strip().splitlines()]
        except Exception:
            return None
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[0]))
                mx.append(float(r[1]))
                for i, n in enumerate(names):
                    if r[4 + i].strip().lower() == "active":
                        reasons.add(n)
            except Exception:
                continue
        if not sm:
            return None
        return dict(sm_mhz=statistics.median(sm), sm_max_mhz=max(mx), samples=len(sm),
                    reasons=sorted(reasons))


def profiled_traffic(name, sources):
    """DRAM bytes per launch from the committed ncu summary of a kernel, or
    None when the kernel's sources changed since that capture."""
    import hashlib
    import re
    try:
        txt = open(os.path.join(ROOT, "profiles", name)).read()
        h = hashlib.sha256()
        for f in sources:
            h.update(open(os.path.join(ROOT, "paper_2605_29208_gb300", "csrc", f), "rb").read())
        sha = re.search(r"kernel_source_sha256_16: ([0-9a-f]+)", txt).group(1)
        if sha != h.hexdigest()[:16]:
            return None
        return int(re.search(r"traffic_bytes_per_launch: (\d+)", txt).group(1))
    except Exception:
        return None


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def run_ours(args, emit=True):
    import torch
    import paper_2605_29208_gb300 as H
    from paper_2605_29208_gb300 import _lib, parallel

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    truth, init, values, offsets, mid = workload(args, rank)
    ctx = H.Context(local)
    if args.estep_lanes:
        ctx.set_option(_lib.OPT_ESTEP_LANES, args.estep_lanes)
    if args.viterbi_lanes:
        ctx.set_option(_lib.OPT_VITERBI_LANES, args.viterbi_lanes)
    models = _as_list(init)
    NS = len(models[0]["pi"])
    model = H.Model(ctx, models)
    batch = H.Batch(values, offsets, mid).make_plan(ctx, model)
    tuned_ms = batch.autotune(ctx, model) if not (args.estep_lanes or args.viterbi_lanes) else None
    stats = H.Stats(ctx, model)
    dev = batch.values.device
    S = batch.n_seq
    ll = torch.empty(S, dtype=torch.float64, device=dev)
    path = torch.empty(batch.total_T, dtype=torch.int32, device=dev)
    score = torch.empty(S, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    flush_buf = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    opts = H.mstep_opts()
    b = batch.c()
    L = ctx.lib
    import ctypes as C
    sp = C.c_void_p(stream.cuda_stream)

    # data parallel: the library combines its records across ranks through
    # this all-reduce (after the E-step, and per Newton data pass)
    exchange = parallel.Exchange(stats) if dist is not None else None

    def step():
        H.check(L.hmm_estep_stats(ctx.h, model.h, C.byref(b), stats.h, C.c_void_p(ll.data_ptr()), sp))
        H.check(L.hmm_mstep(ctx.h, model.h, stats.h, C.byref(b), C.byref(opts), sp))
        H.check(L.hmm_viterbi(ctx.h, model.h, C.byref(b), None, C.c_void_p(path.data_ptr()),
                              C.c_void_p(score.data_ptr()), sp))

    def timed(fn, n, flush=True):
        times = []
        for _ in range(n):
            if flush:
                flush_buf.fill_(1)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            times.append((e0, e1))
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in times]

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    ctx.profile(reset=True)
    ctx.set_option(_lib.OPT_PROFILE, 1)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        t_wall = time.perf_counter()
        step_ms = timed(step, args.steps)
        t_wall = time.perf_counter() - t_wall
    ctx.set_option(_lib.OPT_PROFILE, 0)
    prof = ctx.profile(reset=True)
    ms = float(np.sum(step_ms)) / args.steps
    if dist is not None:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    c_step = 2.0 * cells(offsets, NS)
    value = ws * c_step / (ms / 1e3)

    # ---- end to end through the public API with host buffers
    h_vals = torch.from_numpy(np.asarray(values, np.float32)).pin_memory()
    h_off = torch.from_numpy(np.asarray(offsets, np.int64)).pin_memory()
    h_mid = torch.from_numpy(np.asarray(mid, np.int32)).pin_memory()
    h_path = torch.empty(batch.total_T, dtype=torch.int32).pin_memory()
    h_ll = torch.empty(S, dtype=torch.float64).pin_memory()
    h_score = torch.empty(S, dtype=torch.float64).pin_memory()

    def e2e_step():
        batch.values.copy_(h_vals, non_blocking=True)
        batch.offsets.copy_(h_off, non_blocking=True)
        batch.model_id.copy_(h_mid, non_blocking=True)
        step()
        h_path.copy_(path, non_blocking=True)
        h_ll.copy_(ll, non_blocking=True)
        h_score.copy_(score, non_blocking=True)

    e2e_ms = float(np.mean(timed(e2e_step, max(2, args.steps // 2))))
    h2d = h_vals.numel() * 4 + h_off.numel() * 8 + h_mid.numel() * 4
    d2h = h_path.numel() * 4 + h_ll.numel() * 8 + h_score.numel() * 8

    # ---- plain float32 log-space GPU path, same step otherwise
    plain = None
    if not args.no_plain:
        ctx.set_option(_lib.OPT_PLAIN_ESTEP, 1)
        step()
        torch.cuda.synchronize()
        ctx.set_option(_lib.OPT_PROFILE, 1)
        pms = float(np.mean(timed(step, 2)))
        ctx.set_option(_lib.OPT_PROFILE, 0)
        pprof = ctx.profile(reset=True)
        ctx.set_option(_lib.OPT_PLAIN_ESTEP, 0)
        bw_plain = (pprof["plain"][0] + pprof["reduce"][0] + pprof["mstep"][0]) / 2
        plain = dict(ms_per_step=pms, bw_ms=bw_plain, plain_estep_ms=pprof["plain"][0] / 2)

    est_ms = prof["estep"][0] / max(prof["estep"][1], 1)
    bw_ms = (prof["estep"][0] + prof["reduce"][0] + prof["mstep"][0]) / args.steps
    vit_ms = prof["viterbi"][0] / max(prof["viterbi"][1], 1)
    launches = sum(v[1] for v in prof.values())
    # roofline of the fused E-step: 3 N^2 FP32 FMAs per (sequence, t)
    # (forward mat-vec, backward mat-vec, xi accumulation) = 6 N^2 flop
    pk = peaks()
    sm_max = float(pk.get("sm_max_mhz", 2070.0))
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    alu_peak = n_sm * 128 * 2 * sm_max * 1e6 / 1e12          # TFLOP/s, FP32 FMA
    flops = 6.0 * NS * NS * float(offsets[-1])
    achieved = flops / (est_ms / 1e3) / 1e12
    traffic = profiled_traffic("estep_small_N16_S4096_T2000.md",
                               ["estep_small.cuh", "estep_launch.cuh", "common.cuh"])
    if args.quick or args.family != "gamma" or args.workload != "scale":
        traffic = None
    roofline = dict(bound="alu", achieved=achieved, peak=alu_peak, unit="TFLOP/s",
                    frac=achieved / alu_peak, traffic=traffic,
                    algorithmic_bytes=float(offsets[-1]) * (8.0 + 8.0 * NS),
                    kernel="estep_small_kernel (fused emission+forward+backward+gamma/xi+stats)",
                    peak_note=f"FP32 FMA: {n_sm} SMs (device query) x 128 lanes x 2 flop x max SM clock "
                              f"{sm_max:g} MHz (derived)")
    # HBM view of the same launch: 8D + 8N + 16 bytes per (sequence, t)
    hbm_bytes = float(offsets[-1]) * (8.0 + 8.0 * NS + 16.0)
    hbm_peak = float(pk.get("hbm_gbs", 6800.0))
    estep_hbm = dict(bytes_per_seq_t=8.0 + 8.0 * NS + 16.0, achieved_gbs=hbm_bytes / (est_ms / 1e3) / 1e9,
                     peak_gbs=hbm_peak, frac=hbm_bytes / (est_ms / 1e3) / 1e9 / hbm_peak)
    clocks = clk.summary() if rank == 0 else None
    out = None
    if rank == 0:
        line = dict(metric=METRIC, value=value, unit=UNIT, n_gpus=ws, steps=args.steps,
                    warmup=max(args.warmup, 3), ms_per_step=ms, higher_is_better=True,
                    scaling="weak", vs_baseline=None, dtype="f32", data="synthetic",
                    config=arm_config(args, NS, S, offsets, len(models), ws, c_step),
                    clocks=clocks, e2e=dict(value=ws * c_step / (e2e_ms / 1e3), unit=UNIT,
                                            ms_per_step=e2e_ms, h2d_bytes_per_step=h2d,
                                            d2h_bytes_per_step=d2h),
                    gpu_launches=launches * ws, roofline=roofline,
                    breakdown=dict(estep_ms=est_ms, baum_welch_ms=bw_ms, viterbi_ms=vit_ms,
                                   reduce_ms=prof["reduce"][0] / args.steps,
                                   mstep_ms=prof["mstep"][0] / args.steps,
                                   baum_welch_cell_updates_per_s=cells(offsets, NS) / (bw_ms / 1e3),
                                   autotune_ms=tuned_ms,
                                   wall_s=t_wall),
                    estep_hbm=estep_hbm)
        if plain:
            line["plain_gpu"] = plain
            line["vs_plain_gpu"] = plain["bw_ms"] / bw_ms
        if not args.no_cpu_baseline and not args.quick and ws == 1:
            line["cpu_baseline"] = cpu_baseline(init, values, offsets, mid)
            if args.workload == "scale":
                line["cpu_baseline_all_cores"] = cpu_baseline_all_cores(init, values, offsets)
        out = line
        if emit and not (args.workload == "scale" and ws == 1 and not args.quick and not args.no_extras):
            print(json.dumps(out), flush=True)
    if exchange is not None:
        exchange.close()
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return out


def run_precision(args, emit=True):
    """Large dense N: N = 512, Dirichlet(0.1) rows, 1024 sequences x T = 4096,
    diagonal Gaussian D = 32.  One EM iteration + Viterbi with the tensor-core
    recursions, against the same step with the float32 CUDA-core recursions."""
    import ctypes as C
    import torch
    import paper_2605_29208_gb300 as H
    from paper_2605_29208_gb300 import _lib, synth
    n_seq, T = (128, 512) if args.quick else (1024, 4096)
    truth, init, values, offsets, mid = synth.large_state_workload(n_seq=n_seq, T=T)
    D = values.shape[1]
    NS = len(init["pi"])
    ctx = H.Context(0)
    model = H.Model(ctx, [init])
    batch = H.Batch(values, offsets, mid, dim=D).make_plan(ctx, model)
    stats = H.Stats(ctx, model)
    dev = batch.values.device
    S = batch.n_seq
    ll = torch.empty(S, dtype=torch.float64, device=dev)
    path = torch.empty(batch.total_T, dtype=torch.int32, device=dev)
    score = torch.empty(S, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    sp = C.c_void_p(stream.cuda_stream)
    flush_buf = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    opts = H.mstep_opts()
    b = batch.c()
    L = ctx.lib

    def step():
        H.check(L.hmm_estep_stats(ctx.h, model.h, C.byref(b), stats.h, C.c_void_p(ll.data_ptr()), sp))
        H.check(L.hmm_mstep(ctx.h, model.h, stats.h, C.byref(b), C.byref(opts), sp))
        H.check(L.hmm_viterbi(ctx.h, model.h, C.byref(b), None, C.c_void_p(path.data_ptr()),
                              C.c_void_p(score.data_ptr()), sp))

    def measure(tensor, steps, warmup):
        ctx.set_option(_lib.OPT_TENSOR_RECURRENCE, 1 if tensor else 0)
        model.set([init])
        for _ in range(warmup):
            step()
        torch.cuda.synchronize()
        ctx.profile(reset=True)
        ctx.set_option(_lib.OPT_PROFILE, 1)
        evs = []
        with ClockSampler(0) as clk:
            for _ in range(steps):
                flush_buf.fill_(1)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                step()
                e1.record(stream)
                evs.append((e0, e1))
            torch.cuda.synchronize()
        ctx.set_option(_lib.OPT_PROFILE, 0)
        prof = ctx.profile(reset=True)
        ms = float(np.mean([a.elapsed_time(b) for a, b in evs]))
        # log-likelihoods of the first E-step from the initial parameters
        model.set([init])
        H.check(L.hmm_estep_stats(ctx.h, model.h, C.byref(b), stats.h, C.c_void_p(ll.data_ptr()), sp))
        torch.cuda.synchronize()
        return ms, prof, clk.summary(), ll.cpu().numpy().copy()

    ms_tc, prof_tc, clk_tc, ll_tc = measure(True, args.steps, max(args.warmup, 3))
    ms_32, prof_32, _, ll_32 = measure(False, max(1, min(args.steps, 2)), 1)
    nst = max(prof_tc["estep"][1], 1)
    rec_ms = prof_tc["estep"][0] / nst
    # tensor work of one recursion launch: forward and backward GEMMs, 2 N^2 flop per (sequence, t) each
    flops = 4.0 * NS * NS * float(offsets[-1])
    pk = peaks()
    peak = float(pk.get("bf16_tflops", 1900.0))   # FP16 dense rate = BF16 dense rate
    achieved = flops / (rec_ms / 1e3) / 1e12
    c_step = 2.0 * cells(offsets, NS)
    rel = np.abs(ll_tc - ll_32) / np.maximum(1.0, np.abs(ll_32))
    steps = args.steps

    def per(prof, k, n):
        return prof[k][0] / n
    line = dict(metric=METRIC, value=c_step / (ms_tc / 1e3), unit=UNIT, n_gpus=1, steps=steps,
                warmup=max(args.warmup, 3), ms_per_step=ms_tc, higher_is_better=True, scaling="weak",
                vs_baseline=None, dtype="f16 operands, f32 accumulate (recursions); f32/f64 elsewhere",
                data="synthetic",
                config=dict(workload=f"precision: N={NS} states (Dirichlet(0.1) rows), {S} sequences x T={T}, "
                                     f"diagonal Gaussian D={D}; one EM iteration + Viterbi",
                            n_states=NS, n_seq_per_gpu=S, total_T=int(offsets[-1]), dim=D,
                            l2="flushed before every timed step (256 MiB write, outside the events)"),
                clocks=clk_tc,
                roofline=dict(bound="tensor", achieved=achieved, peak=peak, unit="TFLOP/s", frac=achieved / peak,
                              traffic=None, kernel="tc_fb_kernel (tcgen05 forward + backward recursions)",
                              peak_note="measured bf16 dense GEMM peak (FP16 runs at the BF16 rate)"),
                breakdown=dict(recursion_ms=rec_ms, emission_ms=per(prof_tc, "emission", steps),
                               posterior_stats_xi_ms=per(prof_tc, "reduce", steps),
                               xi_gemm_ms=per(prof_tc, "xi", steps),
                               mstep_ms=per(prof_tc, "mstep", steps), viterbi_ms=per(prof_tc, "viterbi", steps)),
                fp32_path=dict(ms_per_step=ms_32,
                               recursion_ms=prof_32["estep"][0] / max(prof_32["estep"][1], 1),
                               speedup_recursion=(prof_32["estep"][0] / max(prof_32["estep"][1], 1)) / rec_ms,
                               speedup_step=ms_32 / ms_tc),
                tensor_vs_fp32=dict(loglik_max_rel=float(rel.max()), loglik_median_rel=float(np.median(rel))),
                gpu_launches=int(sum(v[1] for v in prof_tc.values())))
    if emit:
        print(json.dumps(line), flush=True)
    return line


def run_serving(args, emit=True):
    """Request server under Poisson arrivals: decode / posterior / 10-iteration
    fit requests, N in {4, 16, 64, 256}, T log-uniform in [100, t_max],
    full-covariance Gaussian D = 8 or Gamma emissions, each request its own
    model.  Reports p50 / p99 latency (submit to completion) beside the
    throughput."""
    import torch
    import paper_2605_29208_gb300 as H
    from paper_2605_29208_gb300 import synth
    n_req = 100 if args.quick else args.requests
    t_max = 5000 if args.quick else args.t_max
    reqs = synth.serving_workload(n_req=n_req, rate=args.rate, t_max=t_max)
    ctx = H.Context(0)
    # warm the slots (model and buffer caches) with a short replay of the mix
    srv = H.Server(ctx, n_slots=args.slots, max_batch=16)
    warm = [srv.submit(r["kind"], r["model"], r["values"][:200], r["n_iter"]) for r in reqs[:64]]
    for t, r in zip(warm, reqs[:64]):
        x = srv.wait(t)
        if x["status"] != 0:
            print(f"warm-up request failed ({r['kind']}, {r['model']['family']}, N={len(r['model']['pi'])}): "
                  f"{x.get('error')}", file=sys.stderr)
    srv.close()
    srv = H.Server(ctx, n_slots=args.slots, max_batch=16)
    torch.cuda.synchronize()
    with ClockSampler(0) as clk:
        t0 = time.perf_counter()
        tickets = []
        for r in reqs:
            while time.perf_counter() - t0 < r["arrival_s"]:
                pass
            tickets.append(srv.submit(r["kind"], r["model"], r["values"], r["n_iter"]))
        results = [srv.wait(t, 3600e3) for t in tickets]
        makespan = time.perf_counter() - t0
    st = srv.stats()
    srv.close()
    lat = np.array([x["latency_ms"] for x in results])
    cells = 0.0
    for r in reqs:
        N = len(r["model"]["pi"])
        cells += N * N * len(r["values"]) * (r["n_iter"] if r["kind"] == "fit" else 1)
    by_kind = {}
    for r, x in zip(reqs, results):
        by_kind.setdefault(r["kind"], []).append(x["latency_ms"])
    line = dict(metric="serving latency p99 (submit to result), Poisson arrivals", value=float(np.percentile(lat, 99)),
                unit="ms", higher_is_better=False, n_gpus=1, steps=n_req, warmup=64, ms_per_step=None,
                scaling="weak", vs_baseline=None, dtype="f32 (f64 reductions)", data="synthetic",
                config=dict(workload=f"serving: {n_req} requests at {args.rate:g}/s, decode/posterior/fit(10) = "
                                     f"0.5/0.3/0.2, N in {{4,16,64,256}}, T log-uniform [100, {t_max}], "
                                     f"full-cov Gaussian D=8 or Gamma, each request its own model",
                            slots=args.slots, max_batch=16),
                p50_ms=float(np.percentile(lat, 50)), p99_ms=float(np.percentile(lat, 99)),
                mean_ms=float(lat.mean()), server_stats=st,
                p50_by_kind={k: float(np.percentile(v, 50)) for k, v in by_kind.items()},
                p99_by_kind={k: float(np.percentile(v, 99)) for k, v in by_kind.items()},
                offered_rate=args.rate, completed_per_s=n_req / makespan, makespan_s=makespan,
                cell_updates_per_s=cells / makespan, clocks=clk.summary(),
                failed=int(sum(1 for x in results if x["status"] != 0)),
                errors=sorted({x.get("error", "") for x in results if x["status"] != 0})[:5])
    if emit:
        print(json.dumps(line), flush=True)
    return line


def run_discrete(args):
    """Forward-backward throughput on small discrete HMMs (2 states / 2
    symbols and 3 states / 3 symbols) over sequence lengths 1e2 .. 1e6, in
    observations per millisecond: one sequence at a time (the setting of the
    paper's CPU table), and batches that fill the GPU (4096 sequences, or
    8e6 observations for the long ones)."""
    import torch
    import paper_2605_29208_gb300 as H
    from paper_2605_29208_gb300 import synth
    Ts = [100, 500, 1000, 5000, 10000, 50000, 100000, 500000, 1000000]
    if args.quick:
        Ts = [100, 1000, 10000]
    ctx = H.Context(0)
    stream = torch.cuda.current_stream()
    out = {}
    for N, K in ((2, 2), (3, 3)):
        rng = np.random.default_rng(synth.MASTER_SEED + 6 + N)
        A = synth.dirichlet_rows(rng, N, 1.0) * 0.2 + 0.8 * np.eye(N)
        model_d = synth.make_model("discrete", np.full(N, 1.0 / N), A / A.sum(1, keepdims=True),
                                   p=rng.dirichlet(np.ones(K), size=N))
        model = H.Model(ctx, [model_d])
        res = {}
        for T in Ts:
            row = {}
            for mode, S in (("single", 1), ("batched", int(max(1, min(4096, 8_000_000 // T))))):
                values, offsets, mid = synth.make_batch_many(synth.MASTER_SEED + T + S, [model_d], [T] * S,
                                                             [0] * S)
                batch = H.Batch(values, offsets, mid).make_plan(ctx, model)
                for _ in range(3):
                    H.forward_backward(ctx, model, batch)
                torch.cuda.synchronize()
                reps = 5
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(reps):
                    H.forward_backward(ctx, model, batch)
                e1.record(stream)
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1) / reps
                row[mode] = dict(n_seq=S, ms=ms, obs_per_ms=S * T / ms)
            res[T] = row
        sel = [T for T in Ts if 1000 <= T <= 1000000]
        out[f"N{N}_K{K}"] = dict(
            per_T={str(T): res[T] for T in Ts},
            mean_obs_per_ms_single=float(np.mean([res[T]["single"]["obs_per_ms"] for T in sel])) if sel else None,
            mean_obs_per_ms_batched=float(np.mean([res[T]["batched"]["obs_per_ms"] for T in sel])) if sel else None)
    line = dict(metric="forward-backward throughput, small discrete HMMs", unit="obs/ms", higher_is_better=True,
                value=out["N2_K2"]["mean_obs_per_ms_batched"], n_gpus=1, dtype="f32", data="synthetic",
                config=dict(workload="2-state 2-symbol and 3-state 3-symbol discrete HMMs, T in 1e2..1e6, "
                                     "posteriors written (gamma), mean over T in 1e3..1e6"),
                results=out,
                context="the paper's CPU library: ~9,300 obs/ms single-threaded on one sequence "
                        "(2-state discrete, mean over T in 1e3..1e6; other hardware)")
    print(json.dumps(line), flush=True)
    return line


def main():
    args = args_parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "precision":
        run_precision(args)
    elif args.workload == "serving":
        run_serving(args)
    elif args.workload == "discrete":
        run_discrete(args)
    else:
        line = run_ours(args)
        ws = dist_env()[0]
        if line is not None and args.workload == "scale" and ws == 1 and not args.quick and not args.no_extras:
            line.update(extra_workloads(args))
            print(json.dumps(line), flush=True)


def _sub(args, **kw):
    a = argparse.Namespace(**vars(args))
    for k, v in kw.items():
        setattr(a, k, v)
    return a


def _free_gpu():
    import gc
    import torch
    gc.collect()
    torch.cuda.synchronize()
    torch.cuda.empty_cache()


def extra_workloads(args):
    """The other configurations of the metric, measured in the same run
    after the headline line: the batching step (with its E-step HBM
    fraction and the plain-path ratio), the precision step (tensor-core
    recursion fraction of the tensor peak) and serving latency (a rate the
    server sustains, and the configured arrival rate)."""
    out = {}
    t0 = time.perf_counter()
    _free_gpu()
    try:
        b = run_ours(_sub(args, workload="batching", steps=5, warmup=3, no_cpu_baseline=True), emit=False)
        keep = ("ms_per_step", "value", "config", "breakdown", "estep_hbm", "vs_plain_gpu", "plain_gpu", "clocks")
        out["batching"] = {k: b.get(k) for k in keep}
    except Exception as e:                       # reported, never silently dropped
        out["batching"] = dict(error=repr(e))
    _free_gpu()
    try:
        p = run_precision(_sub(args, workload="precision", steps=2, warmup=1), emit=False)
        keep = ("ms_per_step", "value", "config", "roofline", "breakdown", "fp32_path", "tensor_vs_fp32", "clocks")
        out["precision"] = {k: p.get(k) for k in keep}
    except Exception as e:
        out["precision"] = dict(error=repr(e))
    _free_gpu()
    serving = {}
    for name, rate, n in (("sustained", args.serve_rate, args.serve_requests),
                          ("offered_2000_per_s", 2000.0, args.serve_requests)):
        try:
            r = run_serving(_sub(args, workload="serving", rate=rate, requests=n), emit=False)
            serving[name] = {k: r.get(k) for k in ("p50_ms", "p99_ms", "mean_ms", "offered_rate", "completed_per_s",
                                                   "makespan_s", "cell_updates_per_s", "failed", "config",
                                                   "p99_by_kind", "clocks")}
            serving[name]["sustained"] = r["completed_per_s"] >= 0.9 * rate
        except Exception as e:
            serving[name] = dict(error=repr(e))
        _free_gpu()
    out["serving"] = serving
    out["extras_wall_s"] = time.perf_counter() - t0
    return out


if __name__ == "__main__":
    main()

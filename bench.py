"""Throughput benchmark: energyscapes/s at 32 ch x 16384 samples x 2048 directions.

A step is one seeded synthetic measurement (32 mics, 16384 int16 samples,
20 reflectors on the frontal hemisphere, 20 dB SNR) through the whole chain
on one GPU: matched filter -> delay-and-sum over 2048 Fibonacci half-sphere
directions in both forms (time domain with Catmull-Rom fractional delays,
and frequency domain with exact phase ramps) -> envelope, low-pass,
subsample -> two energyscapes 2048 x 1638 (FP32).  The input sits in HBM when the clock starts; L2 is
flushed (a 512 MiB write, then a 256 MiB read so that its write-backs end) between steps, outside the
timed events.

Printed (rank 0, one JSON line): value = energyscapes/s over all ranks,
e2e = the same through rtis_process with pinned host buffers (H2D input and
D2H energyscape inside the timed region), roofline of the dominant kernel
(whichever beamformer takes longer; both are FP32-FMA bound), the FP64 oracle timed on the host as
cpu_baseline, and SM clocks sampled during the timed region.

--impl reference times the FP64 oracle itself (on a bounded sample of
directions per step) with the same metric.  Multi-GPU: independent replicas
(the work shards by measurement; no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np

# The end-to-end loop runs compute, H2D and two D2H streams at once.  With the default 8
# hardware work queues streams can share a queue, and then a step's kernels wait behind the
# previous step's D2H copy (measured: 51.4 ms per step with copies of 9.4 ms beside 39.6 ms of
# compute); 32 queues keep the four streams apart.  Read when CUDA starts, so set it first.
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

N_SAMPLES, N_DIRS, N_MICS = 16384, 2048, 32
METRIC = "energyscapes/s at 32ch x 16384 samples x 2048 dirs; error vs FP64 oracle"
WORKLOAD = "hemisphere: 32 mics (12 cm square, seeded), 16384 samples @ 450 kHz, 2048 Fibonacci half-sphere dirs, " \
           "20 reflectors 0.3-6 m, 20 dB SNR, int16; matched filter + time-domain and frequency-domain DAS, FP32"
FP32_LANES_PER_SM = 128     # FP32 FMA lanes per SM (4 SMSPs x 32)
SM_MAX_MHZ_NOMINAL = 2070.0
# dram__bytes_read.sum + dram__bytes_write.sum of one launch of each beamformer (ncu capture of this
# workload, see profiles/); set to None whenever that kernel changes until it is re-captured
TD_TRAFFIC_BYTES = 5552896
FD_TRAFFIC_BYTES = None  # the per-direction kernel (--batch 1); changed since its last capture
# bb_beamform_kernel on the hemisphere workload (the <8, 4> layout; z and the tables, E stays in L2)
BB_TRAFFIC_BYTES = 2937344 + 512
# td_adjoint_kernel on the calibration workload (32 x 16384 x 2048)
ADJ_TRAFFIC_BYTES = 20026112 + 44800
# fd_gemm_kernel_ws<BF16> captured at 400 bins (DRAM read + write), per bin; X and Y both grow with the bins
FD_GEMM_TRAFFIC_PER_BIN = (13974784 + 358491648) / 400
N_REF_DIRS = 16   # directions per step of the reference arm (the FP64 oracle)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(values, dev=None):
    """Element-wise max of per-rank timings (the slowest replica sets the clock).
    With one process the values come back unchanged; NCCL reduces on the GPU,
    gloo on the CPU."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [float(v) for v in values]
    on = dev if (dev is not None and dist.get_backend() == "nccl") else "cpu"
    tt = torch.tensor([float(v) for v in values], dtype=torch.float64, device=on)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return [float(v) for v in tt.cpu()]


def replica_rate(units_per_rank: int, world: int, seconds: float) -> float:
    """Whole-job throughput of independent replicas: every rank's units over the slowest time."""
    return world * units_per_rank / seconds


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clock / throttle-reason sampling while the timed region runs."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.15)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out = ""
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


class L2Flush:
    """Between timed steps: write 512 MiB (evicts everything the last step left in
    the 129 MB L2), then read 256 MiB more, so the dirty lines of that write are
    written back before the next step's clock starts rather than during it."""

    def __init__(self, dev):
        import torch
        self.w = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
        self.r = torch.ones(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
        self.sink = None

    def __call__(self, v=0.0):
        self.w.fill_(float(v))
        self.sink = self.r.sum()


def oracle_sample(cfg, n_dirs_sample: int, seed: int = 0):
    """The FP64 oracle on a seeded sample of directions: (seconds for one step scaled to all
    directions, matched-filter seconds, sampled-DAS seconds, sampled direction indices, TD rows,
    FD rows)."""
    import oracle
    rng = np.random.default_rng(seed)
    pick = np.sort(rng.choice(cfg["dirs"].shape[0], n_dirs_sample, replace=False))
    t0 = time.perf_counter()
    a = oracle.matched_filter(cfg["x"], cfg["chirp"], cfg["fs"])
    A, k_lo, F = oracle.mf_spectrum(cfg["x"], cfg["chirp"], cfg["fs"])
    t1 = time.perf_counter()
    delta = oracle.steering_delays(cfg["mic_xyz"], cfg["dirs"][pick], cfg["fs"], cfg["c"])
    h = oracle.lpf_taps()
    e_td = oracle.envelope_decimate(oracle.das_td(a, delta), h)
    e_fd = oracle.envelope_decimate(oracle.das_fd(A, k_lo, F, cfg["n_samples"], delta), h)
    t2 = time.perf_counter()
    D = cfg["dirs"].shape[0]
    return (t1 - t0) + (t2 - t1) * D / n_dirs_sample, (t1 - t0), (t2 - t1), pick, e_td, e_fd


def oracle_sample_time(cfg, n_dirs_sample: int, seed: int = 0):
    """Seconds the FP64 oracle needs for one step (both energyscapes), from a direction sample."""
    return oracle_sample(cfg, n_dirs_sample, seed)[:3]


def oracle_error_entry(pick, pairs):
    """The bench line's error against the FP64 oracle on the sampled directions.  pairs: name ->
    (oracle rows [n][n_out], the GPU energyscape [D][n_out] as a tensor or array).  Reported, not
    a pass/fail: the tests hold the tolerance."""
    out = {"directions_sampled": int(len(pick)), "fp32_tolerance_over_peak": 1e-4}
    for name, (ref, E) in pairs.items():
        got = np.asarray(E.cpu().numpy() if hasattr(E, "cpu") else E, dtype=np.float64)[pick]
        ref = np.asarray(ref, dtype=np.float64)
        peak = float(ref.max())
        out[name] = {"max_abs_err_over_peak": float(np.max(np.abs(got - ref)) / peak),
                     "peak_index_match": bool(np.argmax(got) == np.argmax(ref))}
    return out


def _oracle_worker(job):
    """One spawn worker of oracle_pool_rate: time the oracle on its own measurement."""
    seed, n_dirs_sample = job
    import synth
    cfg = synth.hemisphere(seed_scene=1 + seed)
    return oracle_sample_time(cfg, n_dirs_sample, seed=seed)[0]


def oracle_pool_rate(n_dirs_sample: int, procs: int = 0):
    """Energyscapes/s of the FP64 oracle on all host cores, the way the paper's CPU workers run:
    `procs` spawned processes (default: the cores this process may use), each timing one
    measurement on a bounded direction sample (scaled to all directions), all at once; the rate is
    procs / the slowest worker's time.  Spawned, not forked, so it is safe after CUDA is up."""
    import multiprocessing as mp
    procs = procs or len(os.sched_getaffinity(0))
    with mp.get_context("spawn").Pool(procs) as pool:  # leaving the block terminates the workers
        jobs = pool.map_async(_oracle_worker, [(k, n_dirs_sample) for k in range(procs)], chunksize=1)
        times = jobs.get(timeout=600)  # a worker that died would otherwise leave map() waiting
    return procs / max(times), procs


def all_cores_baseline(n_dirs_sample: int):
    """The cpu_baseline_all_cores entry of a bench line; a failure of the process pool is
    reported in the entry rather than ending the benchmark."""
    try:
        rate, procs = oracle_pool_rate(n_dirs_sample)
    except Exception as exc:  # noqa: BLE001 -- a host-side extra must not cost the GPU measurement
        return {"unavailable": f"oracle process pool failed: {type(exc).__name__}: {exc}"[:300]}
    return {"value": rate, "unit": "energyscapes/s", "cores": procs, "kind": "oracle",
            "sample": f"FP64 oracle in {procs} spawned processes at once, one measurement each: matched filter "
                      f"on all 32 channels + both DAS forms on {n_dirs_sample} of {N_DIRS} directions, scaled to "
                      f"{N_DIRS}; rate = processes / slowest"}


def run_reference(args, rank, world):
    """The FP64 oracle timed on the host.  A step is a bounded sample of one measurement's
    work: the matched filter of all 32 channels and both DAS forms on N_REF_DIRS of the 2048
    directions.  ms_per_step is that step's measured wall time; value scales the DAS part to
    all directions (scale_factor) to give energyscapes/s of the whole workload."""
    if rank != 0:
        return
    import synth
    cfg = synth.hemisphere()
    n_s = N_REF_DIRS
    scale = N_DIRS / n_s
    for _ in range(args.warmup):
        oracle_sample_time(cfg, n_s)
    wall, t_mf, t_das = [], [], []
    for k in range(args.steps):
        t0 = time.perf_counter()
        _, mf, das = oracle_sample_time(cfg, n_s, seed=k + 1)
        wall.append(time.perf_counter() - t0)
        t_mf.append(mf)
        t_das.append(das)
    t_full = float(np.sum(t_mf) + scale * np.sum(t_das))  # seconds for `steps` whole energyscapes
    value = args.steps / t_full
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "energyscapes/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(wall)),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_mics": N_MICS, "n_samples": N_SAMPLES, "n_dirs": N_DIRS,
                   "n_out": N_SAMPLES // 10, "decim": 10,
                   "paths_per_step": "time-domain (Catmull-Rom) and frequency-domain (phase ramp) energyscapes "
                                     "of the same measurement; value counts measurements",
                   "parallelism": "single process (NumPy, FP64)"},
        "value_basis": {"scale_factor": scale, "dirs_per_step": n_s,
                        "formula": "value = steps / (sum of matched-filter seconds + scale_factor x sum of "
                                   "sampled-direction DAS seconds); ms_per_step = measured wall time of a step",
                        "matched_filter_s_per_step": float(np.mean(t_mf)),
                        "das_s_per_step": float(np.mean(t_das))},
        "cpu_baseline": {"value": value, "unit": "energyscapes/s", "cores": 1, "kind": "oracle",
                         "sample": f"per step: matched filter on all 32 channels + time- and frequency-domain "
                                   f"DAS/envelope on {n_s} of {N_DIRS} directions (measured), the DAS time "
                                   f"scaled by {scale:g} to {N_DIRS} directions"},
        "e2e": {"value": value, "unit": "energyscapes/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_fd_gemm(args, rank, world, local):
    """Frequency-domain beamforming GEMM: 1200 bins x 32 mics x 64 frames -> 2048 directions."""
    import torch
    import torch.distributed as dist

    import synth
    from paper_2208_10839_gb300 import FdGemm
    from paper_2208_10839_gb300 import build as _b
    _b.build()
    dev = torch.device("cuda", local)
    cfg = synth.gemm_frames(n_bins=args.bins, seed0=100 + 1000 * rank)
    K, M, T = cfg["X"].shape
    D = cfg["dirs"].shape[0]
    g = FdGemm(cfg["mic_xyz"], cfg["dirs"], cfg["freqs"], T, precision=args.precision)
    X = torch.from_numpy(cfg["X"].astype(np.complex64)).to(dev)
    Y = torch.empty((K, D, T), dtype=torch.complex64, device=dev)
    flush = L2Flush(dev)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        flush(1.0)
        g.run(X, Y)
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            flush(float(k))
            evs[k][0].record(stream)
            g.run(X, Y)
            evs[k][1].record(stream)
        torch.cuda.synchronize()
    ms = [a.elapsed_time(b) for a, b in evs]
    t = sum(ms) / 1e3
    if world > 1:
        (t,) = max_over_ranks([t], dev)
    # error against the FP64 oracle on sampled bins (test infrastructure)
    import oracle
    picks = sorted({0, K // 4, K // 2, (3 * K) // 4, K - 1})
    Ys = Y[picks].cpu().numpy().astype(np.complex128)
    W = oracle.steering_matrix(cfg["freqs"][picks], cfg["mic_xyz"], cfg["dirs"], cfg["c"])
    Yr = oracle.fd_gemm(W, cfg["X"][picks].astype(np.complex64).astype(np.complex128))
    err = float(np.max(np.abs(Ys - Yr)) / np.max(np.abs(Yr)))
    peaks = load_peaks()
    bytes_alg = K * M * T * 8 + K * D * T * 8
    launch_s = statistics.mean(ms) / 1e3
    hbm = peaks.get("hbm_gbs")
    line = {
        "metric": "frames/s (1200-bin x 2048-dir x 32-mic steering GEMM per frame)", "value": replica_rate(args.steps * T, world, t),
        "unit": "frames/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": args.precision, "data": "synthetic",
        "config": {"workload": cfg["name"], "precision": args.precision, "l2": "flushed between steps (512 MiB write, then a 256 MiB read so write-backs finish), outside the timed events"},
        "error_vs_fp64_oracle": {"max_abs_over_max": err, "bins_checked": picks},
        "gpu_launches": 2 * args.steps,
        "roofline": {"bound": "hbm", "kernel": "fd_gemm_kernel", "achieved": bytes_alg / launch_s / 1e9,
                     "peak": hbm, "unit": "GB/s", "frac": (bytes_alg / launch_s / 1e9) / hbm if hbm else None,
                     "traffic": (FD_GEMM_TRAFFIC_PER_BIN * K) if args.precision == "bf16" else None,
                     "traffic_note": "BF16 capture at 400 bins scaled by the bin count", "algorithmic_bytes_per_launch": bytes_alg, "launch_ms": launch_s * 1e3,
                     "tensor_flops_per_launch": 8.0 * K * D * M * T * (3 if args.precision == "fp32" else 1)},
        "clocks": clk.summary(),
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    g.close()


def run_ring(args, rank, world, local):
    """8 sensors on a ring, N in {4096..32768}, D in {512..4096}: one batch per step."""
    import torch
    import torch.distributed as dist

    import synth
    from paper_2208_10839_gb300 import Batch, Plan
    from paper_2208_10839_gb300 import build as _b
    _b.build()
    dev = torch.device("cuda", local)
    ring = synth.ring_sensors(seed_scene=3 + 1000 * rank)
    sensors = ring["sensors"]
    if args.precision not in ("fp32", "bf16"):
        raise SystemExit("ring: --precision fp32 or bf16 (storage of the analytic signal)")
    plans = [Plan(s["mic_xyz"], s["fs"], s["chirp"], s["dirs"], s["n_samples"], precision=args.precision)
             for s in sensors]
    xs = [torch.from_numpy(s["x"]).to(dev) for s in sensors]
    outs = [torch.empty((p.D, p.n_out), dtype=torch.float32, device=dev) for p in plans]
    flush = L2Flush(dev)
    stream = torch.cuda.current_stream()
    batch = Batch(plans)
    for _ in range(args.warmup):  # the first run autotunes
        flush(1.0)
        batch.run(xs, outs)
    torch.cuda.synchronize()
    assert batch.sync() == 0
    info = batch.info
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            flush(float(k))
            evs[k][0].record(stream)
            batch.run(xs, outs)
            evs[k][1].record(stream)
        torch.cuda.synchronize()
    t = sum(a.elapsed_time(b) for a, b in evs) / 1e3
    # the same sensors one rtis_process at a time, for comparison
    seq = []
    for k in range(max(3, args.steps // 4)):
        flush(float(k))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for p, x, o in zip(plans, xs, outs):
            p.process(x, o)
        e1.record(stream)
        torch.cuda.synchronize()
        seq.append(e0.elapsed_time(e1))
    if world > 1:
        (t,) = max_over_ranks([t], dev)
    n_s = len(sensors)
    line = {
        "metric": "energyscapes/s (ring of 8 sensors, ragged N and D, one batch per step)",
        "value": replica_rate(args.steps * n_s, world, t), "unit": "energyscapes/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else "bf16 storage, f32 arithmetic",
        "data": "synthetic",
        "config": {"workload": ring["name"], "storage": args.precision, "sensors": [(s["n_samples"], int(s["dirs"].shape[0])) for s in sensors],
                   "l2": "flushed between steps (512 MiB write, then a 256 MiB read so write-backs finish), outside the timed events"},
        "autotune": {"variant": info.variant, "grid": info.grid, "tiles": info.total_tiles,
                     "beamformer_ms": info.tuned_ms},
        "sequential_rtis_process_ms": statistics.mean(seq),
        "gpu_launches": args.steps * 3,  # two ragged matched-filter launches + the beamformer
        "clocks": clk.summary(),
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    batch.close()
    for p in plans:
        p.close()


def run_calibration(args, rank, world, local):
    """Self-calibration gradient: 32 perturbed mics x 16384 samples x 2048 directions,
    10 known reflectors; a step = energyscape + L2 loss + adjoint w.r.t. xyz/gain/delay."""
    import torch
    import torch.distributed as dist

    import synth
    from paper_2208_10839_gb300 import Calibrator, Plan, _native as nat
    from paper_2208_10839_gb300 import build as _b
    _b.build()
    dev = torch.device("cuda", local)
    cfg = synth.calibration(seed=4 + 1000 * rank)
    plan = Plan(cfg["mic_nominal"], cfg["fs"], cfg["chirp"], cfg["dirs"], cfg["n_samples"], c=cfg["c"])
    x = torch.from_numpy(cfg["x"]).to(dev)
    E_ref = plan.process(torch.from_numpy(cfg["x_ref"]).to(dev)).clone()
    cal = Calibrator(plan, cfg["mic_nominal"])
    for _ in range(3):  # a few descent steps so the estimate is off nominal
        cal.step(x, E_ref)
    p_, g_, d_ = cal.params()
    plan.set_calibration(p_, g_, d_)
    M, N, D = plan.M, plan.N, plan.D
    h = plan.handle
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream
    E = torch.empty((D, plan.n_out), dtype=torch.float32, device=dev)
    G = torch.empty_like(E)
    loss = torch.empty(1, dtype=torch.float32, device=dev)
    gx = torch.empty((M, 3), dtype=torch.float32, device=dev)
    gg = torch.empty(M, dtype=torch.float32, device=dev)
    gd = torch.empty(M, dtype=torch.float32, device=dev)
    flush = L2Flush(dev)

    def step(xin, ev=None):
        if ev:
            ev[0].record(stream)
        nat.rtis_set_calibration(h, p_, g_, d_, sh)
        nat.rtis_process(h, xin, E, sh)
        nat.rtis_loss_l2(h, E, E_ref, G, loss, sh)
        if ev:
            ev[1].record(stream)
        nat.rtis_backward(h, xin, G, gx, gg, gd, sh)
        if ev:
            ev[2].record(stream)

    for _ in range(args.warmup):
        flush(1.0)
        step(x)
    torch.cuda.synchronize()
    assert plan.sync() == 0
    evs = [tuple(torch.cuda.Event(enable_timing=True) for _ in range(3)) for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            flush(float(k))
            step(x, evs[k])
        torch.cuda.synchronize()
    step_ms = [e[0].elapsed_time(e[2]) for e in evs]
    fwd_ms = [e[0].elapsed_time(e[1]) for e in evs]
    bwd_ms = [e[1].elapsed_time(e[2]) for e in evs]
    t = sum(step_ms) / 1e3
    # the matched filter alone (rtis_backward recomputes it first), to split the backward time
    a_buf = torch.empty((M, N), dtype=torch.complex64, device=dev)
    mf = []
    for k in range(max(3, args.steps // 4)):
        flush(float(k))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        nat.rtis_matched_filter(h, x, a_buf, None, sh)
        e1.record(stream)
        torch.cuda.synchronize()
        mf.append(e0.elapsed_time(e1))
    assert plan.sync() == 0

    # end to end: pinned host recording in, gradients and loss out
    xh = torch.from_numpy(cfg["x"]).pin_memory()
    xd = torch.empty_like(x)
    gh = [torch.empty(v.shape, dtype=torch.float32).pin_memory() for v in (gx, gg, gd, loss)]

    def e2e_step():
        xd.copy_(xh, non_blocking=True)
        step(xd)
        for hv, dv in zip(gh, (gx, gg, gd, loss)):
            hv.copy_(dv, non_blocking=True)

    for _ in range(3):
        e2e_step()
    torch.cuda.synchronize()
    n_e2e = max(args.steps // 2, 3)
    ee0, ee1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ee0.record(stream)
    for _ in range(n_e2e):
        e2e_step()
    ee1.record(stream)
    torch.cuda.synchronize()
    t_e2e = ee0.elapsed_time(ee1) / 1e3
    if world > 1:
        t, t_e2e = max_over_ranks([t, t_e2e], dev)
    props = torch.cuda.get_device_properties(dev)
    n_sm = props.multi_processor_count
    peak_tf = n_sm * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ_NOMINAL * 1e6 / 1e12
    # adjoint: recomputed beams (4 taps x 2 FMAs) + tap correlations (4 taps x 2 FMAs) per (d, n, m)
    flops = float(D) * N * M * 16 * 2
    adj_s = (statistics.mean(bwd_ms) - statistics.mean(mf)) / 1e3
    line = {
        "metric": "calibration gradients/s (energyscape + L2 loss + adjoint wrt mic xyz, gain, delay; "
                  "32ch x 16384 samples x 2048 dirs)",
        "value": replica_rate(args.steps, world, t), "unit": "gradients/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "calibration: 32 mics perturbed by N(0, 1 mm), gains U(0.8, 1.2), delays "
                               "U(-2, 2) us; 16384 samples, 2048 Fibonacci half-sphere dirs, 10 known reflectors",
                   "l2": "flushed between steps (512 MiB write, then a 256 MiB read so write-backs finish), outside the timed events"},
        "e2e": {"value": replica_rate(n_e2e, world, t_e2e), "unit": "gradients/s", "h2d_bytes_per_step": int(x.numel() * 2),
                "d2h_bytes_per_step": int(4 * (gx.numel() + gg.numel() + gd.numel() + 1))},
        "gpu_launches": 11 * args.steps,
        "kernels_ms": {"forward_and_loss": statistics.mean(fwd_ms), "backward": statistics.mean(bwd_ms),
                       "matched_filter": statistics.mean(mf),
                       "adjoint_and_reduce": statistics.mean(bwd_ms) - statistics.mean(mf)},
        "roofline": {"bound": "alu", "kernel": "td_adjoint_kernel (+ adj_reduce_kernel)",
                     "achieved": flops / adj_s / 1e12, "peak": peak_tf, "unit": "TFLOP/s",
                     "frac": flops / adj_s / 1e12 / peak_tf, "traffic": ADJ_TRAFFIC_BYTES,
                     "peak_basis": f"{n_sm} SMs x {FP32_LANES_PER_SM} FP32 FMA lanes x 2 flop x "
                                   f"{SM_MAX_MHZ_NOMINAL:.0f} MHz",
                     "algorithmic_flops_per_launch": flops, "launch_ms": adj_s * 1e3},
        "clocks": clk.summary(),
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        rng = np.random.default_rng(0)
        pick = np.sort(rng.choice(D, 32, replace=False))
        Gs = G.cpu().numpy()[pick].astype(np.float64)
        pn, gn, dn = (v.cpu().numpy().astype(np.float64) for v in (p_, g_, d_))
        t0 = time.perf_counter()
        oracle.energyscape_vjp(cfg["x"], cfg["chirp"], pn, cfg["dirs"][pick], cfg["fs"], cfg["c"], Gs, gain=gn,
                               delay_s=dn)
        t_or = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": 32.0 / D / t_or, "unit": "gradients/s", "cores": 1, "kind": "oracle",
                                "sample": f"FP64 oracle energyscape_vjp on 32 of {D} directions "
                                          f"({t_or:.2f} s), scaled to {D}"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    plan.close()


def run_stream(args, rank, world, local):
    """The streaming service: hemisphere measurements submitted from host memory and
    collected, energyscape in host memory, through a ring of 4 pinned slots; wall-clock
    throughput and per-measurement latency (submit to result in host memory)."""
    import torch
    import torch.distributed as dist

    import synth
    from paper_2208_10839_gb300 import Plan, _native as nat
    from paper_2208_10839_gb300 import build as _b
    _b.build()
    depth = 4
    cfgs = [synth.hemisphere(seed_scene=1 + 1000 * rank + i) for i in range(8)]
    xs = [np.ascontiguousarray(c["x"]) for c in cfgs]
    plan = Plan(cfgs[0]["mic_xyz"], cfgs[0]["fs"], cfgs[0]["chirp"], cfgs[0]["dirs"], cfgs[0]["n_samples"])
    s = nat.rtis_stream_create(plan.handle, depth)
    # one pinned result buffer per ring slot (ticket t lands in outs[t % depth])
    outs = [torch.empty((plan.D, plan.n_out), dtype=torch.float32).pin_memory() for _ in range(depth)]
    nxt = [0]

    def run(n):
        t_sub, lat = {}, []
        pending = []
        for i in range(n):
            if len(pending) == depth:
                tk = pending.pop(0)
                nat.rtis_stream_wait(s, tk, 10000)
                lat.append(time.perf_counter() - t_sub.pop(tk))
            t0 = time.perf_counter()
            tk = nat.rtis_stream_submit(s, xs[i % len(xs)], outs[nxt[0] % depth])
            nxt[0] += 1
            t_sub[tk] = t0
            pending.append(tk)
        for tk in pending:
            nat.rtis_stream_wait(s, tk, 10000)
            lat.append(time.perf_counter() - t_sub.pop(tk))
        return lat

    run(max(args.warmup, 3) * depth)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t0 = time.perf_counter()
        lat = run(args.steps)
        t = time.perf_counter() - t0
    assert plan.sync() == 0
    (t,) = max_over_ranks([t])
    lat_ms = sorted(1e3 * v for v in lat)
    line = {
        "metric": "measurements/s through rtis_stream (int16 host in, TD energyscape host out), wall clock",
        "value": replica_rate(args.steps, world, t), "unit": "measurements/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD.replace("matched filter + time-domain and frequency-domain DAS",
                                                "time-domain path, streamed"), "ring_depth": depth,
                   "l2": "not flushed: a service loop, each input arrives fresh by H2D"},
        "latency_ms": {"p50": lat_ms[len(lat_ms) // 2], "p99": lat_ms[min(len(lat_ms) - 1, int(0.99 * len(lat_ms)))],
                       "max": lat_ms[-1]},
        "paper_rate_check": "at 20 Hz per sensor this sustains the measurements of "
                            f"{int(replica_rate(args.steps, world, t) / 20)} sensors on one GPU",
        "gpu_launches": 3 * args.steps,
        "clocks": clk.summary(),
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    nat.rtis_stream_destroy(s)
    plan.close()


def run_paper_design(args, rank, world, local):
    """The time-domain chain built the paper's way (cuFFT matched filter, one thread per
    (direction, sample) delay-and-sum, envelope in device memory, separate low-pass kernel)
    against the fused kernels, one measurement per step each."""
    import torch
    import torch.distributed as dist

    import synth
    from paper_2208_10839_gb300 import Plan, _native as nat
    from paper_2208_10839_gb300 import build as _b
    _b.build()
    dev = torch.device("cuda", local)
    cfg = synth.hemisphere(seed_scene=1 + 1000 * rank)
    plan = Plan(cfg["mic_xyz"], cfg["fs"], cfg["chirp"], cfg["dirs"], cfg["n_samples"])
    x = torch.from_numpy(cfg["x"]).to(dev)
    E = torch.empty((N_DIRS, plan.n_out), dtype=torch.float32, device=dev)
    Eb = torch.empty_like(E)
    plan.process(x, E)  # builds the steering table the baseline reads
    b = nat.rtis_baseline_create(plan.handle)
    flush = L2Flush(dev)
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream

    def timed(fn):
        for _ in range(args.warmup):
            flush(1.0)
            fn()
        torch.cuda.synchronize()
        ms = []
        for k in range(args.steps):
            flush(float(k))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            ms.append((e0, e1))
        torch.cuda.synchronize()
        return [a.elapsed_time(c) for a, c in ms]

    if world > 1:
        dist.barrier()
    with ClockSampler(local) as clk:
        base_ms = timed(lambda: nat.rtis_baseline_process(b, x, Eb, sh))
        fused_ms = timed(lambda: nat.rtis_process(plan.handle, x, E, sh))
    torch.cuda.synchronize()
    assert plan.sync() == 0
    err = float((Eb - E).abs().max() / E.abs().max())
    t_base, t_fused = sum(base_ms) / 1e3, sum(fused_ms) / 1e3
    if world > 1:
        t_base, t_fused = max_over_ranks([t_base, t_fused], dev)
    nat.rtis_baseline_destroy(b)
    line = {
        "metric": "energyscapes/s, time-domain path, paper-style GPU design (cuFFT + per-sample DAS)",
        "value": replica_rate(args.steps, world, t_base), "unit": "energyscapes/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_base / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD.replace("matched filter + time-domain and frequency-domain DAS",
                                                "time-domain path only"),
                   "l2": "flushed between steps (512 MiB write, then a 256 MiB read so write-backs finish), "
                         "outside the timed events"},
        "fused_rtis_process": {"value": replica_rate(args.steps, world, t_fused), "unit": "energyscapes/s",
                               "ms_per_step": 1e3 * t_fused / args.steps},
        "speedup_fused_over_paper_design": t_base / t_fused,
        "max_abs_diff_over_max": err,
        "gpu_launches": 6 * args.steps,
        "clocks": clk.summary(),
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    plan.close()


def run_baseband(args, rank, world, local):
    """The complex-baseband path (the analytic signal demodulated to 0 Hz and beamformed on
    every 4th sample) against the full-rate time-domain path, one measurement per step each;
    the baseband beamformer's roofline from its own stage entry point."""
    import torch
    import torch.distributed as dist

    import synth
    from paper_2208_10839_gb300 import Plan, _native as nat
    from paper_2208_10839_gb300 import build as _b
    _b.build()
    dev = torch.device("cuda", local)
    cfg = synth.hemisphere(seed_scene=1 + 1000 * rank)
    mk = lambda path: Plan(cfg["mic_xyz"], cfg["fs"], cfg["chirp"], cfg["dirs"], cfg["n_samples"], path=path)
    p_bb, p_td, p_fd = mk("bb"), mk("td"), mk("fd")
    x = torch.from_numpy(cfg["x"]).to(dev)
    E_bb = torch.empty((N_DIRS, p_bb.n_out), dtype=torch.float32, device=dev)
    E_td, E_fd, E_st = torch.empty_like(E_bb), torch.empty_like(E_bb), torch.empty_like(E_bb)
    z = p_bb.baseband_signal(x)
    a, _ = p_td.matched_filter(x)
    flush = L2Flush(dev)
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream

    def timed(fn):
        for _ in range(args.warmup):
            flush(1.0)
            fn()
        torch.cuda.synchronize()
        ms = []
        for k in range(args.steps):
            flush(float(k))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            ms.append((e0, e1))
        torch.cuda.synchronize()
        return [q.elapsed_time(r) for q, r in ms]

    if world > 1:
        dist.barrier()
    with ClockSampler(local) as clk:
        bb_ms = timed(lambda: nat.rtis_process(p_bb.handle, x, E_bb, sh))
        td_ms = timed(lambda: nat.rtis_process(p_td.handle, x, E_td, sh))
        bbk_ms = timed(lambda: nat.rtis_beamform_bb(p_bb.handle, z, E_st, sh))
        tdk_ms = timed(lambda: nat.rtis_beamform_td(p_td.handle, a, E_st, sh))
    nat.rtis_process(p_fd.handle, x, E_fd, sh)
    torch.cuda.synchronize()
    for p_ in (p_bb, p_td, p_fd):
        assert p_.sync() == 0
    peak = float(E_fd.abs().max())
    err_fd = float((E_bb - E_fd).abs().max()) / peak
    err_td_fd = float((E_td - E_fd).abs().max()) / peak
    t_bb, t_td = sum(bb_ms) / 1e3, sum(td_ms) / 1e3
    if world > 1:
        t_bb, t_td = max_over_ranks([t_bb, t_td], dev)
    clocks = clk.summary()
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    peak_tf = n_sm * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ_NOMINAL * 1e6 / 1e12
    Nb = N_SAMPLES // 4
    # per (direction, coarse sample, mic): 4 Catmull-Rom taps on (re, im) = 16 flop, and the
    # carrier rotation and accumulation, complex x complex + add = 8 flop
    bb_flops = float(N_DIRS) * Nb * N_MICS * 24
    td_flops = float(N_DIRS) * N_SAMPLES * N_MICS * 4 * 2 * 2
    bbk_s, tdk_s = statistics.mean(bbk_ms) / 1e3, statistics.mean(tdk_ms) / 1e3
    ach = bb_flops / bbk_s / 1e12
    line = {
        "metric": "energyscapes/s, complex-baseband path (demodulated, every 4th sample)",
        "value": replica_rate(args.steps, world, t_bb), "unit": "energyscapes/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_bb / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD.replace("matched filter + time-domain and frequency-domain DAS",
                                                "matched filter + complex-baseband DAS (Q = 4)"),
                   "l2": "flushed between steps (512 MiB write, then a 256 MiB read so write-backs finish), "
                         "outside the timed events"},
        "td_rtis_process": {"value": replica_rate(args.steps, world, t_td), "unit": "energyscapes/s",
                            "ms_per_step": 1e3 * t_td / args.steps},
        "speedup_bb_over_td_chain": t_td / t_bb,
        "beamformer_ms": {"bb_beamform_kernel": bbk_s * 1e3, "td_beamform_kernel": tdk_s * 1e3,
                          "speedup": tdk_s / bbk_s},
        "max_abs_diff_over_peak_vs_exact_delay_fd": {"bb": err_fd, "td": err_td_fd},
        "roofline": {"bound": "alu", "kernel": "bb_beamform_kernel", "achieved": ach, "peak": peak_tf,
                     "unit": "TFLOP/s", "frac": ach / peak_tf, "traffic": BB_TRAFFIC_BYTES,
                     "peak_basis": f"{n_sm} SMs x {FP32_LANES_PER_SM} FP32 FMA lanes x 2 flop x "
                                   f"{SM_MAX_MHZ_NOMINAL:.0f} MHz",
                     "algorithmic_flops_per_launch": bb_flops, "launch_ms": bbk_s * 1e3,
                     "tuned_variant_grid": [p_bb.info.bb_variant, p_bb.info.bb_grid],
                     "td_beamform_kernel": {"flops": td_flops, "frac": td_flops / tdk_s / 1e12 / peak_tf}},
        "gpu_launches": 3 * args.steps,
        "clocks": clocks,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    for p_ in (p_bb, p_td, p_fd):
        p_.close()


def run_pdm(args, rank, world, local):
    """The PDM front end ahead of the time-domain chain: each step demodulates one
    hemisphere measurement's 1-bit stream (32 mics x 163840 ticks, one uint32 word per
    tick) into int16 and runs rtis_process on it."""
    import torch
    import torch.distributed as dist

    import synth
    from paper_2208_10839_gb300 import Plan, _native as nat
    from paper_2208_10839_gb300 import build as _b
    _b.build()
    dev = torch.device("cuda", local)
    cfg = synth.hemisphere_pdm(seed_scene=1 + 1000 * rank)
    D = cfg["decim"]
    plan = Plan(cfg["mic_xyz"], cfg["fs"], cfg["chirp"], cfg["dirs"], cfg["n_samples"])
    words = torch.from_numpy(cfg["words"].view(np.int32)).to(dev)
    K = int(words.numel())
    x = torch.empty((N_MICS, N_SAMPLES), dtype=torch.int16, device=dev)
    E = torch.empty((N_DIRS, plan.n_out), dtype=torch.float32, device=dev)
    flush = L2Flush(dev)
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream

    def timed(fn):
        for _ in range(args.warmup):
            flush(1.0)
            fn()
        torch.cuda.synchronize()
        ms = []
        for k in range(args.steps):
            flush(float(k))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            ms.append((e0, e1))
        torch.cuda.synchronize()
        return [q.elapsed_time(r) for q, r in ms]

    def demod():
        nat.rtis_pdm_demodulate(words, K, N_MICS, N_SAMPLES, D, None, 0, x, sh)

    def chain():
        demod()
        nat.rtis_process(plan.handle, x, E, sh)

    if world > 1:
        dist.barrier()
    with ClockSampler(local) as clk:
        chain_ms = timed(chain)
        demod_ms = timed(demod)
        td_ms = timed(lambda: nat.rtis_process(plan.handle, x, E, sh))
    torch.cuda.synchronize()
    assert plan.sync() == 0
    t_chain = sum(chain_ms) / 1e3
    if world > 1:
        (t_chain,) = max_over_ranks([t_chain], dev)
    dm = statistics.mean(demod_ms) / 1e3
    bytes_alg = K * 4 + N_MICS * N_SAMPLES * 2        # the words once, the int16 recording once
    peaks = load_peaks()
    hbm = float(peaks.get("hbm_gbs", 6773.0))
    line = {
        "metric": "energyscapes/s from 1-bit PDM words (demodulation + time-domain chain)",
        "value": replica_rate(args.steps, world, t_chain), "unit": "energyscapes/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_chain / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "i32 (demodulation), f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD.replace("int16; matched filter + time-domain and frequency-domain DAS",
                                                "second-order sigma-delta PDM at 4.5 MHz (uint32 word per tick); "
                                                "order-4 CIC demodulation by 10 + time-domain chain"),
                   "l2": "flushed between steps (512 MiB write, then a 256 MiB read so write-backs finish), "
                         "outside the timed events"},
        "pdm_demod": {"kernel": "pdm_demod_kernel", "ms": dm * 1e3, "bound": "hbm",
                      "achieved_gbs": bytes_alg / dm / 1e9, "peak_gbs": hbm, "frac": bytes_alg / dm / 1e9 / hbm,
                      "algorithmic_bytes": bytes_alg,
                      "note": "1.7 MB per launch: launch- and latency-bound at this size"},
        "td_rtis_process_ms": statistics.mean(td_ms),
        "gpu_launches": 4 * args.steps,
        "clocks": clk.summary(),
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    plan.close()


def run_fd_many(args, rank, world, local):
    """The frequency-domain path alone over --batch hemisphere measurements per step
    (rtis_process_many): batched matched filters, the steering GEMM with the measurements as
    frames, and the IFFT/envelope/low-pass kernel reading its output.  Used for profiling."""
    import torch
    import torch.distributed as dist

    import synth
    from paper_2208_10839_gb300 import Plan
    from paper_2208_10839_gb300 import build as _b
    _b.build()
    dev = torch.device("cuda", local)
    B = args.batch
    cfgs = [synth.hemisphere(seed_scene=1 + 1000 * rank + i) for i in range(B)]
    cfg = cfgs[0]
    plan = Plan(cfg["mic_xyz"], cfg["fs"], cfg["chirp"], cfg["dirs"], cfg["n_samples"], max_batch=B, path="fd",
                fd_ifft=args.fd_ifft)
    x = torch.from_numpy(np.stack([c["x"] for c in cfgs])).to(dev)
    E = torch.empty((B, N_DIRS, plan.n_out), dtype=torch.float32, device=dev)
    flush = L2Flush(dev)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        flush(1.0)
        plan.process_many(x, paths=("fd",), out_fd=E)
    torch.cuda.synchronize()
    assert plan.sync() == 0
    plan.set_tracing(True)
    evs, traces = [], []
    if world > 1:
        dist.barrier()
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            flush(float(k))
            e = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
            e[0].record(stream)
            plan.process_many(x, paths=("fd",), out_fd=E)
            e[1].record(stream)
            traces.append(plan.trace())
            evs.append(e)
        torch.cuda.synchronize()
    plan.set_tracing(False)
    assert plan.sync() == 0
    t = sum(a.elapsed_time(b) for a, b in evs) / 1e3
    if world > 1:
        (t,) = max_over_ranks([t], dev)
    launch = {}
    for tr in traces:
        for name, ms in tr:
            launch.setdefault(name, []).append(ms)
    P = plan.info.fft_len // 4
    fdes_flops = float(N_DIRS) * (4 * 5.0 * P * np.log2(P) + 3 * 6.0 * plan.Kb + 3.0 * N_SAMPLES + 2.0 * 41 * plan.n_out)
    fdes_ms = statistics.mean(launch["fd_energyscape"])
    peak_tf = _fp32_peak_tflops(dev)
    line = {
        "metric": "frequency-domain energyscapes/s at 32ch x 16384 samples x 2048 dirs",
        "value": replica_rate(args.steps * B, world, t), "unit": "energyscapes/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD.replace("time-domain and frequency-domain DAS", "frequency-domain DAS"),
                   "batch_per_step": B, "l2": "flushed between steps, outside the timed events"},
        "kernel_ms_per_step": {k: sum(v) / args.steps for k, v in launch.items()},
        "roofline": {"bound": "alu", "kernel": "fd_energyscape_kernel", "achieved": fdes_flops * B / fdes_ms / 1e9,
                     "peak": peak_tf, "unit": "TFLOP/s", "frac": fdes_flops * B / fdes_ms / 1e9 / peak_tf,
                     "launch_ms": fdes_ms, "algorithmic_flops_per_launch": fdes_flops * B,
                     "timing": "the library's CUDA events around this kernel's launches (rtis tracing)"},
        "gpu_launches": args.steps * 5,
        "clocks": clk.summary(),
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    plan.close()


def run_hemisphere_batched(args, rank, world, local):
    """B measurements per step through rtis_process_many: per measurement the matched
    filter and the time-domain energyscape, and for the whole batch the frequency-domain
    energyscapes via one tcgen05 GEMM with the measurements as frames."""
    import torch
    import torch.distributed as dist

    import synth
    from paper_2208_10839_gb300 import Plan, _native as nat
    from paper_2208_10839_gb300 import build as _b
    _b.build()
    dev = torch.device("cuda", local)
    B = args.batch
    cfgs = [synth.hemisphere(seed_scene=1 + 1000 * rank + i) for i in range(B)]
    cfg = cfgs[0]
    plan = Plan(cfg["mic_xyz"], cfg["fs"], cfg["chirp"], cfg["dirs"], cfg["n_samples"], max_batch=B,
                fd_ifft=args.fd_ifft)
    h = plan.handle
    xs_host = np.stack([c["x"] for c in cfgs])
    x = torch.from_numpy(xs_host).to(dev)
    shape = (B, N_DIRS, plan.n_out)
    E_td = torch.empty(shape, dtype=torch.float32, device=dev)
    E_fd = torch.empty(shape, dtype=torch.float32, device=dev)
    flush = L2Flush(dev)
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream

    def step():
        nat.rtis_process_many(h, x, B, E_td, E_fd, sh)

    for _ in range(args.warmup):
        flush(1.0)
        step()
    torch.cuda.synchronize()
    assert plan.sync() == 0
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    # the library's own CUDA events around each of its launches in every timed step (rtis
    # tracing, on this stream); a step's trace is read after its end event is recorded
    plan.set_tracing(True)
    traces = []
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            flush(float(k))
            evs[k][0].record(stream)
            step()
            evs[k][1].record(stream)
            traces.append(plan.trace())
        torch.cuda.synchronize()
    plan.set_tracing(False)
    step_ms = [a.elapsed_time(b) for a, b in evs]
    t_total = sum(step_ms) / 1e3
    assert plan.sync() == 0
    launch_ms = {}
    for tr in traces:
        for name, ms in tr:
            launch_ms.setdefault(name, []).append(ms)

    # breakdown, same calls split by path, and the beamformer kernels alone (per launch)
    nb = max(3, min(args.steps, 10))
    brk = {"td_path": [], "fd_path": [], "matched_filter": [], "td_beamform": []}
    a = torch.empty((N_MICS, N_SAMPLES), dtype=torch.complex64, device=dev)
    for k in range(nb):
        flush(float(k))
        e = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
        e[0].record(stream)
        nat.rtis_process_many(h, x, B, E_td, None, sh)
        e[1].record(stream)
        nat.rtis_process_many(h, x, B, None, E_fd, sh)
        e[2].record(stream)
        nat.rtis_matched_filter(h, x[k % B], a, None, sh)
        e[3].record(stream)
        nat.rtis_beamform_td(h, a, E_td[k % B], sh)
        e[4].record(stream)
        torch.cuda.synchronize()
        for name, i in (("td_path", 0), ("fd_path", 1), ("matched_filter", 2), ("td_beamform", 3)):
            brk[name].append(e[i].elapsed_time(e[i + 1]))
    bk = {k: statistics.median(v) for k, v in brk.items()}
    td_ms = bk["td_beamform"]  # one single-measurement launch (the batched launches are a little faster)
    assert plan.sync() == 0

    # end to end: pinned host batch in, both energyscape batches out, every step;
    # copies on their own streams, two buffer sets, overlapping the next batch
    hs, cs, cs2, ks = (torch.cuda.Stream(device=dev) for _ in range(4))
    ksh = ks.cuda_stream
    xh = torch.from_numpy(xs_host).pin_memory()
    Eh_td = [torch.empty(shape, dtype=torch.float32).pin_memory() for _ in range(2)]
    Eh_fd = [torch.empty(shape, dtype=torch.float32).pin_memory() for _ in range(2)]
    xd = [x, torch.empty_like(x)]
    Ed_td = [E_td, torch.empty_like(E_td)]
    Ed_fd = [E_fd, torch.empty_like(E_fd)]
    ev_in, ev_done, ev_out, ev_out2 = ([torch.cuda.Event() for _ in range(2)] for _ in range(4))
    ks.wait_stream(stream)
    for e_ in ev_done + ev_out + ev_out2:
        e_.record(ks)

    copy_ev = []  # per timed e2e step: events around its compute and its two D2H copies
    h2d_ev = []   # per timed e2e step: events around its H2D

    def h2d(i, timed):
        # step i's input into buffer i & 1, once the compute that last read that buffer is done
        b = i & 1
        hs.wait_event(ev_done[b])
        e = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) if timed else None
        with torch.cuda.stream(hs):
            if e:
                e[0].record(hs)
            xd[b].copy_(xh, non_blocking=True)
            if e:
                e[1].record(hs)
        ev_in[b].record(hs)
        if e:
            h2d_ev.append(e)

    def e2e_step(i, n, timed):
        # step i: the next step's H2D is queued before this step's D2H copies, which wait for
        # this step's compute; the copy engines run their queues in order, so queued behind
        # them the next input would hold up the next step's compute
        b = i & 1
        ce = [torch.cuda.Event(enable_timing=True) for _ in range(6)] if timed else None
        if i + 1 < n:
            h2d(i + 1, timed)
        ks.wait_event(ev_in[b])
        ks.wait_event(ev_out[b])
        ks.wait_event(ev_out2[b])
        if ce:
            ce[4].record(ks)
        nat.rtis_process_many(h, xd[b], B, Ed_td[b], Ed_fd[b], ksh)
        if ce:
            ce[5].record(ks)
        ev_done[b].record(ks)
        cs.wait_event(ev_done[b])
        cs2.wait_event(ev_done[b])
        with torch.cuda.stream(cs):
            if ce:
                ce[0].record(cs)
            Eh_td[b].copy_(Ed_td[b], non_blocking=True)
            if ce:
                ce[1].record(cs)
        with torch.cuda.stream(cs2):
            if ce:
                ce[2].record(cs2)
            Eh_fd[b].copy_(Ed_fd[b], non_blocking=True)
            if ce:
                ce[3].record(cs2)
        ev_out[b].record(cs)
        ev_out2[b].record(cs2)
        if ce:
            copy_ev.append(ce)

    def run_e2e(n, timed):
        h2d(0, timed)
        for i in range(n):
            e2e_step(i, n, timed)

    run_e2e(2, False)
    torch.cuda.synchronize()
    e2e_steps = max(args.steps // 2, 3)
    ee0, ee1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ee0.record(ks)
    for c in (hs, cs, cs2):
        c.wait_event(ee0)
    run_e2e(e2e_steps, True)
    for e_ in ev_out + ev_out2:
        ks.wait_event(e_)
    ee1.record(ks)
    torch.cuda.synchronize()
    t_e2e = ee0.elapsed_time(ee1) / 1e3
    assert torch.equal(Eh_td[0], Eh_td[1]) and torch.equal(Eh_fd[0], Eh_fd[1])
    assert plan.sync() == 0
    link = pinned_link_gbs(cs, xh, xd[1], Ed_td[0], Eh_td[0])
    # the same copies' durations inside the loop, where they overlap compute and each other
    link["in_loop_ms_per_step"] = {
        name: statistics.median(ce[a].elapsed_time(ce[a + 1]) for ce in copy_ev)
        for name, a in (("d2h_td", 0), ("d2h_fd", 2), ("compute", 4))}
    link["in_loop_ms_per_step"]["h2d"] = statistics.median(e[0].elapsed_time(e[1]) for e in h2d_ev)
    # idle time of the compute stream between one step's compute and the next one's
    gaps = [copy_ev[i][5].elapsed_time(copy_ev[i + 1][4]) for i in range(len(copy_ev) - 1)]
    link["compute_gap_ms"] = {"mean": statistics.mean(gaps), "max": max(gaps)} if gaps else None
    link["compute_ms_mean"] = statistics.mean(ce[4].elapsed_time(ce[5]) for ce in copy_ev)
    link["before_first_compute_ms"] = ee0.elapsed_time(copy_ev[0][4])
    link["after_last_compute_ms"] = copy_ev[-1][5].elapsed_time(ee1)
    link["e2e_ms_per_step"] = 1e3 * t_e2e / e2e_steps

    if world > 1:
        t_total, t_e2e = max_over_ranks([t_total, t_e2e], dev)
    value = replica_rate(args.steps * B, world, t_total)
    e2e_value = replica_rate(e2e_steps * B, world, t_e2e)
    clocks = clk.summary()

    props = torch.cuda.get_device_properties(dev)
    n_sm = props.multi_processor_count
    peak_tf = n_sm * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ_NOMINAL * 1e6 / 1e12
    basis = f"{n_sm} SMs x {FP32_LANES_PER_SM} FP32 FMA lanes x 2 flop x {SM_MAX_MHZ_NOMINAL:.0f} MHz"
    timing = "the library's CUDA events around this kernel's launches in every timed step (rtis tracing)"
    # time-domain beamformer: launches of 16 measurements (the step's last one may hold fewer)
    per_td = [min(16, B - 16 * i) for i in range((B + 15) // 16)]
    td_flops = float(N_DIRS) * N_SAMPLES * N_MICS * 4 * 2 * 2  # per measurement
    td_launch = launch_ms.get("td_beamform", [float("nan")])
    td_meas_ms = sum(td_launch) / (args.steps * B)  # per measurement
    ach = td_flops / (td_meas_ms / 1e3) / 1e12
    roofline = {"bound": "alu", "kernel": "td_beamform_kernel", "achieved": ach, "peak": peak_tf, "unit": "TFLOP/s",
                "frac": ach / peak_tf, "traffic": TD_TRAFFIC_BYTES, "peak_basis": basis,
                "algorithmic_flops_per_launch": td_flops * per_td[0], "launch_ms": statistics.mean(td_launch),
                "measurements_per_launch": per_td, "timing": timing,
                "single_measurement_launch_ms": td_ms,
                "single_measurement_frac": td_flops / (td_ms / 1e3) / 1e12 / peak_tf}
    # frequency-domain path: the steering GEMM (HBM-bound: X in, Y out) and the IFFTs from Y
    P = plan.info.fft_len // 4
    fdes_flops = float(N_DIRS) * (4 * 5.0 * P * np.log2(P) + 3 * 6.0 * plan.Kb + 3.0 * N_SAMPLES
                                  + 2.0 * 41 * plan.n_out)  # per measurement
    fdes_ms = statistics.mean(launch_ms.get("fd_energyscape", [float("nan")]))
    gemm_ms = statistics.mean(launch_ms.get("fd_gemm", [float("nan")]))
    gemm_bytes = float(plan.Kb) * N_MICS * B * 8 + float(plan.Kb) * N_DIRS * B * 8
    hbm = load_peaks().get("hbm_gbs")
    # the IFFT kernel's memory side: Y read once (K_b x D complex per measurement), E written once
    fdes_bytes = (float(plan.Kb) * N_DIRS * 8 + float(N_DIRS) * plan.n_out * 4) * B
    fdes_gbs = fdes_bytes / (fdes_ms / 1e3) / 1e9
    rooflines_other = {
        "fd_energyscape_kernel": {"bound": "alu", "achieved": fdes_flops * B / (fdes_ms / 1e3) / 1e12, "peak": peak_tf,
                                  "unit": "TFLOP/s", "frac": fdes_flops * B / (fdes_ms / 1e3) / 1e12 / peak_tf,
                                  "launch_ms": fdes_ms, "measurements_per_launch": B,
                                  "algorithmic_flops_per_launch": fdes_flops * B, "timing": timing,
                                  "hbm": {"algorithmic_bytes_per_launch": fdes_bytes, "achieved": fdes_gbs,
                                          "peak": hbm, "unit": "GB/s",
                                          "frac": fdes_gbs / hbm if hbm else None}},
        "fd_gemm_kernel": {"bound": "hbm", "achieved": gemm_bytes / (gemm_ms / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
                           "frac": gemm_bytes / (gemm_ms / 1e3) / 1e9 / hbm if hbm else None, "launch_ms": gemm_ms,
                           "algorithmic_bytes_per_launch": gemm_bytes, "precision": "fp32 (3 x bf16)",
                           "peak_source": "MEASURED_PEAKS.json hbm_gbs", "timing": timing},
    }
    share = {k: sum(v) / (args.steps) for k, v in launch_ms.items()}
    line = {
        "metric": METRIC, "value": value, "unit": "energyscapes/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_mics": N_MICS, "n_samples": N_SAMPLES, "n_dirs": N_DIRS,
                   "n_out": plan.n_out, "decim": 10, "batch_per_step": B,
                   "paths_per_step": "time-domain (Catmull-Rom) and frequency-domain (phase ramp, batched "
                                     "tcgen05 GEMM over the step's measurements) energyscapes of every "
                                     "measurement; value counts measurements",
                   "l2": "flushed between steps (512 MiB write, then a 256 MiB read so write-backs finish), "
                         "outside the timed events; the step's GEMM output (4.6 GB) exceeds L2 anyway",
                   "parallelism": f"{world} independent replica(s), {B} measurements per rank per step"},
        "e2e": {"value": e2e_value, "unit": "energyscapes/s", "h2d_bytes_per_step": int(x.numel() * 2),
                "d2h_bytes_per_step": int(E_td.numel() * 4 + E_fd.numel() * 4), "calls": "rtis_process_many",
                "pipelining": "H2D and D2H on their own streams, two buffer sets; copies overlap the next step",
                "pinned_link": link},
        "gpu_launches": args.steps * (2 + (B + 15) // 16 + 3),
        "kernels_ms": {"td_path_per_measurement": bk["td_path"] / B,
                       "fd_path_per_measurement": bk["fd_path"] / B,
                       "td_beamform_single_launch": td_ms,
                       "matched_filter_single_call": bk["matched_filter"],
                       "note": "td_path = batched matched filters + TD beamformer; fd_path = batched matched "
                               "filters + GEMM + per-direction IFFTs; the two share one matched filter per "
                               "measurement in the timed step"},
        "roofline": roofline,
        "rooflines_other": rooflines_other,
        "kernel_ms_per_step": share,
        "clocks": clocks,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        t_es, t_mf, t_das, pick, o_td, o_fd = oracle_sample(cfg, args.cpu_dirs)
        if not args.no_legs:
            line["precision_and_batching"] = precision_and_batching_legs(dev, flush, cfg, pick, o_td)
        try:
            line["error_vs_oracle"] = oracle_error_entry(pick, {"td": (o_td, E_td[0] if E_td.dim() == 3 else E_td),
                                                                "fd": (o_fd, E_fd[0] if E_fd.dim() == 3 else E_fd)})
        except Exception as exc:  # noqa: BLE001 -- a reporting extra must not cost the GPU measurement
            line["error_vs_oracle"] = {"unavailable": f"{type(exc).__name__}: {exc}"[:300]}
        line["cpu_baseline"] = {"value": 1.0 / t_es, "unit": "energyscapes/s", "cores": 1, "kind": "oracle",
                                "sample": f"FP64 oracle, one process: matched filter on all 32 channels "
                                          f"({t_mf:.2f} s) + time- and frequency-domain DAS/envelope on "
                                          f"{args.cpu_dirs} of {N_DIRS} directions ({t_das:.2f} s), scaled to "
                                          f"{N_DIRS} directions"}
        line["cpu_baseline_all_cores"] = all_cores_baseline(args.cpu_pool_dirs)
    if rank == 0:
        print(json.dumps(line), flush=True)
    plan.close()
    if world > 1:
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# precision and batching legs of the default bench line: each one short, each with its
# own CUDA-event time, roofline fraction and error against the FP64 oracle
# ---------------------------------------------------------------------------
def pinned_link_gbs(stream, h_in, d_in, d_out, h_out, reps=3):
    """Bandwidth of this box's pinned host copies, measured alone on one stream with CUDA
    events (the host side of the end-to-end figure): H2D of the input batch, D2H of one
    energyscape batch."""
    import torch
    out = {}
    for name, dst, src in (("h2d_gbs", d_in, h_in), ("d2h_gbs", h_out, d_out)):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            dst.copy_(src, non_blocking=True)
            e0.record(stream)
            for _ in range(reps):
                dst.copy_(src, non_blocking=True)
            e1.record(stream)
        e1.synchronize()
        out[name] = reps * src.numel() * src.element_size() / (e0.elapsed_time(e1) / 1e3) / 1e9
    out["how"] = "pinned host buffers, one stream, CUDA events, best effort (other copies idle)"
    return out


def _timed(fn, flush, stream, reps):
    """CUDA-event milliseconds of fn() per rep, L2 flushed before each (outside the events)."""
    import torch
    out = []
    for k in range(reps):
        flush(float(k))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        out.append(e0.elapsed_time(e1))
    return out


def _fp32_peak_tflops(dev):
    import torch
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    return n_sm * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ_NOMINAL * 1e6 / 1e12


def _rows_error(got_rows, ref_rows):
    ref = np.asarray(ref_rows, dtype=np.float64)
    got = np.asarray(got_rows, dtype=np.float64)
    return {"max_abs_err_over_peak": float(np.max(np.abs(got - ref)) / ref.max()),
            "peak_index_match": bool(np.argmax(got) == np.argmax(ref))}


def leg_fd_gemm(dev, flush, precision, reps):
    """The 1200-bin x 2048-dir x 32-mic x 64-frame steering GEMM in one precision."""
    import torch

    import oracle
    import synth
    from paper_2208_10839_gb300 import FdGemm
    cfg = synth.gemm_frames()
    K, M, T = cfg["X"].shape
    D = cfg["dirs"].shape[0]
    stream = torch.cuda.current_stream()
    with FdGemm(cfg["mic_xyz"], cfg["dirs"], cfg["freqs"], T, precision=precision) as g:
        X = torch.from_numpy(cfg["X"].astype(np.complex64)).to(dev)
        Y = torch.empty((K, D, T), dtype=torch.complex64, device=dev)
        g.run(X, Y)
        ms = statistics.median(_timed(lambda: g.run(X, Y), flush, stream, reps))
        picks = sorted({0, K // 4, K // 2, (3 * K) // 4, K - 1})
        Ys = Y[picks].cpu().numpy().astype(np.complex128)
    W = oracle.steering_matrix(cfg["freqs"][picks], cfg["mic_xyz"], cfg["dirs"], cfg["c"])
    Yr = oracle.fd_gemm(W, cfg["X"][picks].astype(np.complex64).astype(np.complex128))
    bytes_alg = K * M * T * 8 + K * D * T * 8
    hbm = load_peaks().get("hbm_gbs")
    gbs = bytes_alg / (ms / 1e3) / 1e9
    return {"precision": precision, "launch_ms": ms, "frames_per_s": T / (ms / 1e3),
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm if hbm else None,
                         "algorithmic_bytes_per_launch": bytes_alg, "peak_source": "MEASURED_PEAKS.json hbm_gbs"},
            "tensor_tflops": 8.0 * K * D * M * T * (3 if precision == "fp32" else 1) / (ms / 1e3) / 1e12,
            "error_vs_fp64_oracle": {"max_abs_over_max_abs": float(np.max(np.abs(Ys - Yr)) / np.max(np.abs(Yr))),
                                     "bins_checked": picks}}


def leg_td_storage(dev, flush, cfg, pick, o_td, precision, reps):
    """The hemisphere measurement through rtis_process on the time-domain path with the
    analytic signal stored in `precision` (FP32 arithmetic either way)."""
    import torch

    from paper_2208_10839_gb300 import Plan
    stream = torch.cuda.current_stream()
    x = torch.from_numpy(cfg["x"]).to(dev)
    with Plan(cfg["mic_xyz"], cfg["fs"], cfg["chirp"], cfg["dirs"], cfg["n_samples"], precision=precision) as p:
        E = p.process(x)
        p.set_tracing(True)
        chain, td = [], []
        for k in range(reps):
            chain += _timed(lambda: p.process(x, E), flush, stream, 1)
            td += [ms for name, ms in p.trace() if name == "td_beamform"]
        assert p.sync() == 0
        got = E.cpu().numpy()[pick]
    flops = float(N_DIRS) * N_SAMPLES * N_MICS * 16
    peak = _fp32_peak_tflops(dev)
    td_ms = statistics.median(td)
    return {"storage": precision, "chain_ms": statistics.median(chain), "energyscapes_per_s": 1e3 / statistics.median(chain),
            "td_beamform_ms": td_ms,
            "roofline": {"bound": "alu", "achieved": flops / td_ms / 1e9, "peak": peak, "unit": "TFLOP/s",
                         "frac": flops / td_ms / 1e9 / peak},
            "error_vs_fp64_oracle": dict(_rows_error(got, o_td), directions_sampled=int(len(pick)))}


def leg_ring(dev, flush, precision, reps):
    """8 sensors with ragged N and D in one autotuned, graph-replayed batch."""
    import torch

    import oracle
    import synth
    from paper_2208_10839_gb300 import Batch, Plan
    ring = synth.ring_sensors()
    sensors = ring["sensors"]
    stream = torch.cuda.current_stream()
    plans = [Plan(s["mic_xyz"], s["fs"], s["chirp"], s["dirs"], s["n_samples"], precision=precision) for s in sensors]
    try:
        xs = [torch.from_numpy(s["x"]).to(dev) for s in sensors]
        outs = [torch.empty((p.D, p.n_out), dtype=torch.float32, device=dev) for p in plans]
        with Batch(plans) as batch:
            batch.run(xs, outs)  # autotunes, then graph replays
            batch.run(xs, outs)
            ms = statistics.median(_timed(lambda: batch.run(xs, outs), flush, stream, reps))
            assert batch.sync() == 0
            info = batch.info
        i_big = int(np.argmax([s["n_samples"] * s["dirs"].shape[0] for s in sensors]))
        s = sensors[i_big]
        rows = np.arange(0, s["dirs"].shape[0], s["dirs"].shape[0] // 8)[:8]
        got = outs[i_big].cpu().numpy()[rows]
    finally:
        for p in plans:
            p.close()
    a = oracle.matched_filter(s["x"], s["chirp"], s["fs"])
    ref = oracle.envelope_decimate(oracle.das_td(a, oracle.steering_delays(s["mic_xyz"], s["dirs"][rows], s["fs"],
                                                                           s["c"])), oracle.lpf_taps())
    flops = float(sum(x["dirs"].shape[0] * x["n_samples"] for x in sensors)) * N_MICS * 16
    peak = _fp32_peak_tflops(dev)
    return {"storage": precision, "batch_ms": ms, "energyscapes_per_s": len(sensors) / (ms / 1e3),
            "beamformer_ms_autotuned": info.tuned_ms, "tiles": info.total_tiles,
            "roofline_beamformer": {"bound": "alu", "achieved": flops / info.tuned_ms / 1e9, "peak": peak,
                                    "unit": "TFLOP/s", "frac": flops / info.tuned_ms / 1e9 / peak},
            "error_vs_fp64_oracle": dict(_rows_error(got, ref), sensor=i_big, directions_sampled=len(rows),
                                         n_samples=int(s["n_samples"]))}


def leg_calibration(dev, flush, reps):
    """One self-calibration gradient (energyscape, L2 loss, adjoint) of the perturbed array; the
    gradient's error against the FP64 oracle's on a cotangent that lives on 16 directions."""
    import torch

    import oracle
    import synth
    from paper_2208_10839_gb300 import Plan
    cfg = synth.calibration()
    stream = torch.cuda.current_stream()
    with Plan(cfg["mic_nominal"], cfg["fs"], cfg["chirp"], cfg["dirs"], cfg["n_samples"], c=cfg["c"]) as p:
        x = torch.from_numpy(cfg["x"]).to(dev)
        E_ref = p.process(torch.from_numpy(cfg["x_ref"]).to(dev)).clone()
        E = torch.empty_like(E_ref)
        G = torch.empty_like(E_ref)
        loss = torch.empty(1, dtype=torch.float32, device=dev)

        def step():
            p.process(x, E)
            from paper_2208_10839_gb300 import _native as nat
            nat.rtis_loss_l2(p.handle, E, E_ref, G, loss, None)
            p.backward(x, G)

        step()
        p.set_tracing(True)
        tot, adj = [], []
        for k in range(reps):
            flush(float(k))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            p.process(x, E)
            from paper_2208_10839_gb300 import _native as nat
            nat.rtis_loss_l2(p.handle, E, E_ref, G, loss, None)
            p.backward(x, G)
            e1.record(stream)
            adj += [ms for name, ms in p.trace() if name == "adjoint"]
            torch.cuda.synchronize()
            tot.append(e0.elapsed_time(e1))
        # gradient accuracy: a cotangent on 16 sampled directions
        rng = np.random.default_rng(1)
        pick = np.sort(rng.choice(p.D, 16, replace=False))
        Gs = np.zeros((p.D, p.n_out), dtype=np.float32)
        Gs[pick] = rng.standard_normal((16, p.n_out)).astype(np.float32)
        gx, gg, gd = p.backward(x, torch.from_numpy(Gs).to(dev))
        got = [v.cpu().numpy().astype(np.float64) for v in (gx, gg, gd)]
        assert p.sync() == 0
    _, gx_r, gg_r, gd_r = oracle.energyscape_vjp(cfg["x"], cfg["chirp"], cfg["mic_nominal"], cfg["dirs"][pick],
                                                 cfg["fs"], cfg["c"], Gs[pick].astype(np.float64))
    err = {name: float(np.max(np.abs(g - r)) / np.max(np.abs(r)))
           for name, g, r in (("xyz", got[0], gx_r), ("gain", got[1], gg_r), ("delay", got[2], gd_r))}
    flops = float(N_DIRS) * N_SAMPLES * N_MICS * 32
    peak = _fp32_peak_tflops(dev)
    adj_ms = statistics.median(adj)
    return {"step_ms": statistics.median(tot), "gradients_per_s": 1e3 / statistics.median(tot), "adjoint_ms": adj_ms,
            "roofline_adjoint": {"bound": "alu", "achieved": flops / adj_ms / 1e9, "peak": peak, "unit": "TFLOP/s",
                                 "frac": flops / adj_ms / 1e9 / peak},
            "gradient_error_vs_fp64_oracle": dict(err, tolerance=1e-6, directions_in_cotangent=16,
                                                  note="max |g - g64| / max |g64| per quantity")}


def precision_and_batching_legs(dev, flush, cfg, pick, o_td, reps=5):
    """The forms the default line compares with plain FP32: every leg fails on its own."""
    out = {}
    legs = [("fd_gemm_bf16", lambda: leg_fd_gemm(dev, flush, "bf16", reps)),
            ("fd_gemm_fp16", lambda: leg_fd_gemm(dev, flush, "fp16", reps)),
            ("fd_gemm_fp32", lambda: leg_fd_gemm(dev, flush, "fp32", reps)),
            ("td_fp32_storage", lambda: leg_td_storage(dev, flush, cfg, pick, o_td, "fp32", reps)),
            ("td_bf16_storage", lambda: leg_td_storage(dev, flush, cfg, pick, o_td, "bf16", reps)),
            ("ring_fp32", lambda: leg_ring(dev, flush, "fp32", reps)),
            ("ring_bf16", lambda: leg_ring(dev, flush, "bf16", reps)),
            ("calibration", lambda: leg_calibration(dev, flush, reps))]
    for name, fn in legs:
        t0 = time.perf_counter()
        try:
            out[name] = fn()
        except Exception as exc:  # noqa: BLE001 -- one leg must not cost the others or the main line
            out[name] = {"unavailable": f"{type(exc).__name__}: {exc}"[:300]}
        out[name]["wall_s"] = round(time.perf_counter() - t0, 2)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-legs", action="store_true",
                    help="default workload: skip the short precision and batching legs (GEMM in BF16/FP16/FP32, "
                         "TD with BF16 storage, the 8-sensor ring in FP32/BF16, a calibration gradient)")
    ap.add_argument("--cpu-pool-dirs", type=int, default=16,
                    help="directions each all-cores oracle worker times (scaled to all directions)")
    ap.add_argument("--cpu-dirs", type=int, default=128, help="directions in the oracle's timed sample")
    ap.add_argument("--workload", default="hemisphere", choices=["hemisphere", "fd_gemm", "ring", "calibration", "paper_design", "stream",
                                                               "fd_many",
                                                               "baseband", "pdm"],
                    help="hemisphere: the energyscape chain (default); fd_gemm: the 1200-bin frequency-domain "
                         "beamforming GEMM (32 mics x 64 frames -> 2048 directions); ring: 8 sensors with "
                         "uneven lengths and direction sets in one autotuned, graph-replayed batch; calibration: "
                         "energyscape + L2 loss + adjoint of a perturbed 32-mic array; paper_design: the "
                         "time-domain chain built the paper's way (cuFFT + per-sample DAS) vs the fused kernels; "
                         "stream: host-to-host streaming through a ring of pinned slots (throughput, latency)")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "bf16", "fp16"])
    ap.add_argument("--fd-ifft", default="auto", choices=["auto", "fft", "tc"],
                    help="batched frequency-domain path: inverse transform as dense DFT stages on the tensor "
                         "cores (tc), as FFTs on the FP32 pipe (fft), or the plan's choice (auto)")
    ap.add_argument("--bins", type=int, default=1200, help="fd_gemm: frequency bins (1200 = the full workload)")
    ap.add_argument("--batch", type=int, default=64,
                    help="hemisphere: measurements per step (1: per-measurement calls; >1: rtis_process_many, "
                         "the frequency-domain form as one batched tensor-core GEMM)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    rank, world, local = dist_env()

    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    import torch.distributed as dist

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if args.workload == "fd_gemm":
        return run_fd_gemm(args, rank, world, local)
    if args.workload == "ring":
        return run_ring(args, rank, world, local)
    if args.workload == "calibration":
        return run_calibration(args, rank, world, local)
    if args.workload == "paper_design":
        return run_paper_design(args, rank, world, local)
    if args.workload == "baseband":
        return run_baseband(args, rank, world, local)
    if args.workload == "pdm":
        return run_pdm(args, rank, world, local)
    if args.workload == "stream":
        return run_stream(args, rank, world, local)
    if args.workload == "fd_many":
        return run_fd_many(args, rank, world, local)
    if args.batch > 1:
        return run_hemisphere_batched(args, rank, world, local)

    import synth
    from paper_2208_10839_gb300 import Plan, _native as nat
    from paper_2208_10839_gb300 import build as _b
    _b.build()

    cfg = synth.hemisphere(seed_scene=1 + 1000 * rank)
    dev = torch.device("cuda", local)
    plan = Plan(cfg["mic_xyz"], cfg["fs"], cfg["chirp"], cfg["dirs"], cfg["n_samples"])
    x = torch.from_numpy(cfg["x"]).to(dev)
    a = torch.empty((N_MICS, N_SAMPLES), dtype=torch.complex64, device=dev)
    A = torch.empty((N_MICS, plan.Kb), dtype=torch.complex64, device=dev)
    E_td = torch.empty((N_DIRS, plan.n_out), dtype=torch.float32, device=dev)
    E_fd = torch.empty((N_DIRS, plan.n_out), dtype=torch.float32, device=dev)
    flush = L2Flush(dev)
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream
    h = plan.handle

    def step(ev=None):
        # one measurement -> matched filter (analytic signal and in-band spectra),
        # time-domain and frequency-domain energyscapes
        if ev:
            ev[0].record(stream)
        nat.rtis_matched_filter(h, x, a, A, sh)
        if ev:
            ev[1].record(stream)
        nat.rtis_beamform_td(h, a, E_td, sh)
        if ev:
            ev[2].record(stream)
        nat.rtis_beamform_fd(h, A, E_fd, sh)
        if ev:
            ev[3].record(stream)

    for _ in range(args.warmup):
        flush(1.0)
        step()
    torch.cuda.synchronize()
    assert plan.sync() == 0

    evs = [tuple(torch.cuda.Event(enable_timing=True) for _ in range(4)) for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            flush(float(k))
            step(evs[k])
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    step_ms = [e[0].elapsed_time(e[3]) for e in evs]
    mf_ms = [e[0].elapsed_time(e[1]) for e in evs]
    td_ms = [e[1].elapsed_time(e[2]) for e in evs]
    fd_ms = [e[2].elapsed_time(e[3]) for e in evs]
    t_total = sum(step_ms) / 1e3
    bits = plan.sync()
    assert bits == 0, f"device status {bits:#x}"

    # end to end through the public calls: pinned host input -> device -> both
    # energyscapes -> pinned host, every step.  Copies run on their own streams
    # (input, and one per energyscape) and two buffer sets alternate, so the
    # copies of one measurement overlap the beamforming of the next; events
    # order each buffer's reuse.
    # both on pool streams: work on the legacy default stream would serialise with the copies
    hs = torch.cuda.Stream(device=dev)   # input copies
    cs = torch.cuda.Stream(device=dev)   # output copies (one stream per energyscape)
    cs2 = torch.cuda.Stream(device=dev)
    ks = torch.cuda.Stream(device=dev)
    ksh = ks.cuda_stream
    xh = torch.from_numpy(cfg["x"]).pin_memory()
    Eh_td = [torch.empty((N_DIRS, plan.n_out), dtype=torch.float32).pin_memory() for _ in range(2)]
    Eh_fd = [torch.empty((N_DIRS, plan.n_out), dtype=torch.float32).pin_memory() for _ in range(2)]
    xd = [torch.empty_like(x) for _ in range(2)]
    Ed_td = [E_td, torch.empty_like(E_td)]
    Ed_fd = [E_fd, torch.empty_like(E_fd)]
    ev_in = [torch.cuda.Event() for _ in range(2)]
    ev_done = [torch.cuda.Event() for _ in range(2)]
    ev_out = [torch.cuda.Event() for _ in range(2)]
    ev_out2 = [torch.cuda.Event() for _ in range(2)]
    ks.wait_stream(stream)
    for e in ev_done + ev_out + ev_out2:
        e.record(ks)

    def e2e_step(i):
        b = i & 1
        hs.wait_event(ev_done[b])  # the beamforming that last read xd[b] has finished
        with torch.cuda.stream(hs):
            xd[b].copy_(xh, non_blocking=True)
        ev_in[b].record(hs)
        ks.wait_event(ev_in[b])
        ks.wait_event(ev_out[b])  # the copies that last read Ed_*[b] have finished
        ks.wait_event(ev_out2[b])
        nat.rtis_matched_filter(h, xd[b], a, A, ksh)
        nat.rtis_beamform_td(h, a, Ed_td[b], ksh)
        nat.rtis_beamform_fd(h, A, Ed_fd[b], ksh)
        ev_done[b].record(ks)
        cs.wait_event(ev_done[b])
        cs2.wait_event(ev_done[b])
        with torch.cuda.stream(cs):
            Eh_td[b].copy_(Ed_td[b], non_blocking=True)
        with torch.cuda.stream(cs2):
            Eh_fd[b].copy_(Ed_fd[b], non_blocking=True)
        ev_out[b].record(cs)
        ev_out2[b].record(cs2)

    for i in range(4):
        e2e_step(i)
    torch.cuda.synchronize()
    ee0, ee1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2e_steps = max(args.steps // 2, 3)
    ee0.record(ks)
    for c in (hs, cs, cs2):
        c.wait_event(ee0)
    for i in range(e2e_steps):
        e2e_step(i)
    for e in ev_out + ev_out2:
        ks.wait_event(e)
    ee1.record(ks)
    torch.cuda.synchronize()
    t_e2e = ee0.elapsed_time(ee1) / 1e3
    # every step beamforms the same measurement, so each host copy must equal the device result
    ref_td, ref_fd = Ed_td[0].cpu(), Ed_fd[0].cpu()
    assert all(torch.equal(hb, ref_td) for hb in Eh_td) and all(torch.equal(hb, ref_fd) for hb in Eh_fd)

    if world > 1:
        t_total, t_e2e = max_over_ranks([t_total, t_e2e], dev)

    value = replica_rate(args.steps, world, t_total)
    e2e_value = replica_rate(e2e_steps, world, t_e2e)
    clocks = clk.summary()

    # rooflines of the two beamformers, both bound by the FP32 ALU (FMA pipe); the
    # JSON's "roofline" is the one that takes longer per step (the dominant kernel)
    props = torch.cuda.get_device_properties(dev)
    n_sm = props.multi_processor_count
    peak_tf = n_sm * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ_NOMINAL * 1e6 / 1e12
    basis = f"{n_sm} SMs x {FP32_LANES_PER_SM} FP32 FMA lanes x 2 flop x {SM_MAX_MHZ_NOMINAL:.0f} MHz"
    td_s = statistics.mean(td_ms) / 1e3
    fd_s = statistics.mean(fd_ms) / 1e3
    P = plan.info.fft_len // 4
    lpf_len = 4 * 10 + 1
    td_flops = float(N_DIRS) * N_SAMPLES * N_MICS * 4 * 2 * 2  # 4 taps x (re, im) FMAs per (d, n, m)
    fd_flops = float(N_DIRS) * (8.0 * plan.Kb * N_MICS                   # steered spectrum: complex MACs
                                + 4 * 5.0 * P * np.log2(P)                # four P-point inverse FFTs
                                + 3 * 6.0 * plan.Kb                        # phase pre-twiddles (q = 1..3)
                                + 3.0 * N_SAMPLES                          # envelope |b|
                                + 2.0 * lpf_len * plan.n_out)              # low-pass at the output bins
    rl = {}
    for name, kern, flops, secs, traffic in (("td", "td_beamform_kernel", td_flops, td_s, TD_TRAFFIC_BYTES),
                                             ("fd", "fd_energyscape_kernel", fd_flops, fd_s, FD_TRAFFIC_BYTES)):
        ach = flops / secs / 1e12
        rl[name] = {"bound": "alu", "kernel": kern, "achieved": ach, "peak": peak_tf, "unit": "TFLOP/s",
                    "frac": ach / peak_tf, "traffic": traffic, "peak_basis": basis,
                    "algorithmic_flops_per_launch": flops, "launch_ms": secs * 1e3}
        if clocks.get("sm_mhz"):
            rl[name]["frac_at_observed_clock"] = ach / (n_sm * FP32_LANES_PER_SM * 2 * clocks["sm_mhz"] * 1e6 / 1e12)
    dominant = "fd" if fd_s > td_s else "td"
    roofline = rl[dominant]

    line = {
        "metric": METRIC, "value": value, "unit": "energyscapes/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_mics": N_MICS, "n_samples": N_SAMPLES, "n_dirs": N_DIRS,
                   "n_out": plan.n_out, "decim": 10, "batch_per_step": 1,
                   "paths_per_step": "time-domain (Catmull-Rom) and frequency-domain (phase ramp) energyscapes "
                                     "of the same measurement; value counts measurements",
                   "l2": "flushed between steps (512 MiB write, then a 256 MiB read so write-backs finish), outside the timed events",
                   "parallelism": f"{world} independent replica(s), one measurement per rank per step"},
        "e2e": {"value": e2e_value, "unit": "energyscapes/s", "h2d_bytes_per_step": int(x.numel() * 2),
                "d2h_bytes_per_step": int(E_td.numel() * 4 + E_fd.numel() * 4),
                "calls": "rtis_matched_filter, rtis_beamform_td, rtis_beamform_fd",
                "pipelining": "H2D and D2H on their own streams, two buffer sets; copies overlap the next step"},
        "gpu_launches": 4 * args.steps,
        "kernels_ms": {"matched_filter": statistics.mean(mf_ms), "td_beamform": statistics.mean(td_ms),
                       "fd_energyscape": statistics.mean(fd_ms)},
        "path_rates": {"td_only_energyscapes_per_s": 1e3 / (statistics.mean(mf_ms) + statistics.mean(td_ms)),
                       "fd_only_energyscapes_per_s": 1e3 / (statistics.mean(mf_ms) + statistics.mean(fd_ms))},
        "roofline": roofline,
        "roofline_other": rl["td" if dominant == "fd" else "fd"],
        "clocks": clocks,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        t_es, t_mf, t_das, pick, o_td, o_fd = oracle_sample(cfg, args.cpu_dirs)
        try:
            line["error_vs_oracle"] = oracle_error_entry(pick, {"td": (o_td, E_td[0] if E_td.dim() == 3 else E_td),
                                                                "fd": (o_fd, E_fd[0] if E_fd.dim() == 3 else E_fd)})
        except Exception as exc:  # noqa: BLE001 -- a reporting extra must not cost the GPU measurement
            line["error_vs_oracle"] = {"unavailable": f"{type(exc).__name__}: {exc}"[:300]}
        line["cpu_baseline"] = {"value": 1.0 / t_es, "unit": "energyscapes/s", "cores": 1, "kind": "oracle",
                                "sample": f"FP64 oracle, one process: matched filter on all 32 channels "
                                          f"({t_mf:.2f} s) + time- and frequency-domain DAS/envelope on "
                                          f"{args.cpu_dirs} of {N_DIRS} directions ({t_das:.2f} s), scaled to "
                                          f"{N_DIRS} directions"}
        line["cpu_baseline_all_cores"] = all_cores_baseline(args.cpu_pool_dirs)
    if rank == 0:
        print(json.dumps(line), flush=True)
    plan.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

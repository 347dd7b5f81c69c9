"""Benchmark: 3D complex FFT through the cyclic four-step method on one GB300.

A step is one forward and one inverse transform of the 512^3 complex64
workload (cyclic grid p = 8x8x8 by default) through the C ABI, i.e. one pass of
the whole hot path in each direction.  Inputs (1 GiB) are larger than L2
(129 MB), so no flush is needed between steps.  Metric: algorithmic HBM GB/s,
B_alg = 4 * N * 8 bytes per transform (one round trip for phase A, one for
phase B), divided by the measured time.

Prints one JSON line (rank 0).  With --impl reference it times the FP64 CPU
oracle instead (the reference arm of this single-GPU tier).
Under torchrun with N > 1, every rank runs its own replica (no collective on
the data path; the method's single all-to-all is not exercised on one node of
replicas) and value is the sum over ranks at the max-over-ranks time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

FALLBACK_HBM_GBS = 6800.0
NOMINAL_HBM_GBS = 8000.0  # the nominal HBM3e figure the target is also quoted against
FP64_PEAK_GFLOPS = 1250.0  # nominal; used only if the device measurement fails
REF_BUDGET_S = 240.0  # wall-time budget of the reference arm's steps  # GB300 FP64 nominal: complex128 transforms are bound by FP64 arithmetic
METRIC = "3D FFT HBM GB/s & % roofline at 512^3 c64; mixed-request p50/p99 latency"
METRIC_DETAIL = ("value: algorithmic HBM GB/s, B_alg = 4 N b bytes per transform (b = element size), "
                 "one forward + one inverse transform per step; the mixed-request p50/p99 latency is the "
                 "'serving' object (native serving loop, Poisson arrivals)")


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--shape", default="512,512,512")
    ap.add_argument("--p", default="8,8,8", help="cyclic grid, or 'tune' to let the plan-time tuner choose")
    ap.add_argument("--serve", action="store_true", help="print only the serving run's line")
    ap.add_argument("--pointwise", action="store_true",
                    help="time forward -> pointwise product -> inverse (fftu_exec_pointwise) instead")
    ap.add_argument("--no-serve", action="store_true", help="leave the serving run out of the default line")
    ap.add_argument("--serve-requests", type=int, default=10000)
    ap.add_argument("--serve-rate", type=float, default=0.0,
                    help="offered Poisson rate, requests per second (0 = 0.7 x the measured saturation rate)")
    ap.add_argument("--serve-warmup", type=int, default=400)
    ap.add_argument("--serve-streams", type=int, default=8)
    ap.add_argument("--serve-inflight", type=int, default=0, help="0 = 2 x streams")
    ap.add_argument("--serve-piece-mib", type=int, default=0, help="host copies in pieces of this many MiB")
    ap.add_argument("--serve-solo", type=int, default=0,
                    help="solo (large) launches in flight at once; 0 = the server's default (one per solo stream)")
    ap.add_argument("--batch-cubes", action="store_true", help="batch of cubes n^3 only (n in 32, 64, 128)")
    ap.add_argument("--batch", type=int, default=0,
                    help="K > 0: time K uneven 3D transforms (n_l in {32, 64, 128}) in one persistent launch "
                         "per direction instead of the single-array workload")
    ap.add_argument("--schedule", type=int, default=0, help="0 auto, 1 generic, 2 fused")
    ap.add_argument("--dtype", choices=["c64", "c128"], default="c64")
    ap.add_argument("--precision", choices=["native", "bf16", "fp16"], default="native",
                    help="radix-16 stages on CUDA cores (native) or as split bf16/fp16 tensor-core contractions")
    ap.add_argument("--inputs", choices=["uniform", "loguniform", "device", "device_loguniform"], default="uniform",
                    help="uniform / loguniform: fftu_inputs on the host; device / device_loguniform: the same "
                         "distributions drawn on the GPU by torch's seeded generator (large secondary runs)")
    ap.add_argument("--tile", type=int, default=0, help="strided-pass tile target (0 = default)")
    ap.add_argument("--radix", type=int, default=0, help="strided-pass stage radix (0 = default)")
    ap.add_argument("--no-secondary", action="store_true",
                    help="leave the secondary configurations out of the default line")
    ap.add_argument("--seed", type=int, default=2024)
    ap.add_argument("--flush-l2", action="store_true",
                    help="write a 256 MB buffer between steps (for arrays that fit in L2); the step time is "
                         "then the sum of the phases' event intervals, the flush excluded")
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--e2e-copy-streams", type=int, default=1, help="streams per copy direction in the e2e run")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cufft", action="store_true", help="leave out the torch.fft (cuFFT) context timing")
    ap.add_argument("--cpu-sample", default="512,512,512", help="oracle sample shape for cpu_baseline")
    ap.add_argument("--cpu-reps", type=int, default=3, help="oracle forward+inverse repetitions for cpu_baseline")
    a = ap.parse_args()
    a.warmup = max(3, a.warmup)
    return a


def shape_of(s):
    return tuple(int(v) for v in s.split(","))


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def alg_bytes(shape, esize):
    return 4 * math.prod(shape) * esize


def device_inputs(shape, t_dtype, seed, dev, loguniform=False):
    """Seeded synthetic inputs drawn on the GPU (torch's Philox generator): Re and Im i.i.d.
    uniform[-1, 1), or (loguniform) magnitudes 10^U[-3, 3) with a uniform phase.  Used for the large
    secondary runs, whose host-side generation would dominate the bench's wall time; the parity tests
    use fftu_inputs' SplitMix64 arrays."""
    import torch
    g = torch.Generator(device=dev)
    g.manual_seed(int(seed))
    real = torch.float32 if t_dtype == torch.complex64 else torch.float64
    n = math.prod(shape)
    u = torch.rand(2 * n, generator=g, device=dev, dtype=real)
    if loguniform:
        mag = torch.pow(10.0, -3.0 + 6.0 * u[0::2])
        ph = 2.0 * math.pi * u[1::2]
        x = torch.polar(mag, ph)
    else:
        x = torch.view_as_complex((2.0 * u - 1.0).view(n, 2))
    x = x.reshape(shape).contiguous()
    del u
    return x


def workload_config(shape, p, esize, args, world):
    """The benchmark's workload: what is computed on which data (the same keys on both arms)."""
    N = math.prod(shape)
    prec = args.precision
    return {"workload": f"{'x'.join(map(str, shape))} complex{'64' if esize == 8 else '128'} "
                        + (f"({prec} split radix-16 stages) " if prec != "native" else "")
                        + f"forward+inverse FFT, cyclic p={'x'.join(map(str, p))}",
            "shape": list(shape), "p": list(p), "inputs": args.inputs, "seed": args.seed,
            "l2": ("L2 flushed between steps (256 MB written); step time = sum of phase events"
                   if args.flush_l2 else
                   "inputs larger than L2 (129 MB); no flush" if N * esize > 129e6 else
                   "inputs smaller than L2: L2-resident, not an HBM measurement"),
            "parallelism": f"replicas x{world}" if world > 1 else "single GPU"}


def oracle_cpu_run(shape, seed, reps=1):
    """Time the FP64 oracle (forward + inverse) on a sample; returns (seconds per fwd+inv, cores)."""
    import numpy as np
    import oracle
    from fftu_inputs import complex_uniform
    x = complex_uniform(seed, shape, dtype=np.complex64).astype(np.complex128)
    cores = oracle.max_threads()
    t0 = time.perf_counter()
    for _ in range(reps):
        y = oracle.fftn(x)
        oracle.fftn(y, inverse=True)
    return (time.perf_counter() - t0) / reps, cores


def torch_cpu_fft_run(shape, seed, reps=3):
    """torch.fft on the host (complex64, torch's own threads): context for the oracle's numbers."""
    import numpy as np
    import torch
    from fftu_inputs import complex_uniform
    x = torch.from_numpy(complex_uniform(seed, shape, dtype=np.complex64))
    torch.fft.ifftn(torch.fft.fftn(x))  # warm-up (plans, allocations)
    t0 = time.perf_counter()
    for _ in range(reps):
        torch.fft.ifftn(torch.fft.fftn(x))
    dt = (time.perf_counter() - t0) / reps
    return {"impl": "torch.fft.fftn + ifftn on the host (complex64)", "threads": torch.get_num_threads(),
            "shape": "x".join(map(str, shape)), "reps": reps, "seconds_per_rep": dt,
            "value": 2 * alg_bytes(shape, 8) / dt / 1e9, "unit": "GB/s",
            "note": "context, not a baseline: an optimized CPU FFT library, not the oracle"}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu_index = gpu_index
        self.proc = None
        self.out = os.path.join("/tmp", f"fftu_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            f = open(self.out, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "100",
                 "-i", str(self.gpu_index)], stdout=f, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.out) as f:
            for line in f:
                parts = [v.strip() for v in line.split(",")]
                if len(parts) >= 9 and parts[1].replace(".", "").isdigit():
                    rows.append(parts)
        os.unlink(self.out)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": float(rows[0][2]), "samples": len(rows),
                "power_w_max": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit()),
                "reasons": reasons}


def traffic_for(kernel):
    """DRAM bytes per launch from the committed ncu summary, if the kernel source is unchanged."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            table = json.load(f)
        ent = table[kernel]
        src = os.path.join(ROOT, ent["source"])
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        if sha != ent["source_sha"]:
            return None
        return float(ent["bytes_per_launch"])
    except Exception:
        return None


def max_over_ranks(ms, device):
    """Slowest rank's time (ms); plain value without a process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(ms)
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(bytes_per_rank, ms, world):
    """Whole-job GB/s: the bytes of every replica over the slowest replica's time."""
    return world * bytes_per_rank / (ms * 1e-3) / 1e9


def run_reference(args):
    """The reference arm: the FP64 CPU oracle, as it stands, on the host cores, on the same workload.

    Each step is one forward + inverse transform of the benchmark's own array (512^3 by default,
    about 2.7 s on 16 Grace cores) when warm-up plus timed steps of it fit REF_BUDGET_S; otherwise
    each step takes the largest power-of-two sub-sample that fits, and the line says so."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    shape = shape_of(args.shape)
    esize = 8 if args.dtype == "c64" else 16
    p = args.p if args.p == "tune" else list(shape_of(args.p))
    total = args.warmup + args.steps
    t_first, cores = oracle_cpu_run(shape, args.seed)  # the first warm-up step, at the full size
    sample = shape
    while t_first * total > REF_BUDGET_S and math.prod(sample) > 1 << 15:
        sample = tuple(max(1, v // 2) for v in sample)
        t_first /= 8.0
    times = []
    for i in range(1, total):
        t, cores = oracle_cpu_run(sample, args.seed)
        if i >= args.warmup:
            times.append(t)
    if not times:
        times = [t_first]
    t = sum(times) / len(times)
    value = 2 * alg_bytes(sample, esize) / t / 1e9
    same = tuple(sample) == tuple(shape)
    line = {
        "metric": METRIC, "metric_detail": METRIC_DETAIL,
        "value": value, "unit": "GB/s", "impl": "reference", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(shape, p, esize, args, 1),
        "cpu_baseline": {"value": value, "unit": "GB/s", "cores": cores, "kind": "oracle",
                         "sample": (f"FP64 oracle (plain row-column FFT, not an optimized library) forward+inverse "
                                    f"of the {'whole ' if same else ''}{'x'.join(map(str, sample))} array per step "
                                    f"(seeded uniform inputs), GB/s from 4*N*{esize} bytes per transform"
                                    + ("" if same else "; a sub-sample, the full array would not fit the budget"))},
        "same_workload_per_step": same,
        "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_2203_11795_gb300 import _build
    _build.build()
    import paper_2203_11795_gb300 as fftu
    from fftu_inputs import complex_uniform

    shape = shape_of(args.shape)
    tune = args.p == "tune"
    p = None if tune else shape_of(args.p)
    N = math.prod(shape)
    np_dtype, t_dtype = (np.complex64, torch.complex64) if args.dtype == "c64" else (np.complex128, torch.complex128)
    esize = 8 if args.dtype == "c64" else 16
    if args.inputs.startswith("device"):
        x = device_inputs(shape, t_dtype, args.seed + rank, dev, loguniform=args.inputs == "device_loguniform")
        x_host = None if args.no_e2e else x.cpu().pin_memory()
    else:
        if args.inputs == "loguniform":
            from fftu_inputs import complex_loguniform
            x_host = torch.from_numpy(complex_loguniform(args.seed + rank, shape, dtype=np_dtype)).pin_memory()
        else:
            x_host = torch.from_numpy(complex_uniform(args.seed + rank, shape, dtype=np_dtype)).pin_memory()
        x = x_host.to(dev)
    prec = {"native": 0, "bf16": 1, "fp16": 2}[args.precision]
    y = torch.empty_like(x)
    z = torch.empty_like(x)
    t_plan = time.perf_counter()
    fwd = fftu.Plan(shape, p, dtype=t_dtype, schedule=args.schedule, tune=tune, precision=prec, tile=args.tile,
                    radix=args.radix)
    inv = fftu.Plan(shape, p, dtype=t_dtype, inverse=True, schedule=args.schedule, tune=tune, precision=prec,
                    tile=args.tile, radix=args.radix)
    t_plan = time.perf_counter() - t_plan
    if tune:
        p = tuple(fwd.info["p"])
    stream = torch.cuda.Stream(dev)
    sh = stream.cuda_stream
    A, B = fftu.FFTU_PHASE_A, fftu.FFTU_PHASE_B

    flush = torch.empty(64 << 20, dtype=torch.float32, device=dev) if args.flush_l2 else None

    def step(ev=None):
        if flush is not None:
            flush.zero_()
        if ev is not None:
            ev[0].record(stream)
        fftu.fftu_exec_phase(fwd.handle, A, x.data_ptr(), y.data_ptr(), sh)
        if ev is not None:
            ev[1].record(stream)
        fftu.fftu_exec_phase(fwd.handle, B, None, y.data_ptr(), sh)
        if ev is not None:
            ev[2].record(stream)
        fftu.fftu_exec_phase(inv.handle, A, y.data_ptr(), z.data_ptr(), sh)
        if ev is not None:
            ev[3].record(stream)
        fftu.fftu_exec_phase(inv.handle, B, None, z.data_ptr(), sh)
        if ev is not None:
            ev[4].record(stream)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
    torch.cuda.synchronize(dev)

    events = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(args.steps)]
    sampler = ClockSampler(local) if rank == 0 else None
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    if sampler:
        sampler.start()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for k in range(args.steps):
        step(events[k])
    t_end.record(stream)
    torch.cuda.synchronize(dev)
    clocks = sampler.stop() if sampler else None
    if world > 1:
        dist.barrier()
    total_ms = t_start.elapsed_time(t_end)
    if flush is not None:  # the flushes are not part of the step
        total_ms = sum(ev[0].elapsed_time(ev[4]) for ev in events)
    phase_a = [ev[0].elapsed_time(ev[1]) for ev in events] + [ev[2].elapsed_time(ev[3]) for ev in events]
    phase_b = [ev[1].elapsed_time(ev[2]) for ev in events] + [ev[3].elapsed_time(ev[4]) for ev in events]
    total_ms = max_over_ranks(total_ms, dev)

    # parity of the timed output (round trip) so a fast wrong kernel cannot pass unnoticed
    rt_err = float((torch.linalg.vector_norm(z - x) / torch.linalg.vector_norm(x)).item())
    vs_native = vs_fp64 = None
    if prec:  # the same forward transform through the FP32 CUDA-core stages on the same schedule
        with fftu.Plan(shape, p, dtype=t_dtype, schedule=fftu.FFTU_SCHED_GENERIC_A) as nat:
            fftu.fftu_exec(fwd.handle, x.data_ptr(), y.data_ptr(), sh)
            y_nat = torch.empty_like(x)
            fftu.fftu_exec(nat.handle, x.data_ptr(), y_nat.data_ptr(), sh)
            torch.cuda.synchronize(dev)
            vs_native = float((torch.linalg.vector_norm(y - y_nat) / torch.linalg.vector_norm(y_nat)).item())
            del y_nat
        # and against an FP64 transform of the same input (cuFFT in complex128, run as a library); the
        # element-by-element comparison with the FP64 oracle is in the test suite
        with torch.cuda.stream(stream):
            ref = torch.fft.fftn(x.to(torch.complex128))
            vs_fp64 = float((torch.linalg.vector_norm(y.to(torch.complex128) - ref) /
                             torch.linalg.vector_norm(ref)).item())
            del ref
        torch.cuda.synchronize(dev)
        torch.cuda.empty_cache()

    # context only: the same forward + inverse through torch.fft (cuFFT), run as a library
    cufft = None
    if not args.no_cufft and rank == 0:
        try:
            with torch.cuda.stream(stream):
                for _ in range(3):
                    torch.fft.ifftn(torch.fft.fftn(x))
                torch.cuda.synchronize(dev)
                c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                reps = max(3, min(20, args.steps))
                c0.record(stream)
                for _ in range(reps):
                    torch.fft.ifftn(torch.fft.fftn(x))
                c1.record(stream)
            torch.cuda.synchronize(dev)
            cms = c0.elapsed_time(c1) / reps
            cufft = {"impl": "torch.fft.fftn + ifftn (cuFFT)",
                     "ms_per_step": cms, "value": 2 * alg_bytes(shape, esize) / (cms * 1e-3) / 1e9, "unit": "GB/s",
                     "note": "context, not a target: cuFFT's own schedule (not the cyclic method), allocations "
                             "included, same array and metric"}
        except Exception as exc:
            cufft = {"error": repr(exc)}

    e2e = None
    if not args.no_e2e:
        # The step through the public API with host buffers: pinned H2D of the input, forward, inverse,
        # D2H of the result, every step.  Copies in, transforms and copies out run on three streams, two
        # device buffer sets deep, so that step i + 1's upload and step i - 1's download overlap step i's
        # transforms (the transforms stay on one stream: the plans' workspaces are never shared).
        out_host = torch.empty_like(x_host).pin_memory()
        xs_d = [torch.empty_like(x) for _ in range(2)]
        zs_d = [z, torch.empty_like(x)]
        K = max(1, args.e2e_copy_streams)  # each direction's copy in K pieces on K streams (copy engines)
        s_ins = [torch.cuda.Stream(dev) for _ in range(K)]
        s_outs = [torch.cuda.Stream(dev) for _ in range(K)]
        s_out = s_outs[0]
        flat_host_in, flat_host_out = x_host.view(-1), out_host.view(-1)
        bounds = [N * k // K for k in range(K + 1)]
        steps_e = 2 + args.e2e_steps
        ev_in = [[torch.cuda.Event() for _ in range(K)] for _ in range(steps_e)]
        ev_tf = [torch.cuda.Event() for _ in range(steps_e)]
        ev_out = [[torch.cuda.Event() for _ in range(K)] for _ in range(steps_e)]
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        for i in range(steps_e):
            b = i % 2
            if i == 2:
                torch.cuda.synchronize(dev)
                e0.record(s_ins[0])
                for k in range(1, K):
                    s_ins[k].wait_event(e0)
            xf, zf = xs_d[b].view(-1), zs_d[b].view(-1)
            for k in range(K):
                if i >= 2:
                    s_ins[k].wait_event(ev_tf[i - 2])  # buffer b's previous input has been transformed
                with torch.cuda.stream(s_ins[k]):
                    xf[bounds[k]:bounds[k + 1]].copy_(flat_host_in[bounds[k]:bounds[k + 1]], non_blocking=True)
                ev_in[i][k].record(s_ins[k])
                stream.wait_event(ev_in[i][k])
            if i >= 2:
                for k in range(K):
                    stream.wait_event(ev_out[i - 2][k])  # buffer b's previous result has been downloaded
            fftu.fftu_exec(fwd.handle, xs_d[b].data_ptr(), y.data_ptr(), sh)
            fftu.fftu_exec(inv.handle, y.data_ptr(), zs_d[b].data_ptr(), sh)
            ev_tf[i].record(stream)
            for k in range(K):
                s_outs[k].wait_event(ev_tf[i])
                with torch.cuda.stream(s_outs[k]):
                    flat_host_out[bounds[k]:bounds[k + 1]].copy_(zf[bounds[k]:bounds[k + 1]], non_blocking=True)
                ev_out[i][k].record(s_outs[k])
        for k in range(1, K):
            s_out.wait_event(ev_out[steps_e - 1][k])
        e1.record(s_out)
        torch.cuda.synchronize(dev)
        e2e_ms = max_over_ranks(e0.elapsed_time(e1) / args.e2e_steps, dev)
        e2e = {"value": whole_job_value(2 * alg_bytes(shape, esize), e2e_ms, world), "unit": "GB/s",
               "h2d_bytes_per_step": N * esize, "d2h_bytes_per_step": N * esize, "ms_per_step": e2e_ms,
               "includes": "pinned H2D of the input, forward, inverse, D2H of the result, every step; copies "
                           "and transforms of neighbouring steps overlap (two buffer sets; each copy direction "
                           f"in {K} pieces on {K} streams)"}

    if rank == 0:
        ms_per_step = total_ms / args.steps
        value = whole_job_value(2 * alg_bytes(shape, esize), ms_per_step, world)
        peak, peak_kind = measured_peak()
        ta, tb = statistics.mean(phase_a), statistics.mean(phase_b)
        half = 2 * N * esize  # one HBM round trip: the algorithmic bytes of one phase
        la, lb = fwd.info["launches_phase_a"], fwd.info["launches_phase_b"]
        if ta >= tb:
            dom, t_dom, launches = "phase_a", ta, la
        else:
            dom, t_dom, launches = "phase_b", tb, lb
        kernel_name = f"{dom}_{'x'.join(map(str, shape))}_p{'x'.join(map(str, p))}"
        achieved = half / (t_dom * 1e-3) / 1e9
        roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                    "traffic": traffic_for(kernel_name), "kernel": dom, "launches_in_phase": launches,
                    "peak_source": f"{peak_kind} hbm_gbs",
                    "frac_of_nominal": achieved / NOMINAL_HBM_GBS, "nominal_gbs": NOMINAL_HBM_GBS,
                    "step_frac": value / peak, "step_frac_of_nominal": value / NOMINAL_HBM_GBS,
                    "phase_ms": {"phase_a": ta, "phase_b": tb},
                    "phase_frac": {"phase_a": half / (ta * 1e-3) / 1e9 / peak,
                                   "phase_b": half / (tb * 1e-3) / 1e9 / peak}}
        if esize == 16:
            # complex128: FP64 arithmetic, not HBM, bounds the path on GB300 (about 1.3 TFLOP/s FP64 against
            # 6.7 TB/s; about 5 log2 N flops per element per transform need 16 B of traffic per flop-pass)
            gf = 2 * 5 * N * math.log2(N) / (ms_per_step * 1e-3) / 1e9
            try:
                fp64_peak, fp64_src = fftu.fftu_measure_fp64_rate(3), "measured FP64 FMA rate on this GPU"
            except Exception:
                fp64_peak, fp64_src = FP64_PEAK_GFLOPS, "GB300 FP64 nominal (1.25 TFLOP/s)"
            roofline = {"bound": "alu", "achieved": gf, "peak": fp64_peak, "unit": "GFLOP/s",
                        "frac": gf / fp64_peak, "traffic": None, "kernel": "whole step",
                        "peak_source": fp64_src + "; flops counted as 5 N log2 N per transform",
                        "hbm": roofline}
        serving = None
        if not args.no_serve and world == 1 and tuple(shape) == (512, 512, 512):
            try:
                serving = run_serving(fftu, args, local)
            except Exception as exc:  # reported, never silently dropped
                serving = {"error": repr(exc)}
        cpu = None
        if not args.no_cpu_baseline and world == 1:
            sample = shape_of(args.cpu_sample)
            t_cpu, cores = oracle_cpu_run(sample, args.seed, reps=args.cpu_reps)
            cpu = {"value": 2 * alg_bytes(sample, esize) / t_cpu / 1e9, "unit": "GB/s", "cores": cores,
                   "kind": "oracle", "seconds_per_rep": t_cpu,
                   "sample": f"plain FP64 oracle (not an optimized FFT), forward+inverse of one "
                             f"{'x'.join(map(str, sample))} array, {args.cpu_reps} repetitions (same seeded "
                             f"inputs), all {cores} host cores, GB/s scaled by 4*N*8 bytes per transform"}
            import oracle
            oracle.set_threads(1)
            try:
                one = (128, 128, 128)
                t1, _ = oracle_cpu_run(one, args.seed, reps=3)
            finally:
                oracle.set_threads(0)
            cpu["single_thread"] = {"value": 2 * alg_bytes(one, esize) / t1 / 1e9, "unit": "GB/s", "cores": 1,
                                    "seconds_per_rep": t1,
                                    "sample": "same oracle, 1 thread, forward+inverse of one 128^3 array, 3 reps"}
            small = (64, 64, 64)
            oracle.set_threads(1)
            try:
                ts1, _ = oracle_cpu_run(small, args.seed, reps=3)
            finally:
                oracle.set_threads(0)
            tsa, _ = oracle_cpu_run(small, args.seed, reps=3)
            cpu["sizes"] = [{"shape": "x".join(map(str, sh)), "cores": c, "reps": r, "seconds_per_rep": t,
                             "value": 2 * alg_bytes(sh, esize) / t / 1e9, "unit": "GB/s"}
                            for sh, c, r, t in ((small, 1, 3, ts1), (small, cores, 3, tsa), (one, 1, 3, t1),
                                                (sample, cores, args.cpu_reps, t_cpu))]
            cpu["skipped"] = ("1024^3: one forward+inverse pair of the oracle takes about 8x the 512^3 time and "
                              "16 GiB per FP64 array; left out to keep the CPU sample bounded")
            if esize == 8:
                try:
                    cpu["torch_cpu_context"] = torch_cpu_fft_run(sample, args.seed)
                except Exception as exc:  # context only; reported, never silently dropped
                    cpu["torch_cpu_context"] = {"error": repr(exc)}
        line = {
            "metric": METRIC, "metric_detail": METRIC_DETAIL,
            "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": ("f32" if esize == 8 else "f64") if not prec else
                     f"{args.precision} hi+lo tensor-core radix-16 stages, f32 elsewhere",
            "data": "synthetic",
            "config": workload_config(shape, p, esize, args, world),
            "plan": {"schedule": fwd.info["schedule"], "precision": args.precision, "p_inverse": inv.info["p"],
                     "tuned": tune, "plan_seconds": t_plan, "strided_tile": fwd.info["tile"],
                     "strided_radix": fwd.info["radix"]},
            "gflops_5NlogN": world * 2 * 5 * N * math.log2(N) / (ms_per_step * 1e-3) / 1e9,
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": args.steps * 2 * (la + lb),
            "clocks": clocks,
            "round_trip_rel_l2": rt_err,
            "forward_vs_fp32_stages_rel_l2": vs_native,
            "forward_vs_fp64_rel_l2": vs_fp64,
            "cufft_context": cufft,
            "serving": serving,
        }
    err = None
    if not rt_err < (1e-3 if prec != 1 else 5e-3):
        err = f"round trip relative L2 error {rt_err:.3g}: the timed transforms are wrong"
    fwd.close()
    inv.close()
    del x, y, z
    torch.cuda.empty_cache()
    if world > 1:
        dist.destroy_process_group()
    return (line if rank == 0 else None), err


SERVE_SHAPES = [(32, 32, 32), (64, 64, 64), (128, 128, 128), (256, 256, 256), (1024, 1024), (2048, 2048),
                (4096, 4096)]


def run_serving(fftu, args, local):
    """Poisson stream of mixed requests through the native serving loop (fftu_server_*).

    Shapes uniform over SERVE_SHAPES, complex128 with probability 0.1, forward/inverse
    equiprobable.  Host buffers are page-locked pools per (shape, dtype), inputs seeded.
    The offered rate is --serve-rate, or (default) 0.7 x the saturation throughput measured
    first by a closed-loop burst of the same mix.  Latency = completion seen by the server
    minus submission, on the server's clock."""
    import threading

    import numpy as np
    import torch
    from fftu_inputs import complex_uniform

    rng = np.random.default_rng(args.seed + 77)

    def draw(count):
        return [(SERVE_SHAPES[rng.integers(len(SERVE_SHAPES))], bool(rng.random() < 0.1), bool(rng.integers(2)))
                for _ in range(count)]

    pools, free = {}, {}
    t_alloc = time.perf_counter()
    for shape in SERVE_SHAPES:
        for c128 in (False, True):
            dt = np.complex128 if c128 else np.complex64
            x0 = torch.from_numpy(complex_uniform(args.seed + len(pools), shape, dtype=dt))
            size = 8 if math.prod(shape) >= (1 << 22) else 24 if math.prod(shape) >= (1 << 20) else 48
            slots = []
            for _ in range(size):
                xi = torch.empty_like(x0).pin_memory()
                xi.copy_(x0)
                slots.append((xi, torch.empty_like(x0).pin_memory()))
            pools[(shape, c128)] = slots
            free[(shape, c128)] = list(range(size))
    t_alloc = time.perf_counter() - t_alloc
    cv = threading.Condition(threading.Lock())
    server = fftu.fftu_server_create(max_batch=64, streams=args.serve_streams, max_inflight=args.serve_inflight,
                                     copy_piece_mib=args.serve_piece_mib, max_inflight_solo=args.serve_solo)
    # every key's instances and graphs, for every batch size, before any request is timed
    t_warm = time.perf_counter()
    for (shape, c128), slots in pools.items():
        for inverse in (False, True):
            xi, yi = slots[0]
            fftu.fftu_server_warm(server, shape, fftu.FFTU_C128 if c128 else fftu.FFTU_C64,
                                  fftu.FFTU_INVERSE if inverse else fftu.FFTU_FORWARD, xi.data_ptr(), yi.data_ptr(),
                                  16)
    t_warm = time.perf_counter() - t_warm

    def phase(kinds, gaps, tag0):
        """Submit kinds[i] at the cumulative gaps (None: as soon as a buffer is free); wait for all."""
        slot_of, meta, stalls, done = {}, {}, [0], []

        def generator():
            t_next = time.perf_counter()
            for i, (shape, c128, inverse) in enumerate(kinds):
                if gaps is not None:
                    t_next += gaps[i]
                    while True:
                        dt_ = t_next - time.perf_counter()
                        if dt_ <= 0:
                            break
                        time.sleep(dt_ if dt_ > 2e-4 else 0)
                key = (shape, c128)
                with cv:
                    if not free[key]:
                        stalls[0] += 1
                    while not free[key]:
                        cv.wait(0.01)
                    j = free[key].pop()
                    slot_of[tag0 + i] = (key, j)
                    meta[tag0 + i] = (shape, c128, inverse)
                xi, yi = pools[key][j]
                fftu.fftu_server_submit(server, shape, fftu.FFTU_C128 if c128 else fftu.FFTU_C64,
                                        fftu.FFTU_INVERSE if inverse else fftu.FFTU_FORWARD, xi.data_ptr(),
                                        yi.data_ptr(), tag0 + i)

        gen = threading.Thread(target=generator)
        gen.start()
        while len(done) < len(kinds):
            got = fftu.fftu_server_poll(server, 4096)
            if got:
                with cv:
                    for c in got:
                        key, j = slot_of.pop(c["tag"])
                        free[key].append(j)
                    cv.notify_all()
                done.extend(got)
            else:
                time.sleep(2e-4)
        gen.join()
        return done, meta, stalls[0]

    # saturation: a closed-loop burst of the same mix (as many in flight as the buffer pools allow)
    sat_done, _, _ = phase(draw(args.serve_warmup + 2000), None, 0)
    sat = sorted(sat_done, key=lambda c: c["done_s"])[args.serve_warmup:]
    sat_rate = (len(sat) - 1) / (sat[-1]["done_s"] - sat[0]["done_s"])
    rate = args.serve_rate if args.serve_rate > 0 else 0.7 * sat_rate
    total = args.serve_warmup + args.serve_requests
    kinds = draw(total)
    gaps = rng.exponential(1.0 / rate, size=total)
    stats0 = fftu.fftu_server_stats_get(server)
    wall0 = time.perf_counter()
    done, meta, stalls = phase(kinds, gaps, 10 ** 6)
    wall = time.perf_counter() - wall0
    stats1 = fftu.fftu_server_stats_get(server)
    timed = [c for c in done if c["tag"] >= 10 ** 6 + args.serve_warmup]
    bad = [c for c in done + sat_done if c["status"] != 0]
    lat = np.array([c["done_s"] - c["submit_s"] for c in timed]) * 1e3
    wait = np.array([c["start_s"] - c["submit_s"] for c in timed]) * 1e3   # queued in the server
    serve = np.array([c["done_s"] - c["start_s"] for c in timed]) * 1e3    # issued -> completion seen
    t_first = min(c["submit_s"] for c in timed)
    t_last = max(c["done_s"] for c in timed)
    span = t_last - t_first
    alg = sum(4 * math.prod(meta[c["tag"]][0]) * (16 if meta[c["tag"]][1] else 8) for c in timed)
    moved = sum(2 * math.prod(meta[c["tag"]][0]) * (16 if meta[c["tag"]][1] else 8) for c in timed)
    d = {k: stats1[k] - stats0[k] for k in ("batches", "graph_replays", "direct_launches", "kernel_launches",
                                              "rejected", "evictions", "instance_creations", "creation_s")}
    d["max_launch_ms"] = stats1["max_launch_s"] * 1e3
    d["max_loop_gap_ms"] = stats1["max_loop_gap_s"] * 1e3
    per_class = {}
    for shape in SERVE_SHAPES:
        for c128 in (False, True):
            ls = np.array([(c["done_s"] - c["submit_s"]) * 1e3 for c in timed
                           if meta[c["tag"]][0] == shape and meta[c["tag"]][1] == c128])
            if ls.size:
                per_class[f"{'x'.join(map(str, shape))}{' c128' if c128 else ''}"] = {
                    "n": int(ls.size), "p50_ms": round(float(np.percentile(ls, 50)), 3),
                    "p99_ms": round(float(np.percentile(ls, 99)), 3)}

    # parity of the served path: one request per class, compared with the same plan run directly
    worst = 0.0
    for (shape, c128), slots in pools.items():
        xi, yi = slots[0]
        for inverse in (False, True):
            fftu.fftu_server_submit(server, shape, fftu.FFTU_C128 if c128 else fftu.FFTU_C64,
                                    fftu.FFTU_INVERSE if inverse else fftu.FFTU_FORWARD, xi.data_ptr(),
                                    yi.data_ptr(), 10 ** 9)
            fftu.fftu_server_drain(server, 60.0)
            fftu.fftu_server_poll(server, 16)
            xd = xi.to(f"cuda:{local}")
            with fftu.Plan(shape, None, dtype=xd.dtype, inverse=inverse) as pl:
                ref = pl.exec(xd).cpu()
            worst = max(worst, float((torch.linalg.vector_norm(yi - ref) /
                                      torch.linalg.vector_norm(ref)).item()))
    fftu.fftu_server_destroy(server)
    return {
        "requests": len(timed), "warmup_requests": args.serve_warmup,
        "saturation_rate_per_s": sat_rate, "offered_rate_per_s": rate,
        "offered_fraction_of_saturation": rate / sat_rate,
        "achieved_rate_per_s": len(timed) / span, "p50_ms": float(np.percentile(lat, 50)),
        "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()), "max_ms": float(lat.max()),
        "queue_wait_ms": {"p50": float(np.percentile(wait, 50)), "p99": float(np.percentile(wait, 99))},
        "issue_to_done_ms": {"p50": float(np.percentile(serve, 50)), "p99": float(np.percentile(serve, 99))},
        "gbs_algorithmic": alg / span / 1e9, "gbs_host_copies": moved / span / 1e9,
        "failed": len(bad), "pool_stalls": stalls, "wall_s": wall, "pinned_pool_alloc_s": t_alloc,
        "warm_s": t_warm,
        "served_vs_direct_max_rel_l2": worst, **d, "per_class": per_class,
        "server": {"streams": args.serve_streams, "max_inflight": args.serve_inflight or 2 * args.serve_streams,
                   "max_inflight_solo": args.serve_solo or args.serve_streams - args.serve_streams // 2,
                   "max_batch": 64, "copy_piece_mib": args.serve_piece_mib},
        "mix": "shapes uniform over 32^3, 64^3, 128^3, 256^3, 1024^2, 2048^2, 4096^2; complex128 w.p. 0.1; "
               "forward/inverse equiprobable; Poisson arrivals at the offered rate (0.7 x the closed-loop "
               "saturation rate unless --serve-rate is given); latency = server completion - submission",
    }


def run_serve_only(args):
    import torch
    rank, world, local = dist_env()
    if rank != 0:
        return
    torch.cuda.set_device(local)
    from paper_2203_11795_gb300 import _build
    _build.build()
    import paper_2203_11795_gb300 as fftu
    r = run_serving(fftu, args, local)
    line = {"metric": "mixed-request p50/p99 latency (ms) and GB/s through the serving loop",
            "value": r["p99_ms"], "unit": "ms (p99)", "n_gpus": 1, "higher_is_better": False,
            "steps": r["requests"], "warmup": r["warmup_requests"], "scaling": "weak", "vs_baseline": None,
            "dtype": "f32/f64", "data": "synthetic", "config": {"workload": "serving mix", **r},
            "gpu_launches": r["kernel_launches"]}
    print(json.dumps(line), flush=True)
    if r["failed"] or not r["served_vs_direct_max_rel_l2"] < 1e-6:
        sys.exit(1)


def run_pointwise(args):
    """Forward transform, elementwise product in the frequency domain, inverse transform
    (fftu_exec_pointwise), with no reordering between them; one step = one such convolution."""
    import numpy as np
    import torch
    import torch.distributed as dist

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2203_11795_gb300 import _build
    _build.build()
    import paper_2203_11795_gb300 as fftu
    from fftu_inputs import complex_uniform

    shape = shape_of(args.shape)
    p = shape_of(args.p)
    N = math.prod(shape)
    x = torch.from_numpy(complex_uniform(args.seed + rank, shape, dtype=np.complex64)).to(dev)
    mul = torch.from_numpy(complex_uniform(args.seed + 5000 + rank, shape, dtype=np.complex64)).to(dev)
    tmp, out = torch.empty_like(x), torch.empty_like(x)
    fwd = fftu.Plan(shape, p)
    inv = fftu.Plan(shape, p, inverse=True)
    stream = torch.cuda.Stream(dev)
    sh = stream.cuda_stream

    def step():
        fftu.fftu_exec_pointwise(fwd.handle, inv.handle, x.data_ptr(), mul.data_ptr(), tmp.data_ptr(),
                                 out.data_ptr(), sh)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
    torch.cuda.synchronize(dev)
    sampler = ClockSampler(local) if rank == 0 else None
    if world > 1:
        dist.barrier()
    if sampler:
        sampler.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    with torch.cuda.stream(stream):
        for _ in range(args.steps):
            step()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    clocks = sampler.stop() if sampler else None
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, dev)
    # the same convolution through two plain transforms and a separate product (torch only for the product)
    ref = torch.empty_like(x)
    with torch.cuda.stream(stream):
        fftu.fftu_exec(fwd.handle, x.data_ptr(), tmp.data_ptr(), sh)
        prod = tmp * mul
        fftu.fftu_exec(inv.handle, prod.data_ptr(), ref.data_ptr(), sh)
    torch.cuda.synchronize(dev)
    err = float((torch.linalg.vector_norm(out - ref) / torch.linalg.vector_norm(ref)).item())
    fwd.check_device_status()
    inv.check_device_status()
    if rank == 0:
        step_bytes = 2 * alg_bytes(shape, 8) + N * 8  # two transforms and one read of the multiplier
        value = whole_job_value(step_bytes, ms, world)
        peak, peak_kind = measured_peak()
        line = {
            "metric": "forward -> pointwise product -> inverse, algorithmic GB/s", "value": value, "unit": "GB/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{'x'.join(map(str, shape))} complex64 convolution step "
                                   f"(fftu_exec_pointwise), cyclic p={'x'.join(map(str, p))}",
                       "bytes_per_step": step_bytes, "separate_product_vs_fused_rel_l2": err,
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
            "roofline": {"bound": "hbm", "achieved": value / world, "peak": peak, "unit": "GB/s",
                         "frac": value / world / peak, "traffic": None, "kernel": "whole step",
                         "peak_source": f"{peak_kind} hbm_gbs"},
            "gpu_launches": args.steps * 2 * (fwd.info["launches_phase_a"] + fwd.info["launches_phase_b"]),
            "clocks": clocks,
        }
    fail = None if err < 1e-5 else f"fused and separate convolutions differ ({err:.3g})"
    fwd.close()
    inv.close()
    del x, mul, tmp, out, ref
    torch.cuda.empty_cache()
    if world > 1:
        dist.destroy_process_group()
    return (line if rank == 0 else None), fail


def uneven_shapes(count, seed, cubes=False):
    """Each n_l drawn independently from {32, 64, 128}: sizes 32^3 to 128^3, cubes included.
    cubes=True: the other reading, cubes n^3 with n drawn from {32, 64, 128}."""
    import numpy as np
    rng = np.random.default_rng(seed)
    if cubes:
        return [(n, n, n) for n in (int(v) for v in rng.choice([32, 64, 128], size=count))]
    return [tuple(int(v) for v in rng.choice([32, 64, 128], size=3)) for _ in range(count)]


def run_batch(args):
    """K uneven complex64 3D transforms, forward then inverse, each direction one persistent launch."""
    import numpy as np
    import torch
    import torch.distributed as dist

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2203_11795_gb300 import _build
    _build.build()
    import paper_2203_11795_gb300 as fftu
    from fftu_inputs import complex_uniform

    shapes = uneven_shapes(args.batch, args.seed, cubes=args.batch_cubes)
    hosts = [torch.from_numpy(complex_uniform(args.seed + 1000 * rank + i, s, dtype=np.complex64)).pin_memory()
             for i, s in enumerate(shapes)]
    xs = [h.to(dev) for h in hosts]
    ys = [torch.empty_like(x) for x in xs]
    zs = [torch.empty_like(x) for x in xs]
    fwd = [fftu.Plan(s, None, dtype=torch.complex64) for s in shapes]
    inv = [fftu.Plan(s, None, dtype=torch.complex64, inverse=True) for s in shapes]
    bf = fftu.fftu_batch_create([q.handle for q in fwd])
    bi = fftu.fftu_batch_create([q.handle for q in inv])
    px, py, pz = ([t.data_ptr() for t in ts] for ts in (xs, ys, zs))
    stream = torch.cuda.Stream(dev)
    sh = stream.cuda_stream
    elems = sum(math.prod(s) for s in shapes)
    step_bytes = 2 * 4 * elems * 8

    def step():
        fftu.fftu_batch_exec(bf, px, py, sh)
        fftu.fftu_batch_exec(bi, py, pz, sh)

    def per_plan_step():
        for q, a, b in zip(fwd, px, py):
            fftu.fftu_exec(q.handle, a, b, sh)
        for q, a, b in zip(inv, py, pz):
            fftu.fftu_exec(q.handle, a, b, sh)

    def timed(fn, k):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                fn()
            torch.cuda.synchronize(dev)
            e0.record(stream)
            for _ in range(k):
                fn()
            e1.record(stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / k

    sampler = ClockSampler(local) if rank == 0 else None
    if world > 1:
        dist.barrier()
    if sampler:
        sampler.start()
    ms = timed(step, args.steps)
    clocks = sampler.stop() if sampler else None
    ms = max_over_ranks(ms, dev)
    fftu.fftu_batch_check_status(bf)
    fftu.fftu_batch_check_status(bi)
    rt = max(float((torch.linalg.vector_norm(z - x) / torch.linalg.vector_norm(x)).item()) for x, z in zip(xs, zs))
    ms_loop = timed(per_plan_step, max(1, args.steps // 4))
    launches_loop = sum(q.info["launches_phase_a"] + q.info["launches_phase_b"] for q in fwd + inv)

    e2e = None
    if not args.no_e2e:
        outs = [torch.empty_like(h).pin_memory() for h in hosts]
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            for i in range(2 + args.e2e_steps):
                if i == 2:
                    torch.cuda.synchronize(dev)
                    e0.record(stream)
                for h, x in zip(hosts, xs):
                    x.copy_(h, non_blocking=True)
                step()
                for o, z in zip(outs, zs):
                    o.copy_(z, non_blocking=True)
            e1.record(stream)
        torch.cuda.synchronize(dev)
        e2e_ms = max_over_ranks(e0.elapsed_time(e1) / args.e2e_steps, dev)
        e2e = {"value": whole_job_value(step_bytes, e2e_ms, world), "unit": "GB/s",
               "h2d_bytes_per_step": elems * 8, "d2h_bytes_per_step": elems * 8, "ms_per_step": e2e_ms,
               "includes": "pinned H2D of every input, batched forward and inverse, D2H of every result"}

    if rank == 0:
        peak, peak_kind = measured_peak()
        achieved = step_bytes / 2 / (ms / 2 * 1e-3) / 1e9
        cpu = None
        if not args.no_cpu_baseline and world == 1:
            t0 = time.perf_counter()
            import oracle
            sample = shapes[:8]
            for i, s in enumerate(sample):
                x = complex_uniform(args.seed + i, s, dtype=np.complex64).astype(np.complex128)
                oracle.fftn(oracle.fftn(x), inverse=True)
            t_cpu = time.perf_counter() - t0
            b_cpu = sum(2 * 4 * math.prod(s) * 8 for s in sample)
            cpu = {"value": b_cpu / t_cpu / 1e9, "unit": "GB/s", "cores": oracle.max_threads(), "kind": "oracle",
                   "sample": "FP64 oracle forward+inverse of the first 8 arrays of the batch, GB/s scaled by "
                             "4*N*8 bytes per transform"}
        line = {
            "metric": "batched uneven 3D FFT algorithmic GB/s", "metric_detail": METRIC_DETAIL,
            "value": whole_job_value(step_bytes, ms, world), "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"batch of {args.batch} uneven complex64 3D transforms "
                                   + ("(cubes n^3, n in 32, 64, 128), " if args.batch_cubes else
                                      "(n_l in 32, 64, 128), ")
                                   + "forward+inverse, one persistent launch per direction",
                       "elements": elems, "bytes_per_array_set": elems * 8,
                       "l2": "arrays total more than L2 but part of a step's working set stays L2-resident",
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None, "kernel": "batch_kernel",
                         "peak_source": f"{peak_kind} hbm_gbs"},
            "per_plan_loop": {"ms_per_step": ms_loop, "gpu_launches_per_step": launches_loop,
                              "value": whole_job_value(step_bytes, ms_loop, world)},
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": 2 * args.steps, "clocks": clocks,
            "round_trip_rel_l2": rt,
        }
    fail = None if rt < 1e-3 else f"round trip relative L2 error {rt:.3g}: the timed transforms are wrong"
    fftu.fftu_batch_destroy(bf)
    fftu.fftu_batch_destroy(bi)
    for q in fwd + inv:
        q.close()
    del xs, ys, zs
    torch.cuda.empty_cache()
    if world > 1:
        dist.destroy_process_group()
    return (line if rank == 0 else None), fail


# Secondary configurations measured after the headline run, each one a short run of its own with its
# own clock record: the other benchmark configurations, the split-precision forms and the batched and
# fused-convolution forms, so that the default line carries every configuration's figure.
SECONDARY = [
    ("1024^3_c64_p16x16x8", "run", dict(shape="1024,1024,1024", p="16,16,8", steps=5, warmup=3, inputs="device")),
    ("1024^3_c64_p8x8x8", "run", dict(shape="1024,1024,1024", p="8,8,8", steps=5, warmup=3, inputs="device")),
    ("1024^3_c64_p4x4x4", "run", dict(shape="1024,1024,1024", p="4,4,4", steps=5, warmup=3, inputs="device")),
    ("512^3_c64_split_bf16", "run", dict(precision="bf16", steps=10, warmup=3, inputs="device")),
    ("512^3_c64_split_fp16", "run", dict(precision="fp16", steps=10, warmup=3, inputs="device")),
    ("512^3_c64_split_bf16_loguniform", "run", dict(precision="bf16", steps=10, warmup=3,
                                                    inputs="device_loguniform")),
    ("512^3_c64_split_fp16_loguniform", "run", dict(precision="fp16", steps=10, warmup=3,
                                                    inputs="device_loguniform")),
    ("16384^2_c64_p16_tuned", "run", dict(shape="16384,16384", p="16,16", schedule=3, tile=4096, steps=10,
                                          warmup=3, inputs="device")),
    ("32^5_c64_p4", "run", dict(shape="32,32,32,32,32", p="4,4,4,4,4", tile=2048, steps=20, warmup=3,
                                inputs="device")),
    ("64^4_c128_p8", "run", dict(shape="64,64,64,64", p="8,8,8,8", dtype="c128", steps=10, warmup=3,
                                 inputs="device")),
    ("batch_64_uneven_c64", "batch", dict(batch=64, steps=20, warmup=3)),
    ("512^3_c64_pointwise", "pointwise", dict(steps=10, warmup=3)),
]
SECONDARY_KEYS = ("value", "unit", "ms_per_step", "steps", "warmup", "dtype", "config", "plan", "roofline",
                  "gflops_5NlogN", "clocks", "gpu_launches", "round_trip_rel_l2", "forward_vs_fp32_stages_rel_l2",
                  "forward_vs_fp64_rel_l2", "per_plan_loop", "metric")


def run_secondary(args):
    """Every SECONDARY configuration on this GPU; a failure is reported in its entry, never dropped."""
    import torch
    torch.cuda.empty_cache()
    out = {}
    for name, kind, over in SECONDARY:
        sub = argparse.Namespace(**vars(args))
        sub.no_serve = sub.no_cpu_baseline = sub.no_e2e = sub.no_cufft = True
        sub.no_secondary = True
        for k, v in over.items():
            setattr(sub, k, v)
        t0 = time.perf_counter()
        try:
            fn = {"run": run_ours, "batch": run_batch, "pointwise": run_pointwise}[kind]
            line, err = fn(sub)
            ent = {k: line[k] for k in SECONDARY_KEYS if k in line}
            if err:
                ent["error"] = err
        except Exception as exc:  # reported, never silently dropped
            ent = {"error": repr(exc)}
        ent["wall_s"] = time.perf_counter() - t0
        out[name] = ent
    return out


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.serve:
        run_serve_only(args)
        return
    fn = run_batch if args.batch > 0 else run_pointwise if args.pointwise else run_ours
    line, err = fn(args)
    rank, world, _ = dist_env()
    if (fn is run_ours and line is not None and world == 1 and not args.no_secondary
            and args.shape == "512,512,512" and args.precision == "native" and args.dtype == "c64"):
        line["secondary"] = run_secondary(args)
    if line is not None:
        print(json.dumps(line), flush=True)
    if err:
        print(err, file=sys.stderr)
        sys.exit(1)


if __name__ == "__main__":
    main()

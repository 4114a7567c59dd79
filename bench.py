#!/usr/bin/env python3
"""Throughput benchmark of the GB300 beamformer on the real-time FP16 workload.

Workload: 32 antennas (BEST-2 4 x 8 grid), 1024 channels over 16 MHz, 1024
beams over +-10 deg, 15625 FP16 complex samples per channel (one 1 s chunk),
noise plus 3 plane waves, integration over 64 samples.

One step = one pass of the per-chunk path on one chunk already resident in
HBM: the weight refresh (delay + weight kernels, the tracking-beam update of
Section 3.1; double-buffered, on the plan's weight stream, so the refresh for
the next chunk overlaps the current beamforming) and the fused tensor-core
beamform + |B|^2 + integrate kernel (no corner turn: the input is already
channel-major).  FLOPs are
counted as 8 N per beam, channel and sample (Section 2.2).

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle instead, on a bounded channel sample of the same workload.
"""
import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "beamform TFLOP/s & roofline %, p99 chunk latency: mixed-prec vs FP32, 1 GB300"
INPUTS = {"c16f": synth.C16F, "ci8": synth.CI8, "ci4": synth.CI4}
INPUT_SIGMA = {synth.CI8: 16.0, synth.CI4: 2.0}   # noise per component of the integer-input variants
UNIT = "TFLOP/s"
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}
PROFILE = os.path.join(ROOT, "profiles", "k_tc_config2.json")


def flops(n_ant, n_beam, n_chan, n_samp):
    return 8.0 * n_ant * n_beam * n_chan * n_samp


def power_errors(P, P_ref):
    """(max relative error with a floor of 1e-3 x mean, L2 relative error)."""
    P = np.asarray(P, dtype=np.float64)
    P_ref = np.asarray(P_ref, dtype=np.float64)
    floor = 1e-3 * max(P_ref.mean(), 1e-300)
    return (float(np.max(np.abs(P - P_ref) / np.maximum(P_ref, floor))),
            float(np.linalg.norm(P - P_ref) / max(np.linalg.norm(P_ref), 1e-300)))


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return FALLBACK_PEAKS, "fallback"


KERNEL_SOURCES = ("k_tc_kernel.cuh", "tc_common.cuh", "ptx.cuh")


def kernel_source_sha():
    """Hash of the fused kernel's code (its source files with comments and
    blank space removed), so that a profile is invalidated by a code change
    and not by an edit of a comment."""
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:   # the kernel's own sources
        text = open(os.path.join(ROOT, "paper_1412_4907_gb300", "csrc", f)).read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
        h.update(" ".join(text.split()).encode())
    return h.hexdigest()[:16]


def profiled_traffic():
    """DRAM bytes per launch of the tensor-core kernel from the committed ncu
    summary, if it was taken on the current kernel source."""
    if not os.path.exists(PROFILE):
        return None
    d = json.load(open(PROFILE))
    if d.get("source_sha") != kernel_source_sha():
        return None
    return d.get("dram_bytes_per_launch")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 50 ms; only the
    samples taken inside [start, stop] of the timed region are kept."""
    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.proc = None
        self.path = None
        self.t0 = self.t1 = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-i", str(self.gpu), "-lms", "50", "-f", self.path],
                stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def mark_start(self):
        self.t0 = time.time()

    def mark_stop(self):
        self.t1 = time.time()

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        import datetime
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                rows.append((ts, float(parts[2]), float(parts[3]), float(parts[4]), parts[6:10]))
            except ValueError:
                continue
        os.unlink(self.path)
        inside = [r for r in rows if self.t0 is not None and self.t0 <= r[0] <= (self.t1 or r[0])]
        use = inside or rows
        if not use:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in use for i, v in enumerate(r[4]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[1] for r in use), "sm_max_mhz": max(r[2] for r in use),
                "power_w_max": max(r[3] for r in use), "samples": len(use),
                "samples_in_timed_region": len(inside), "reasons": reasons}


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def shard_range(n: int, world: int, rank: int):
    """Contiguous share [lo, hi) of n independent units (channels) for one rank:
    the first n % world ranks take one extra."""
    base, extra = divmod(n, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def max_over_ranks(value: float, dist=None, device="cpu") -> float:
    """The slowest rank's time (every rank gets it); identity without a process group."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def cpu_oracle_rate(scene, dirs, t_int, n_chan, threads=0, x_cache=None):
    """FP64 oracle (plain C, one thread per channel range) on the first
    ``n_chan`` channels and the given beams: returns (TFLOP/s, seconds)."""
    import oracle
    chans = list(range(n_chan))
    if x_cache is not None and x_cache.get("n") == n_chan:
        X64 = x_cache["X"]
    else:
        x = synth.voltages(scene, synth.C16F, channels=chans)
        X64 = oracle.decode_voltages(synth.C16F, x)
        if x_cache is not None:
            x_cache.update(n=n_chan, X=X64)
    t0 = time.perf_counter()
    W = oracle.weights(scene.pos, scene.freqs[chans], dirs)
    oracle.power(W, X64, t_int, threads=threads)
    dt = time.perf_counter() - t0
    return flops(scene.n_ant, dirs.shape[0], n_chan, scene.n_samp) / dt / 1e12, dt


def run_reference(args):
    """The FP64 oracle on the host cores, each step a bounded sample of the
    workload (all samples of a channel subset for a beam subset), sized so the
    whole run takes about two minutes."""
    world, rank, _ = dist_env()
    if rank != 0:
        return
    scene, dirs, t_int = synth.config2()
    cores = os.cpu_count() or 1
    n_chan = min(scene.n_chan, cores)
    cache = {}
    _, dt_full = cpu_oracle_rate(scene, dirs[:64], t_int, n_chan, x_cache=cache)   # calibration
    per_beam = dt_full / 64
    budget = 120.0 / (args.steps + args.warmup)
    n_beam = int(max(8, min(dirs.shape[0], budget / max(per_beam, 1e-9))))
    sub = dirs[:n_beam]
    rates = []
    for i in range(args.warmup + args.steps):
        r, dt = cpu_oracle_rate(scene, sub, t_int, n_chan, x_cache=cache)
        if i >= args.warmup:
            rates.append((r, dt))
    value = statistics.mean(r for r, _ in rates)
    ms = 1e3 * statistics.mean(dt for _, dt in rates)
    sample = (f"{n_chan} of 1024 channels x {n_beam} of 1024 beams x all 15625 samples per step, "
              f"FP64 oracle, {cores} threads")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "impl": "reference", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict(scene, dirs, t_int, args.scaling),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def config_dict(scene, dirs, t_int, scaling="weak", mode=synth.C16F):
    name = {synth.C16F: "FP16", synth.CI8: "8-bit integer", synth.CI4: "4-bit integer"}[mode]
    vb = scene.n_chan * scene.n_samp * scene.n_ant * synth.MODE_BYTES[mode] / 1e9
    return {"workload": f"real-time {name} chunk: 32-antenna BEST-2 grid, {scene.n_chan} channels x 15625 "
                        "samples, 1024 beams, T_int 64",
            "n_ant": scene.n_ant, "n_chan": scene.n_chan, "n_beam": int(dirs.shape[0]),
            "n_samp": scene.n_samp, "t_int": t_int,
            "input": f"{synth.MODE_NAMES[mode]}, [c][t][n] (no corner turn)"
                     + ("" if mode == synth.C16F else "; widened to FP16 inside the beamformer"),
            "l2": f"no flush: voltages ({vb:.2f} GB) and weights (0.27 GB) exceed the 129 MB L2",
            "parallelism": ("channels: one independent chunk per GPU, no collective" if scaling == "weak" else
                            "channels: contiguous channel ranges of one chunk per GPU, no collective")}


def run_ours(args):
    import torch

    import paper_1412_4907_gb300 as bf

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    mode = INPUTS[args.input]
    scene, dirs, t_int = synth.config2(INPUT_SIGMA.get(mode))
    if args.channels:   # a band subset with the same per-channel shape (profiling captures)
        scene.freqs = scene.freqs[:args.channels]
    C_job = scene.n_chan
    if args.scaling == "strong" and world > 1:   # one band split into contiguous channel ranges
        lo, hi = shard_range(C_job, world, rank)
        scene.freqs = scene.freqs[lo:hi]
    N, C, B, T = scene.n_ant, scene.n_chan, dirs.shape[0], scene.n_samp
    T_o = T // t_int
    F = flops(N, B, C, T)
    x_host = synth.voltages(scene, mode)
    xd = torch.from_numpy(x_host).cuda()
    stream = torch.cuda.current_stream()
    plan = bf.Plan(scene.pos, scene.freqs, dirs, mode, t_int, stream=stream)
    plan.set_weight_buffers(2)   # the refresh for chunk i+1 overlaps the beamforming of chunk i
    out = torch.empty((B, C, T_o), dtype=torch.float32, device="cuda")
    dirs_alt = [dirs, synth.beam_grid(32, 32, 9.99)]   # re-pointed every chunk

    def step(i, ev=None):
        bf.bf_weights(plan.handle, dirs_alt[i % 2])     # on the plan's weight stream
        if ev is not None:
            ev[0].record(stream)
        bf.bf_execute(plan.handle, xd.data_ptr(), T, out.data_ptr(), stream.cuda_stream)
        if ev is not None:
            ev[1].record(stream)

    # the weight refresh alone (for the breakdown): host-timed, synchronised
    plan.sync()
    t0w = time.perf_counter()
    for i in range(10):
        bf.bf_weights(plan.handle, dirs_alt[i % 2])
        plan.sync()
    w_ms = (time.perf_counter() - t0w) / 10 * 1e3
    for i in range(args.warmup):
        step(i)
    plan.sync()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    if rank == 0:
        clocks.start()
        time.sleep(0.5)   # let nvidia-smi start sampling
        clocks.mark_start()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for i in range(args.steps):
        step(i, evs[i])
    t_end.record(stream)
    torch.cuda.synchronize()
    clocks.mark_stop()
    clk = clocks.stop() if rank == 0 else None
    plan.sync()
    total_ms = t_start.elapsed_time(t_end)
    k_ms = statistics.mean(e[0].elapsed_time(e[1]) for e in evs)
    total_ms = max_over_ranks(total_ms, dist, "cuda")
    ms_step = total_ms / args.steps
    # units all ranks processed / slowest rank's time
    F_job = flops(N, B, C_job, T) if args.scaling == "strong" else world * F
    value = F_job / (ms_step * 1e-3) / 1e12

    # end to end through the public host-memory call (copies inside the timed region)
    e2e = None
    if not args.no_e2e:
        xh = torch.from_numpy(x_host).pin_memory()
        ph = torch.empty((B, C, T_o), dtype=torch.float32).pin_memory()
        n_e2e = max(3, args.steps // 2)
        for i in range(2):
            bf.bf_weights(plan.handle, dirs_alt[i % 2])
            bf.bf_execute_host(plan.handle, xh.data_ptr(), T, ph.data_ptr())
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        for i in range(n_e2e):
            bf.bf_weights(plan.handle, dirs_alt[i % 2])
            bf.bf_execute_host(plan.handle, xh.data_ptr(), T, ph.data_ptr())
        e2e_s = max_over_ranks((time.perf_counter() - t0) / n_e2e, dist, "cuda")
        e2e = {"value": F_job / e2e_s / 1e12, "unit": UNIT, "ms_per_step": e2e_s * 1e3,
               "h2d_bytes_per_step": int(x_host.nbytes), "d2h_bytes_per_step": int(B * C * T_o * 4)}
        del xh, ph

    # the plain FP32 form (IEEE FFMA on CUDA cores) on the same workload
    fp32 = None
    if not args.no_fp32_form:
        x32 = torch.from_numpy(synth.voltages(scene, synth.C32)).cuda()
        p32 = bf.Plan(scene.pos, scene.freqs, dirs, bf.BF_C32, t_int, stream=stream)
        p32.execute(x32, out)
        torch.cuda.synchronize()
        a, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        n32 = 3
        for _ in range(n32):
            p32.execute(x32, out)
        b_.record(stream)
        torch.cuda.synchronize()
        ms32 = a.elapsed_time(b_) / n32
        p32.close()
        del x32
        # the FFMA peak measured now, with the SM clock sampled during the probe
        probe_clk = ClockSampler(local)
        probe_clk.start()
        time.sleep(0.3)
        probe_clk.mark_start()
        ffma = bf.bf_measure_ffma(1.0)
        probe_clk.mark_stop()
        pclk = probe_clk.stop()
        tf32 = F / (ms32 * 1e-3) / 1e12
        fp32 = {"value": tf32, "unit": UNIT, "ms_per_step": ms32, "dtype": "f32",
                "kernel": "k_simt_pipe (FP32 FFMA)",
                "roofline": {"bound": "alu", "achieved": tf32, "peak": ffma, "unit": "TFLOP/s", "frac": tf32 / ffma,
                             "peak_source": "bf_measure_ffma: independent FFMA chains on every SM, 1 s, measured "
                                            "in this run",
                             "peak_clock_sm_mhz": pclk["sm_mhz"] if pclk else None}}

    if rank != 0:
        plan.close()
        if dist:
            dist.destroy_process_group()
        return

    pk, pk_kind = peaks()
    # the timed region (K steps back to back) is held against the burst peak
    # when it lasts under a second, else against the sustained one
    peak, peak_src, burst, sust = roofline_peak(pk, pk_kind, total_ms)
    achieved = F / (k_ms * 1e-3) / 1e12
    alg_bytes = x_host.nbytes + B * C * T_o * 4
    w_bytes = C * (B // 64) * 128 * 64 * 2
    hbm = pk["hbm_gbs"]
    roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "frac_burst": achieved / burst, "frac_sustained": achieved / sust,
            "traffic": profiled_traffic() if mode == synth.C16F else None,
            "kernel": "k_tc (fused beamform+detect+integrate)",
            "peak_source": peak_src + " (FP16 = BF16 rate)", "timed_region_ms": total_ms,
            "algorithmic_bytes": alg_bytes + w_bytes,
            "hbm_frac": (alg_bytes + w_bytes) / (k_ms * 1e-3) / 1e9 / hbm}
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        cores = os.cpu_count() or 1
        n_chan = min(C, cores)
        r, dt = cpu_oracle_rate(scene, dirs, t_int, n_chan)
        if dt < 8.0:   # grow the sample towards ~10-30 s of CPU work
            n_chan = min(C, n_chan * max(1, int(round(12.0 / max(dt, 1e-3)))))
            r, dt = cpu_oracle_rate(scene, dirs, t_int, n_chan)
        cpu = {"value": r, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{n_chan} of 1024 channels (all beams, all samples), {dt:.1f} s"}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": args.scaling,
            "vs_baseline": None, "dtype": {synth.C16F: "f16", synth.CI8: "i8", synth.CI4: "i4"}[mode],
            "data": "synthetic: seeded complex Gaussian noise + 3 plane waves",
            "config": config_dict(scene, dirs, t_int, args.scaling, mode), "roofline": roof, "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": 3 * args.steps * 1,
            "breakdown_ms": {"beamform": k_ms, "weights_alone": w_ms,
                             "weights": "refreshed every chunk on a side stream, overlapped with the beamformer"},
            "fp32_form": fp32, "clocks": clk}
    plan.close()
    del xd, out
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    # the target forms beside the headline chunk (after it, so its buffers are free)
    if not args.no_batched and world == 1 and not args.channels:
        line["batched"] = batched_measure(args, emit=False)
    if not args.no_serve and world == 1 and not args.channels:
        line["serve"] = {f"{r:g}_chunks_per_s": serve_summary(serve_measure(args, r, args.serve_seconds, emit=False))
                         for r in (args.serve_rate, args.serve_rate_within_link)}
        if not args.no_fp32_form:
            line["fp32_serve"] = fp32_serve_measure(args, args.serve_rate, args.serve_seconds, args.serve_fp32_chunks,
                                                    emit=False)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def serve_summary(r):
    """The figures of a serving run that the headline line carries."""
    keys = ("chunks", "rate_hz", "seconds_offered", "latency_ms", "latency_from_step_start_ms", "offered_tflops",
            "device_tflops", "device_busy_frac", "roofline", "h2d_gbps_offered", "h2d_gbps_achieved",
            "h2d_gbps_while_copying", "copy_in_busy_frac", "mean_chunks_per_step")
    d = {k: r[k] for k in keys}
    d["sustained_tflops"] = r["value"]
    return d


def run_sweep(args):
    """Precision sweep on the config-3 shape (256 antennas on a 200 m random
    layout, 2048 beams, 8192 samples, T_int 64) over the first ``--channels``
    channels (default 256): per mode, fused-kernel TFLOP/s and roofline
    fraction, and the power error on two sampled channels against the FP64
    oracle fed the same stored values (kernel error) and fed the unquantised
    FP32 base voltages (end to end).  One JSON line per mode."""
    import torch

    import oracle
    import paper_1412_4907_gb300 as bf
    torch.cuda.set_device(0)
    n_chan = args.channels or 256
    scene, dirs, t_int = synth.config3(n_chan=n_chan)
    N, B, T = scene.n_ant, dirs.shape[0], scene.n_samp
    F = flops(N, B, n_chan, T)
    pk, pk_kind = peaks()
    # tensor peak per operand type: FP8 runs at twice the 16-bit rate; int8 and
    # 4-bit inputs are multiplied as FP16; FP32 runs on the CUDA cores
    ratio = {synth.C16F: 1.0, synth.C16BF: 1.0, synth.C8E4M3: 2.0, synth.CI8: 1.0}
    chans = [3, n_chan - 5]
    x32_sub = synth.voltages(scene, synth.C32, channels=chans).view(np.complex64).astype(np.complex128)
    sub_freqs = scene.freqs[chans]
    W64 = oracle.weights(scene.pos, sub_freqs, dirs)
    P64 = oracle.power(W64, x32_sub, t_int)
    stream = torch.cuda.current_stream()
    for mode in (synth.C32, synth.C16F, synth.C16BF, synth.C8E4M3, synth.CI8):
        x = synth.voltages(scene, mode)
        xd = torch.from_numpy(x).cuda()
        del x
        plan = bf.Plan(scene.pos, scene.freqs, dirs, mode, t_int, stream=stream)
        out = torch.empty((B, n_chan, T // t_int), dtype=torch.float32, device="cuda")
        for _ in range(2):
            plan.execute(xd, out)
        torch.cuda.synchronize()
        a, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        n = max(3, min(args.steps, 20))
        a.record(stream)
        for _ in range(n):
            plan.execute(xd, out)
        b_.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b_) / n
        plan.sync()
        P = out[:, chans, :].cpu().numpy()
        xs = synth.voltages(scene, mode, channels=chans)
        Wq = W64 if mode == synth.C32 else oracle.quantised_weights(W64, mode)[0]
        Pq = oracle.power(Wq, oracle.decode_voltages(mode, xs), t_int)
        kmx, kl2 = power_errors(P, Pq)
        emx, el2 = power_errors(P, P64)
        q = plan.query_tiles()
        plan.close()
        del xd, out
        tf = F / (ms * 1e-3) / 1e12
        pkm, pk_src, _, pks = roofline_peak(pk, pk_kind, ms * n, ratio.get(mode, 1.0), "FP8")
        line = {"metric": "precision sweep: fused beamform TFLOP/s and power error vs FP64", "mode": synth.MODE_NAMES[mode],
                "value": tf, "unit": UNIT, "ms_per_launch": ms,
                "roofline": None if mode == synth.C32 else {"bound": "tensor", "achieved": tf, "peak": pkm,
                                                            "frac": tf / pkm, "frac_sustained": tf / pks,
                                                            "unit": "TFLOP/s", "peak_source": pk_src},
                "error_kernel": {"max_rel": kmx, "l2_rel": kl2},
                "error_vs_fp64": {"max_rel": emx, "l2_rel": el2, "channels": chans},
                "tiling": q, "config": {"workload": f"config-3 shape: 256 antennas, 2048 beams, 8192 samples, T_int 64, "
                                                    f"{n_chan} of 4096 channels", "input_sigma": 16.0}}
        print(json.dumps(line), flush=True)


def config4_inputs(jobs, torch, device="cuda"):
    """Seeded FP16 voltages [C][T][2N] of the batched workload, made on the
    device (74 GB in all: too much to build on the host in a bench run):
    complex Gaussian noise (sigma 1/sqrt(2) per component) plus one plane
    wave per job (SNR 10 dB per antenna and sample, noise-like signal,
    phase exp(+i 2 pi f_c r_n . s / c0))."""
    xs = []
    c0 = 299792458.0
    for j, job in enumerate(jobs):
        N, C, T = job.scene.pos.shape[0], job.scene.freqs.size, job.scene.n_samp
        g = torch.Generator(device=device)
        g.manual_seed(4_000_000 + j)
        x = torch.empty((C, T, 2 * N), dtype=torch.float16, device=device)
        src = job.scene.sources[0]
        a = float(np.sqrt(src.power / 2.0))                           # CN(0, power) per sample
        tau = job.scene.pos @ src.dir / c0                             # [N] seconds
        for c0_ in range(0, C, 64):
            c1 = min(C, c0_ + 64)
            ph = np.outer(job.scene.freqs[c0_:c1], tau)                # [c][N] cycles
            ph = torch.from_numpy(np.exp(2j * np.pi * (ph - np.rint(ph))).astype(np.complex64)).to(device)
            s = torch.randn((c1 - c0_, T, 2), generator=g, device=device) * a
            s = torch.view_as_complex(s)                               # [c][T]
            n = torch.randn((c1 - c0_, T, N, 2), generator=g, device=device) * 0.7071067811865476
            v = torch.view_as_real(s[:, :, None] * ph[:, None, :]) + n
            x[c0_:c1] = v.reshape(c1 - c0_, T, 2 * N).half()
        xs.append(x)
    return xs


def roofline_peak(pk, pk_kind, region_ms, ratio=1.0, what="BF16"):
    """The tensor peak a measured region is held against: the burst figure for
    a region shorter than a second (the GPU has not settled at its power
    limit), the sustained one for longer regions; both fractions are kept."""
    burst, sust = pk["bf16_tflops"] * ratio, pk["bf16_tflops_sustained"] * ratio
    use_burst = region_ms < 1000.0
    src = ("bf16_tflops (burst)" if use_burst else "bf16_tflops_sustained") + f", {pk_kind}"
    if ratio != 1.0:
        src += f" x {ratio:g} (nominal {what} ratio)"
    return (burst if use_burst else sust), src, burst, sust


def run_batched(args):
    batched_measure(args, emit=True)


def batched_measure(args, emit=True):
    """Config 4: 48 sub-array jobs of uneven size (N in {16..256}, B
    log-uniform in 8..4096, C in {128, 512, 2048}, T = 4096, FP16, T_int 64)
    in one graph-captured batch step: the jobs of 128 and 256 antennas in one
    persistent launch, the others in their plans' resident-weight kernel on
    forked streams.  Variants: fixed 128-sample
    tiles, the autotuned tile width, and the jobs run one plan at a time
    through bf_execute (each with the single-plan planner's tiling); plus the
    power error on sampled channels against the oracle.  With ``emit`` one
    JSON line per variant is printed; the summary dict is returned."""
    import torch

    import oracle
    import paper_1412_4907_gb300 as bf
    from paper_1412_4907_gb300 import tune
    torch.cuda.set_device(0)
    div = max(1, args.batched_chan_div)
    jobs = synth.config4_jobs(chan_choices=(128 // div, 512 // div, 2048 // div))
    if args.batched_ant:   # a subset of the jobs by antenna count (diagnostics)
        keep = {int(v) for v in args.batched_ant.split(",")}
        jobs = [j for j in jobs if j.scene.pos.shape[0] in keep]
    stream = torch.cuda.Stream()
    plans, outs, n_samps = [], [], []
    F = 0.0
    for job in jobs:
        N, B, C, T = job.scene.pos.shape[0], job.dirs.shape[0], job.scene.freqs.size, job.scene.n_samp
        plans.append(bf.Plan(job.scene.pos, job.scene.freqs, job.dirs, bf.BF_C16F, job.t_int, stream=stream))
        outs.append(torch.empty((B, C, T // job.t_int), dtype=torch.float32, device="cuda"))
        n_samps.append(T)
        F += flops(N, B, C, T)
    xs = config4_inputs(jobs, torch)
    torch.cuda.synchronize()
    # kernels per batch step: one persistent launch for the streamed-weight
    # plans, one resident-weight launch per other plan
    n_res = sum(bf.bf_plan_query_tiles(p.handle)["x_stages"] > 0 for p in plans)
    step_launches = n_res + (1 if n_res < len(plans) else 0)
    pk, pk_kind = peaks()
    steps = max(3, min(args.steps, 20))
    warm = max(3, min(args.warmup, 5))
    summary = {"workload": "48 sub-array jobs: N in {16,32,64,128,256} of the 256-antenna 200 m layout, "
                           "B log-uniform 8..4096, C in {128,512,2048}" + (f" / {div}" if div > 1 else "")
                           + ", T 4096 FP16, T_int 64, one graph-captured batch step",
               "total_tflop": F / 1e12, "steps": steps, "warmup": warm}

    def timed(run):
        for _ in range(warm):
            run()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        stream.synchronize()
        a.record(stream)
        for _ in range(steps):
            run()
        b.record(stream)
        b.synchronize()
        return a.elapsed_time(b) / steps

    def line(variant, ms, extra, key):
        tf = F / (ms * 1e-3) / 1e12
        peak, src, burst, sust = roofline_peak(pk, pk_kind, ms * steps)
        summary[key] = {"ms_per_step": ms, "tflops": tf, "frac": tf / peak, "frac_burst": tf / burst,
                        "frac_sustained": tf / sust, "peak_source": src,
                        **{k: v for k, v in extra.items() if k != "tuning_table"}}
        if not emit:
            return
        d = {"metric": "batched uneven launch: beamform TFLOP/s", "variant": variant, "value": tf, "unit": UNIT,
             "ms_per_step": ms, "steps": steps, "warmup": warm, "dtype": "f16", "data": "synthetic",
             "roofline": {"bound": "tensor", "achieved": tf, "peak": peak, "unit": "TFLOP/s", "frac": tf / peak,
                          "frac_sustained": tf / sust, "peak_source": src},
             "config": {"workload": "48 sub-array jobs: N in {16,32,64,128,256} of the 256-antenna 200 m layout, "
                                    "B log-uniform 8..4096, C in {128,512,2048}" + (f" / {div}" if div > 1 else "")
                                    + ", T 4096 FP16, T_int 64",
                        "total_tflop": F / 1e12, "jobs": len(jobs),
                        "l2": "no flush: 74 GB of voltages and 21 GB of weights per step exceed the 129 MB L2"}}
        d.update(extra)
        print(json.dumps(d), flush=True)

    if args.batched_tile:
        # one given tile width only: no fixed-width variant, no tuning (the
        # first launches of the run are then the measured steps: for profiling)
        ms_fixed = None
        tuned = {"tile_t": args.batched_tile, "table": []}
    else:
        # fixed tiles
        batch = bf.Batch(plans, tile_t=128, stream=stream)
        for j, (x, o, T) in enumerate(zip(xs, outs, n_samps)):
            batch.set(j, x, o, n_samp=T)
        batch.capture()
        ms_fixed = timed(batch.replay)
        batch.sync()
        line("batched, fixed 128-sample tiles", ms_fixed, {"tile_t": 128, "gpu_launches_per_step": step_launches},
             "fixed_128")
        batch.close()
        # autotuned
        tuned = tune.tune_batch(plans, xs, outs, n_samps, stream=stream, reps=3, cache=None)
    batch = bf.Batch(plans, tile_t=tuned["tile_t"], stream=stream)
    for j, (x, o, T) in enumerate(zip(xs, outs, n_samps)):
        batch.set(j, x, o, n_samp=T)
    batch.capture()
    ms_tuned = timed(batch.replay)
    batch.sync()
    line("batched, autotuned tile" if not args.batched_tile else f"batched, {args.batched_tile}-sample tiles",
         ms_tuned, {"tile_t": tuned["tile_t"], "tuning_table": tuned["table"],
                    "speedup_vs_fixed": ms_fixed / ms_tuned if ms_fixed else None,
                    "gpu_launches_per_step": step_launches},
         "autotuned")
    # one plan at a time
    def per_plan():
        for p, x, o, T in zip(plans, xs, outs, n_samps):
            bf.bf_execute(p.handle, x.data_ptr(), T, o.data_ptr(), stream.cuda_stream)
    ms_seq = timed(per_plan)
    line("one launch per job (bf_execute)", ms_seq, {"gpu_launches_per_step": len(plans),
                                                     "batched_speedup": ms_seq / ms_tuned}, "one_launch_per_job")
    # parity on sampled channels of four jobs (batched, autotuned outputs)
    batch.replay()
    batch.sync()
    errs = []
    order = sorted(range(len(jobs)), key=lambda j: plans[j].N * plans[j].B)
    for j in (order[0], order[len(order) // 3], order[2 * len(order) // 3], order[-1]):
        job, p = jobs[j], plans[j]
        c = p.C // 2
        xh = xs[j][c:c + 1].cpu().numpy().view(np.float16)
        X64 = oracle.decode_voltages(synth.C16F, xh)
        W = oracle.weights(job.scene.pos, job.scene.freqs[c:c + 1], job.dirs)
        Wq = oracle.quantised_weights(W, synth.C16F)[0]
        Pref = oracle.power(Wq, X64, job.t_int)
        mx, l2 = power_errors(outs[j][:, c:c + 1, :].cpu().numpy(), Pref)
        errs.append({"job": j, "N": p.N, "B": p.B, "channel": c, "max_rel": mx, "l2_rel": l2})
    batch.close()
    summary["parity_vs_oracle"] = {"max_rel": max(e["max_rel"] for e in errs), "l2_rel": max(e["l2_rel"] for e in errs),
                                   "jobs_sampled": len(errs)}
    if emit:
        print(json.dumps({"metric": "batched uneven launch: power error vs FP64 oracle (same FP16 inputs and weights)",
                          "samples": errs}), flush=True)
    for p in plans:
        p.close()
    del xs, outs
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    return summary


SERVE_CONFIGS = [(32, 1024, 1024, synth.C16F), (64, 64, 4096, synth.CI8), (128, 512, 2048, synth.C16F),
                 (256, 2048, 512, synth.CI8), (512, 8192, 256, synth.C16F), (512, 256, 4096, synth.CI8)]
SERVE_RATE_HZ = 1024          # samples per second per channel: a chunk of d seconds has round(1024 d) samples


def serve_plans(bf, stream, mode_override=None):
    plans = []
    for i, (N, B, C, mode) in enumerate(SERVE_CONFIGS):
        pos = synth.grid_positions() if N == 32 else synth.random_positions(N, 200.0, 500 + i)
        nx = int(round(np.sqrt(B)))
        dirs = synth.beam_grid(nx, -(-B // nx))[:B]
        freqs = synth.channel_freqs(400e6, 16e6, C)
        plans.append(bf.Plan(pos, freqs, dirs, mode if mode_override is None else mode_override, 64, stream=stream))
    return plans


def serve_arrivals(rate, seconds, seed=5):
    """Poisson arrivals: (time offset s, config, samples per channel)."""
    g = np.random.default_rng(seed)
    t, out = 0.0, []
    while True:
        t += g.exponential(1.0 / rate)
        if t >= seconds:
            return out
        cfg = int(g.integers(0, len(SERVE_CONFIGS)))
        T = int(round(g.uniform(0.25, 1.0) * SERVE_RATE_HZ))
        out.append((t, cfg, T))


def serve_pool(torch, mode, N, C, T, seed):
    """One pinned host chunk [C][T][N] of the mode's dtype (seeded noise made
    on the device: FP16 sigma 1/sqrt(2) per component, int8 sigma 16 clipped)."""
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    v = torch.randn((C, T, 2 * N), generator=g, device="cuda")
    if mode == synth.CI8:
        v = torch.clamp(torch.round(v * 16.0), -127, 127).to(torch.int8)
    else:
        v = (v * 0.7071067811865476).to(torch.float16 if mode == synth.C16F else torch.float32)
    h = torch.empty(v.shape, dtype=v.dtype).pin_memory()
    h.copy_(v)
    return h


def pct(a, q):
    return float(np.percentile(np.asarray(a), q)) if len(a) else None


def run_serve(args):
    serve_measure(args, args.serve_rate, args.serve_seconds, emit=True)
    if not args.no_fp32_form:
        fp32_serve_measure(args, args.serve_rate, args.serve_seconds, args.serve_fp32_chunks, emit=True)


def serve_measure(args, rate, seconds, emit=True):
    """Config 5: Poisson arrivals (``rate`` chunks/s for ``seconds``) of
    0.25-1 s chunks from 6 streams (32-512 antennas, 64-8192 beams, 256-4096
    channels, FP16 or int8), served by bf_server: latency from arrival on the
    host to powers in host memory (p50/p99), sustained and device-only
    TFLOP/s.  Prints one JSON line with ``emit``; returns the result dict."""
    import threading

    import torch

    import paper_1412_4907_gb300 as bf
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    plans = serve_plans(bf, stream)
    pools, rings = [], []
    for i, (N, B, C, mode) in enumerate(SERVE_CONFIGS):
        pools.append(serve_pool(torch, mode, N, C, SERVE_RATE_HZ, 5000 + i))
        rings.append([torch.empty(B * C * (SERVE_RATE_HZ // 64 + 1), dtype=torch.float32).pin_memory()
                      for _ in range(4)])
    torch.cuda.synchronize()
    server = bf.Server(plans, mem_bytes=int(args.serve_mem * 2**30), max_steps=args.serve_steps)
    for i in range(len(SERVE_CONFIGS)):   # warm-up: one chunk per stream
        server.submit(i, pools[i], rings[i][0], n_samp=256)
    server.drain(120000)
    server.poll(64)
    base = server.stats()
    arrivals = serve_arrivals(rate, seconds)
    series, stop = [], [False]

    def sample():   # link and device counters every 0.5 s, to see the rates over the run
        last = server.stats()
        while not stop[0]:
            time.sleep(0.5)
            st_ = server.stats()
            db = st_["copy_in_bytes"] - last["copy_in_bytes"]
            dm = st_["copy_in_ms"] - last["copy_in_ms"]
            series.append({"t": round(bf.bf_server_now() - t0, 2), "copy_gbps": round(db / (dm * 1e-3) / 1e9, 1)
                           if dm else None, "copy_busy": round(dm * 1e-3 / 0.5, 2),
                           "kernel_busy": round((st_["kernel_ms"] - last["kernel_ms"]) * 1e-3 / 0.5, 2),
                           "done": st_["completed"] - base["completed"]})
            last = st_

    t0 = bf.bf_server_now() + 0.05
    sampler = threading.Thread(target=sample, daemon=True)
    sampler.start()
    ids = {}
    for k, (ta, cfg, T) in enumerate(arrivals):
        due = t0 + ta
        while True:
            d = due - bf.bf_server_now()
            if d <= 0:
                break
            if d > 0.002:
                time.sleep(d - 0.001)
        i = server.submit(cfg, pools[cfg], rings[cfg][k % 4], n_samp=T)
        ids[i] = (due, cfg, T)
    t_sub_end = bf.bf_server_now()
    server.drain(600000)
    stop[0] = True
    sampler.join()
    done = {}
    while len(done) < len(ids):
        for c in server.poll(1024, 1000):
            done[c["id"]] = c
    st = server.stats()
    server.close()
    lat, lat_dev, per_cfg = [], [], {}
    t_last = t0
    F = 0.0
    h2d = 0
    for i, (due, cfg, T) in ids.items():
        c = done[i]
        assert c["status"] == 0, c
        lat.append(c["t_done"] - due)
        lat_dev.append(c["t_done"] - c["t_start"])
        per_cfg.setdefault(cfg, []).append(c["t_done"] - due)
        t_last = max(t_last, c["t_done"])
        N, B, C, mode = SERVE_CONFIGS[cfg]
        F += flops(N, B, C, T)
        h2d += C * T * N * (4 if mode == synth.C16F else 2)
    kernel_ms = st["kernel_ms"] - base["kernel_ms"]
    copy_ms = st["copy_in_ms"] - base["copy_in_ms"]
    copy_b = st["copy_in_bytes"] - base["copy_in_bytes"]
    steps = st["steps"] - base["steps"]
    sustained = F / (t_last - t0) / 1e12
    pk, pk_kind = peaks()
    dev_tf = F / (kernel_ms * 1e-3) / 1e12
    peak, src, burst, sust = roofline_peak(pk, pk_kind, kernel_ms)
    res = {"metric": "serving stream: p50/p99 chunk latency and sustained TFLOP/s", "value": sustained,
           "unit": UNIT, "higher_is_better": True, "dtype": "f16 (int8 inputs widened to f16)", "data": "synthetic",
           "chunks": len(ids), "seconds_offered": seconds, "rate_hz": rate,
           "latency_ms": {"p50": 1e3 * pct(lat, 50), "p99": 1e3 * pct(lat, 99), "mean": 1e3 * float(np.mean(lat)),
                          "max": 1e3 * float(np.max(lat))},
           "latency_from_step_start_ms": {"p50": 1e3 * pct(lat_dev, 50), "p99": 1e3 * pct(lat_dev, 99)},
           "latency_p99_ms_per_config": {str(k): 1e3 * pct(v, 99) for k, v in sorted(per_cfg.items())},
           "offered_tflops": F / seconds / 1e12, "device_tflops": dev_tf,
           "device_busy_frac": kernel_ms * 1e-3 / (t_last - t0),
           "roofline": {"bound": "tensor", "achieved": dev_tf, "peak": peak, "unit": "TFLOP/s", "frac": dev_tf / peak,
                        "frac_sustained": dev_tf / sust, "peak_source": src},
           "h2d_gbps_offered": h2d / seconds / 1e9, "h2d_gbps_achieved": h2d / (t_last - t0) / 1e9,
           "h2d_gbps_while_copying": copy_b / (copy_ms * 1e-3) / 1e9 if copy_ms else None,
           "copy_in_busy_frac": copy_ms * 1e-3 / (t_last - t0),
           "steps": steps, "mean_chunks_per_step": len(ids) / max(1, steps), "max_chunks_per_step": st["max_jobs_per_step"],
           "arena_gb": st["arena_bytes"] / 2**30, "arena_peak_gb": st["arena_peak"] / 2**30,
           "submit_lag_s": t_sub_end - (t0 + arrivals[-1][0]) if arrivals else 0.0,
           "config": {"workload": "6 streams (32,1024,1024,f16) (64,64,4096,i8) (128,512,2048,f16) (256,2048,512,i8) "
                                  "(512,8192,256,f16) (512,256,4096,i8) as (N,B,C,dtype); Poisson arrivals, chunk "
                                  "0.25-1 s at 1024 samples/s per channel, T_int 64 with the open window carried",
                      "tile_t": st["tile_t"], "max_steps": args.serve_steps, "arena_gib": args.serve_mem}}
    if emit:
        print(json.dumps({**res, "series_0p5s": series}), flush=True)
    for p in plans:
        p.close()
    del pools, rings
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    return res


def fp32_serve_measure(args, rate, seconds, n_chunks, emit=True):
    """The plain FP32 single-job path (bf_execute_host: one chunk at a time,
    FP32 voltages, the CUDA-core kernel) served on the first ``n_chunks``
    arrivals of the same Poisson list, in real time: each chunk starts when
    it has arrived and the previous one is done, and its latency runs from its
    arrival to its powers in host memory (a FIFO single-job server)."""
    import torch

    import paper_1412_4907_gb300 as bf
    torch.cuda.set_device(0)
    arrivals = serve_arrivals(rate, seconds)
    plans32 = serve_plans(bf, torch.cuda.current_stream(), mode_override=synth.C32)
    n32 = min(len(arrivals), n_chunks)
    need = max(C * T * N for (_, cfg, T) in arrivals[:n32] for (N, _, C, _) in [SERVE_CONFIGS[cfg]])
    xh = torch.empty(2 * need, dtype=torch.float32).pin_memory()
    xh.normal_(0.0, 0.7071067811865476)
    outh = torch.empty(max(B * C * (SERVE_RATE_HZ // 64 + 1) for (_, B, C, _) in SERVE_CONFIGS),
                       dtype=torch.float32).pin_memory()
    for i in range(len(plans32)):   # warm-up
        bf.bf_execute_host(plans32[i].handle, xh.data_ptr(), 64, outh.data_ptr())
    svc, lat, F32 = [], [], 0.0
    t0 = time.perf_counter() + 0.01
    for (ta, cfg, T) in arrivals[:n32]:
        due = t0 + ta
        while time.perf_counter() < due:
            pass
        a = time.perf_counter()
        bf.bf_execute_host(plans32[cfg].handle, xh.data_ptr(), T, outh.data_ptr())
        b = time.perf_counter()
        svc.append(b - a)
        lat.append(b - due)
        N, B, C, _ = SERVE_CONFIGS[cfg]
        F32 += flops(N, B, C, T)
    busy = sum(svc)
    res = {"metric": "serving stream: plain FP32 single-job path (bf_execute_host, one chunk at a time)",
           "value": F32 / busy / 1e12, "unit": UNIT, "dtype": "f32", "chunks": n32, "rate_hz": rate,
           "latency_ms": {"p50": 1e3 * pct(lat, 50), "p99": 1e3 * pct(lat, 99), "max": 1e3 * max(lat)},
           "service_ms": {"p50": 1e3 * pct(svc, 50), "p99": 1e3 * pct(svc, 99)},
           "offered_tflops": F32 / max(arrivals[n32 - 1][0], 1e-9) / 1e12 if n32 else 0.0,
           "note": "the first chunks of the same arrival list; the queue grows whenever offered > value"}
    if emit:
        print(json.dumps(res), flush=True)
    for p in plans32:
        p.close()
    del xh, outh
    torch.cuda.synchronize()
    return res


def run_peaks(args):
    """Library GEMM rates for the dtypes whose peaks the roofline otherwise
    derives: cuBLAS SGEMM (FP32, TF32 off: the FFMA rate the FP32 beamformer
    is held against) and cuBLASLt FP8 E4M3 (torch._scaled_mm), with cuBLAS
    BF16 beside them as the cross-check against the driver's figure.  Square
    8192 GEMMs; burst = 20 back-to-back calls, sustained = a loop of about
    `--peak-seconds` seconds.  Context only: the roofline denominators stay
    the measured BF16 figures times the nominal dtype ratio."""
    import torch
    torch.cuda.set_device(0)
    dev = torch.device("cuda")
    n = 8192
    flop = 2.0 * n * n * n
    g = torch.Generator(device="cuda")
    g.manual_seed(21)
    a = torch.randn((n, n), generator=g, device=dev, dtype=torch.bfloat16)
    b = torch.randn((n, n), generator=g, device=dev, dtype=torch.bfloat16)

    def rate(fn, reps):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return flop * reps / (e0.elapsed_time(e1) * 1e-3) / 1e12

    def measure(name, fn):
        try:
            burst = rate(fn, 20)
            t_one = flop / (burst * 1e12)
            sustained = rate(fn, max(20, int(args.peak_seconds / t_one)))
            line = {"metric": "library GEMM rate (peak context)", "dtype": name, "burst_tflops": burst,
                    "sustained_tflops": sustained, "shape": [n, n, n]}
        except Exception as e:   # a dtype the installed torch/cuBLAS cannot run
            line = {"metric": "library GEMM rate (peak context)", "dtype": name, "unavailable": str(e)[:200]}
        print(json.dumps(line), flush=True)

    measure("bf16", lambda: torch.matmul(a, b))
    allow = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    a32, b32 = a.float(), b.float()
    measure("fp32 (SGEMM, TF32 off)", lambda: torch.matmul(a32, b32))
    torch.backends.cuda.matmul.allow_tf32 = allow
    del a32, b32
    a8 = a.to(torch.float8_e4m3fn)
    b8 = b.t().contiguous().to(torch.float8_e4m3fn).t()   # column-major second operand
    one = torch.ones((), device=dev, dtype=torch.float32)
    measure("fp8 e4m3", lambda: torch._scaled_mm(a8, b8, scale_a=one, scale_b=one, out_dtype=torch.bfloat16))


def run_aux(args):
    """The HBM-bound kernels on the real-time chunk's sizes (32 antennas, 1024
    channels, 15625 samples, 1024 beams, T_int 64): corner turn, incoherent
    beam, detrend-and-threshold of the powers.  One JSON line per kernel:
    algorithmic bytes / CUDA-event time against the measured copy bandwidth."""
    import torch

    import paper_1412_4907_gb300 as bf
    torch.cuda.set_device(0)
    scene, dirs, t_int = synth.config2()
    N, C, B, T = scene.n_ant, scene.n_chan, dirs.shape[0], scene.n_samp
    T_o = T // t_int
    pk, pk_kind = peaks()
    hbm = pk["hbm_gbs"]
    stream = torch.cuda.current_stream()
    g = torch.Generator(device="cuda")
    g.manual_seed(11)
    x_nct = (torch.randn((N, C, T, 2), generator=g, device="cuda") * 0.7071).half()
    x_ctn = torch.empty((C, T, N, 2), dtype=torch.float16, device="cuda")
    P = torch.rand((B, C, T_o), generator=g, device="cuda")
    z = torch.empty_like(P)
    hits = torch.empty((1 << 16, 3), dtype=torch.int32, device="cuda")
    nh = torch.zeros(1, dtype=torch.int32, device="cuda")
    plan = bf.Plan(scene.pos, scene.freqs, dirs, bf.BF_C16F, t_int, stream=stream)
    inc = torch.empty((C, T_o), dtype=torch.float32, device="cuda")
    x_ctn_in = torch.from_numpy(synth.voltages(scene, synth.C16F)).cuda()
    cases = [
        ("corner turn [N][C][T] -> [C][T][N], FP16", 2 * x_nct.numel() * 2,
         lambda: bf.bf_corner_turn(x_nct.data_ptr(), bf.BF_C16F, x_ctn.data_ptr(), bf.BF_C16F, N, C, T, None,
                                   stream.cuda_stream)),
        ("incoherent beam (sum of |X|^2 over antennas), FP16 in", x_ctn_in.numel() * 2 + inc.numel() * 4,
         lambda: bf.bf_execute_incoherent(plan.handle, x_ctn_in.data_ptr(), T, inc.data_ptr(), stream.cuda_stream)),
        ("detrend + threshold of the powers (bf_detect, z written)", P.numel() * 8,
         lambda: bf.bf_detect(P.data_ptr(), B, C, T_o, 6.0, z.data_ptr(), hits.data_ptr(), 1 << 16, nh.data_ptr(),
                              stream.cuda_stream)),
    ]
    for name, nbytes, fn in cases:
        for _ in range(3):
            fn()
        n = 10
        a, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(n):
            fn()
        b_.record(stream)
        b_.synchronize()
        ms = a.elapsed_time(b_) / n
        gbs = nbytes / (ms * 1e-3) / 1e9
        print(json.dumps({"metric": "HBM-bound kernel: algorithmic GB/s", "kernel": name, "value": gbs,
                          "unit": "GB/s", "ms": ms, "bytes": nbytes,
                          "roofline": {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s",
                                       "frac": gbs / hbm, "peak_source": f"hbm_gbs {pk_kind}"},
                          "config": {"workload": "real-time chunk sizes: 32 antennas, 1024 channels, 15625 samples, "
                                                 "1024 beams, T_int 64",
                                     "l2": "no flush: every buffer exceeds the 129 MB L2"}}), flush=True)
    plan.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp32-form", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--sweep", action="store_true",
                    help="precision sweep on the config-3 shape (one JSON line per mode) instead of the benchmark")
    ap.add_argument("--batched", action="store_true",
                    help="batched uneven launch of 48 sub-array jobs (one JSON line per variant)")
    ap.add_argument("--scaling", default="weak", choices=["weak", "strong"],
                    help="weak: every rank beamforms its own chunk; strong: the chunk's channels are split over ranks")
    ap.add_argument("--batched-ant", default="",
                    help="batched: only the jobs with these antenna counts (comma list; diagnostics)")
    ap.add_argument("--batched-tile", type=int, default=0,
                    help="batched: this tile width only, no fixed-width variant or tuning (profiling)")
    ap.add_argument("--batched-chan-div", type=int, default=1,
                    help="divide every job's channel count (smaller case of the same jobs, for profiling)")
    ap.add_argument("--peaks", action="store_true",
                    help="cuBLAS FP32 / FP8 / BF16 GEMM rates (context for the derived FP32 and FP8 peaks)")
    ap.add_argument("--peak-seconds", type=float, default=3.0, help="length of the sustained GEMM loop")
    ap.add_argument("--aux", action="store_true",
                    help="HBM-bound kernels (corner turn, incoherent beam, detection) on the chunk's sizes")
    ap.add_argument("--serve", action="store_true",
                    help="serving stream of 6 configurations with Poisson arrivals (p50/p99 latency)")
    ap.add_argument("--serve-rate", type=float, default=400.0, help="chunk arrivals per second")
    ap.add_argument("--serve-seconds", type=float, default=10.0, help="seconds of arrivals")
    ap.add_argument("--serve-mem", type=float, default=96.0, help="server arena in GiB")
    ap.add_argument("--serve-steps", type=int, default=3, help="server steps in flight (1..8)")
    ap.add_argument("--serve-fp32-chunks", type=int, default=24, help="chunks for the FP32 single-job comparison")
    ap.add_argument("--serve-rate-within-link", type=float, default=250.0,
                    help="second arrival rate of the default run (within the host link's rate)")
    ap.add_argument("--no-batched", action="store_true", help="default run: skip the batched uneven launch")
    ap.add_argument("--no-serve", action="store_true", help="default run: skip the serving runs")
    ap.add_argument("--input", default="c16f", choices=sorted(INPUTS),
                    help="sample format of the real-time chunk (default FP16; ci8/ci4: integer samples widened "
                         "inside the beamformer)")
    ap.add_argument("--channels", type=int, default=0,
                    help="run only the first C channels (same per-channel shape; for profiling)")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)   # at least 3 untimed warm-up steps
    if args.impl == "reference":
        run_reference(args)
    elif args.sweep:
        run_sweep(args)
    elif args.batched:
        run_batched(args)
    elif args.serve:
        run_serve(args)
    elif args.aux:
        run_aux(args)
    elif args.peaks:
        run_peaks(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

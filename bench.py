#!/usr/bin/env python3
"""Throughput benchmark of the GB300 beamformer on the real-time FP16 workload.

Workload: 32 antennas (BEST-2 4 x 8 grid), 1024 channels over 16 MHz, 1024
beams over +-10 deg, 15625 FP16 complex samples per channel (one 1 s chunk),
noise plus 3 plane waves, integration over 64 samples.

One step = one pass of the per-chunk path on one chunk already resident in
HBM: the weight refresh (delay + weight kernels, the tracking-beam update of
Section 3.1) followed by the fused tensor-core beamform + |B|^2 + integrate
kernel (no corner turn: the input is already channel-major).  FLOPs are
counted as 8 N per beam, channel and sample (Section 2.2).

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle instead, on a bounded channel sample of the same workload.
"""
import argparse
import hashlib
import json
import os
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


def kernel_source_sha():
    h = hashlib.sha256()
    for f in ("k_tc.cu", "tc_common.cuh", "ptx.cuh", "bf_internal.h"):
        h.update(open(os.path.join(ROOT, "paper_1412_4907_gb300", "csrc", f), "rb").read())
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
    """nvidia-smi clocks and throttle reasons sampled every 100 ms; only the
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
                 "-i", str(self.gpu), "-lms", "100", "-f", self.path],
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
            "config": config_dict(scene, dirs, t_int),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def config_dict(scene, dirs, t_int):
    return {"workload": f"real-time FP16 chunk: 32-antenna BEST-2 grid, {scene.n_chan} channels x 15625 "
                        "samples, 1024 beams, T_int 64",
            "n_ant": scene.n_ant, "n_chan": scene.n_chan, "n_beam": int(dirs.shape[0]),
            "n_samp": scene.n_samp, "t_int": t_int, "input": "c16f, [c][t][n] (no corner turn)",
            "l2": "no flush: voltages (2.05 GB) and weights (0.27 GB) exceed the 129 MB L2",
            "parallelism": "channels: one independent chunk per GPU, no collective"}


def run_ours(args):
    import torch

    import paper_1412_4907_gb300 as bf

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    scene, dirs, t_int = synth.config2()
    if args.channels:   # a band subset with the same per-channel shape (profiling captures)
        scene.freqs = scene.freqs[:args.channels]
    N, C, B, T = scene.n_ant, scene.n_chan, dirs.shape[0], scene.n_samp
    T_o = T // t_int
    F = flops(N, B, C, T)
    x_host = synth.voltages(scene, synth.C16F)
    xd = torch.from_numpy(x_host).cuda()
    stream = torch.cuda.current_stream()
    plan = bf.Plan(scene.pos, scene.freqs, dirs, bf.BF_C16F, t_int, stream=stream)
    out = torch.empty((B, C, T_o), dtype=torch.float32, device="cuda")
    dirs_alt = [dirs, synth.beam_grid(32, 32, 9.99)]   # re-pointed every chunk

    def step(i, ev=None):
        if ev is not None:
            ev[0].record(stream)
        bf.bf_weights(plan.handle, dirs_alt[i % 2])
        if ev is not None:
            ev[1].record(stream)
        bf.bf_execute(plan.handle, xd.data_ptr(), T, out.data_ptr(), stream.cuda_stream)
        if ev is not None:
            ev[2].record(stream)

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
    w_ms = statistics.mean(e[0].elapsed_time(e[1]) for e in evs)
    k_ms = statistics.mean(e[1].elapsed_time(e[2]) for e in evs)
    if dist:
        t = torch.tensor([total_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_step = total_ms / args.steps
    value = world * F / (ms_step * 1e-3) / 1e12

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
        e2e_s = (time.perf_counter() - t0) / n_e2e
        if dist:
            t = torch.tensor([e2e_s], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e2e_s = float(t.item())
        e2e = {"value": world * F / e2e_s / 1e12, "unit": UNIT, "ms_per_step": e2e_s * 1e3,
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
        fp32 = {"value": F / (ms32 * 1e-3) / 1e12, "unit": UNIT, "ms_per_step": ms32, "dtype": "f32",
                "kernel": "k_simt (FP32 FFMA)"}

    if rank != 0:
        plan.close()
        if dist:
            dist.destroy_process_group()
        return

    pk, pk_kind = peaks()
    peak = pk["bf16_tflops_sustained"]
    achieved = F / (k_ms * 1e-3) / 1e12
    alg_bytes = x_host.nbytes + B * C * T_o * 4
    w_bytes = C * (B // 64) * 128 * 64 * 2
    hbm = pk["hbm_gbs"]
    roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": profiled_traffic(), "kernel": "k_tc (fused beamform+detect+integrate)",
            "peak_source": f"bf16_tflops_sustained, {pk_kind} (FP16 = BF16 rate)",
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
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f16", "data": "synthetic: seeded complex Gaussian noise + 3 plane waves",
            "config": config_dict(scene, dirs, t_int), "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": 3 * args.steps * 1,
            "breakdown_ms": {"weights": w_ms, "beamform": k_ms},
            "fp32_form": fp32, "clocks": clk}
    print(json.dumps(line), flush=True)
    plan.close()
    if dist:
        dist.destroy_process_group()


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
    bf16_peak = pk["bf16_tflops_sustained"]
    # tensor peak per operand type: FP8 runs at twice the 16-bit rate; int8 and
    # 4-bit inputs are multiplied as FP16; FP32 runs on the CUDA cores
    peak = {synth.C16F: bf16_peak, synth.C16BF: bf16_peak, synth.C8E4M3: 2 * bf16_peak,
            synth.CI8: bf16_peak}
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
        line = {"metric": "precision sweep: fused beamform TFLOP/s and power error vs FP64", "mode": synth.MODE_NAMES[mode],
                "value": tf, "unit": UNIT, "ms_per_launch": ms,
                "roofline": None if mode == synth.C32 else {"bound": "tensor", "achieved": tf, "peak": peak[mode],
                                                            "frac": tf / peak[mode], "unit": "TFLOP/s",
                                                            "peak_source": f"bf16_tflops_sustained {pk_kind}"
                                                                           + (" x 2 (FP8 nominal ratio)" if mode == synth.C8E4M3 else "")},
                "error_kernel": {"max_rel": kmx, "l2_rel": kl2},
                "error_vs_fp64": {"max_rel": emx, "l2_rel": el2, "channels": chans},
                "tiling": q, "config": {"workload": f"config-3 shape: 256 antennas, 2048 beams, 8192 samples, T_int 64, "
                                                    f"{n_chan} of 4096 channels", "input_sigma": 16.0}}
        print(json.dumps(line), flush=True)


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
    ap.add_argument("--channels", type=int, default=0,
                    help="run only the first C channels (same per-channel shape; for profiling)")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)   # at least 3 untimed warm-up steps
    if args.impl == "reference":
        run_reference(args)
    elif args.sweep:
        run_sweep(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

"""Benchmark of the FX correlator hot path on one GB300 (or N replicas).

One step = F-engine (FFT + int8 re-packing + corner turn) + X-engine (INT8,
exact) + integration dump to FP64, over one integration of the INT8 workload:
256 antennas x 2 pol = 512 inputs, 1024 channels, 4096 spectra (4.29 GB of raw
complex int8 voltages per step, larger than L2, so no flush is needed).

Prints one JSON line (rank 0). ``--impl reference`` times the FP64 CPU oracle on
a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WORKLOADS = {
    # name: (n_ant, n_pol, n_chan, n_spectra)
    "B": (256, 2, 1024, 4096),
    "small": (64, 2, 256, 1024),
    # same per-channel shape as B with a quarter of the channels: for ncu captures
    "prof": (256, 2, 256, 4096),
    # B's FFT length and spectra with a quarter of the inputs: for F-engine captures
    "prof_f": (64, 2, 1024, 4096),
}
METRIC = "X-engine complex-MAC/s and % tensor peak; F-engine GB/s; vs FP32 baseline at tol"


def _traffic(kernel):
    """DRAM bytes per full-size launch of `kernel` from the committed ncu summary
    (profiles/traffic.json), or None if the kernel's source changed since."""
    import hashlib

    try:
        t = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))[kernel]
        h = hashlib.sha256(b"".join(open(os.path.join(ROOT, f), "rb").read() for f in t["files"])).hexdigest()[:16]
        return float(t["traffic_bytes"]) if h == t["source_sha256_16"] else None
    except (OSError, KeyError, ValueError):
        return None


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return dict(hbm=float(d["hbm_gbs"]), bf16=float(d["bf16_tflops"]),
                    bf16_sus=float(d.get("bf16_tflops_sustained", d["bf16_tflops"])), src="measured")
    return dict(hbm=6800.0, bf16=1900.0, bf16_sus=1700.0, src="fallback")


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
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
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# FP32 lanes of a GB300: 152 SMs x 128 FP32 units, 2 flop per fused multiply-add
FP32_FLOP_PER_CLK = 152 * 128 * 2


def fengine_fp32_rate(n_chan, n_fft, f_ms, clocks):
    """The F-engine's nominal FFT arithmetic (5 N log2 N flop per N-point FFT) as a
    rate and as a fraction of the FP32 peak at the SM clock sampled during the run
    (the maximum clock when no sample was taken)."""
    flop = 5.0 * n_chan * np.log2(n_chan) * n_fft
    mhz = (clocks or {}).get("sm_mhz") or (clocks or {}).get("sm_max_mhz") or 2070.0
    peak = FP32_FLOP_PER_CLK * mhz * 1e6 / 1e12
    ach = flop / (f_ms * 1e-3) / 1e12
    return {"flop_per_launch": flop, "achieved_tflops": ach, "peak_tflops": peak, "frac": ach / peak,
            "peak_note": f"152 SMs x 128 FP32 lanes x 2 flop at {mhz:.0f} MHz"}


def job_time_and_rate(ms_local: float, units_per_rank: float, steps: int, dist=None):
    """Whole-job timing for N replicas: the step time is the slowest rank's (max over
    ranks of the time each spent on its own `steps` steps), and the job's throughput
    is the units all ranks processed divided by it (weak scaling: every rank
    correlates its own data; no data-path collective). Returns (ms_per_step, rate)."""
    ws = 1
    if dist is not None and dist.is_initialized():
        import torch

        ws = dist.get_world_size()
        dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
        t = torch.tensor([ms_local], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_local = float(t.item())
    ms_step = ms_local / steps
    return ms_step, ws * units_per_rank / (ms_step * 1e-3)


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def cpu_oracle_sample(n_ant, n_pol, N, K, seed=0, n_chan_sample=2, spectra_sample=None, volt=None):
    """Time the FP64 oracle on a bounded sample of the workload: the direct DFT of
    `n_chan_sample` channels for every input over `spectra_sample` spectra, their
    int8 re-packing, and the triple-loop CMAC of those channels. `volt` (the raw
    int8 voltages, [n_in, K * N, 2]) is generated if not given. Returns
    (cMAC/s, seconds, cores, description)."""
    import oracle
    import synth

    Ks = K if spectra_sample is None else spectra_sample
    if volt is None:
        volt = synth.volt_int8(n_ant, n_pol, N, Ks, seed=seed)
    v = volt[:, : Ks * N]
    n_in = n_ant * n_pol
    bins = (np.arange(n_chan_sample) * (N // n_chan_sample) + 3 + seed) % N
    scale = np.full(N, 1.0 / np.sqrt(N), np.float32)
    oracle.build()
    t0 = time.perf_counter()
    S = oracle.channelise(v, N, bins)
    q, _ = oracle.requant(S, scale[bins])
    oracle.cmac(q)
    dt = time.perf_counter() - t0
    cmacs = n_chan_sample * (n_in * (n_in + 1) // 2) * Ks
    cores = len(os.sched_getaffinity(0))
    desc = (f"oracle direct DFT + requant + triple-loop CMAC of {n_chan_sample} of {N} channels, all {n_in} "
            f"inputs, {Ks} of {K} spectra (OpenMP over frames / channels)")
    return cmacs / dt, dt, cores, desc


def run_reference(args):
    """The oracle as it stands, on the host cores, one bounded sample per step."""
    import synth

    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    n_ant, n_pol, N, K = WORKLOADS[args.workload]
    volt = synth.volt_int8(n_ant, n_pol, N, K, seed=0)
    rates, secs = [], []
    for s in range(args.warmup + args.steps):
        # one step: 8 channels (all inputs and spectra), a few seconds of host work
        r, dt, cores, desc = cpu_oracle_sample(n_ant, n_pol, N, K, seed=s, n_chan_sample=8, volt=volt)
        if s >= args.warmup:
            rates.append(r)
            secs.append(dt)
    v = float(np.mean(rates))
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "cMAC/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(secs)), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": _workload_name(args.workload)},
        "cpu_baseline": {"value": v, "unit": "cMAC/s", "cores": cores, "kind": "oracle", "sample": desc},
        "e2e": {"value": v, "unit": "cMAC/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def _workload_name(w):
    n_ant, n_pol, N, K = WORKLOADS[w]
    return (f"INT8 FX: {n_ant} antennas x {n_pol} pol = {n_ant * n_pol} inputs, {N}-point FFT / {N} channels, "
            f"{K} spectra per integration, complex int8 voltages sigma=16 + delayed point source")


def run_ours(args):
    import torch

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    from paper_1305_5639_gb300 import build as pbuild

    pbuild.build()
    from paper_1305_5639_gb300 import api
    import synth

    n_ant, n_pol, N, K = WORKLOADS[args.workload]
    n_in = n_ant * n_pol
    B = n_in * (n_in + 1) // 2
    cmac_step = N * B * K

    volt_h = synth.volt_int8(n_ant, n_pol, N, K, seed=rank)
    volt_pin = torch.from_numpy(volt_h).pin_memory()
    volt = volt_pin.to(dev, non_blocking=False)
    planar = args.layout == "planar"
    fused = planar and args.fused_dump
    corr = api.Correlator(n_ant, n_pol, N, K, precision="int8", xengine=args.xengine, planar=planar,
                          fused_dump=fused)
    chan = corr.chan_buffer()
    if args.pfb > 0:
        # polyphase filter bank: a Hann-windowed sinc of args.pfb taps
        P = args.pfb
        x = (np.arange(P * N) - P * N / 2 + 0.5) / N
        corr.set_pfb((np.sinc(x) * np.hanning(P * N)).reshape(P, N).astype(np.float32))
    if args.delays:
        # delay compensation: each antenna's integer source delay plus a seeded fractional part
        dly = np.repeat(synth.delays_int8(n_ant, seed=rank), n_pol).astype(np.float64)
        dly += np.random.default_rng(rank).uniform(-0.5, 0.5, dly.size)
        corr.set_delays(dly.astype(np.float32))
    # requantisation scale from a calibration pass: 16 / per-component RMS of each channel
    power = corr.fengine_power(volt)
    scale = (16.0 / torch.sqrt(power)).contiguous()
    stream = torch.cuda.current_stream()

    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731

    def step(evs=None):
        if evs:
            evs[0].record(stream)
        corr.fengine(volt, scale, chan)
        if evs:
            evs[1].record(stream)
        corr.xengine(chan)
        if evs:
            evs[2].record(stream)
        corr.dump(copy=False)
        if evs:
            evs[3].record(stream)

    for _ in range(args.warmup):
        step()
    corr.check_status()
    torch.cuda.synchronize()

    evs = [[ev() for _ in range(4)] for _ in range(args.steps)]
    clk = ClockSampler(dev.index)
    clk.start()
    time.sleep(0.3)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    t0 = ev()
    t1 = ev()
    t0.record(stream)
    for s in range(args.steps):
        step(evs[s])
    t1.record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    clocks = clk.stop()
    corr.check_status()
    ms = t0.elapsed_time(t1)
    f_ms = float(np.mean([e[0].elapsed_time(e[1]) for e in evs]))
    x_ms = float(np.mean([e[1].elapsed_time(e[2]) for e in evs]))
    d_ms = float(np.mean([e[2].elapsed_time(e[3]) for e in evs]))
    ms_step, value = job_time_and_rate(ms, cmac_step, args.steps, torch.distributed if ws > 1 else None)

    # ---- end to end through the C ABI with host buffers: pinned raw voltages in, FP64
    # visibilities out, every step (corr_fx_host pipelines the copies with the engines)
    vis_pin = torch.empty((N, B), dtype=torch.complex128).pin_memory()
    e2e_steps = max(1, min(args.steps, 5))
    if planar:
        e2e_step = lambda: corr.fx_host(volt_pin, scale, vis_pin)  # noqa: E731
    else:
        vis_dev = torch.empty((N, B), dtype=torch.complex128, device=dev)

        def e2e_step():
            volt.copy_(volt_pin, non_blocking=True)
            corr.fengine(volt, scale, chan)
            corr.xengine(chan)
            corr.dump(vis_dev)
            vis_pin.copy_(vis_dev, non_blocking=True)

    e2e_step()
    torch.cuda.synchronize()
    # five timed blocks, median reported (the minimum and every block beside it): the
    # host link of a shared machine varies from block to block
    e2e_blocks = []
    for _ in range(5):
        a, b = ev(), ev()
        a.record(stream)
        for _ in range(e2e_steps):
            e2e_step()
        b.record(stream)
        torch.cuda.synchronize()
        e2e_blocks.append(a.elapsed_time(b) / e2e_steps)
    e2e_ms = float(np.median(e2e_blocks))
    corr.check_status()
    corr.reset()

    # ---- short-time visibilities (transient hook): the X-engine with 512-spectrum blocks
    short_time = None
    if args.short_time and planar:
        blk = 512
        stbuf = corr.set_short_time(blk)
        corr.fengine(volt, scale, chan)
        corr.xengine(chan)
        corr.dump(copy=False)
        torch.cuda.synchronize()
        a, b = ev(), ev()
        a.record(stream)
        for _ in range(3):
            corr.xengine(chan)
            corr.dump(copy=False)
        b.record(stream)
        torch.cuda.synchronize()
        corr.check_status()
        corr.set_short_time(out=False)
        s_ms = a.elapsed_time(b) / 3
        short_time = {"block_spectra": blk, "xengine_plus_dump_ms": s_ms,
                      "extra_bytes_per_call": float(stbuf.numel() * 4), "cmac_per_s": cmac_step / (s_ms * 1e-3)}
        del stbuf

    # ---- cross-only rectangle between the two halves of the inputs (space-division block)
    cross = None
    if args.cross and planar:
        h2 = n_in // 2
        rect = torch.empty((N, h2, n_in - h2, 2), dtype=torch.int32, device=dev)
        corr.fengine(volt, scale, chan)
        for _ in range(2):
            corr.xengine_cross(chan, 0, h2, h2, n_in - h2, out=rect)
        torch.cuda.synchronize()
        a, b = ev(), ev()
        a.record(stream)
        for _ in range(3):
            corr.xengine_cross(chan, 0, h2, h2, n_in - h2, out=rect)
        b.record(stream)
        torch.cuda.synchronize()
        corr.check_status()
        r_ms = a.elapsed_time(b) / 3
        r_cmac = float(N) * h2 * (n_in - h2) * K
        pk = _peaks()
        cross = {"inputs": f"[0, {h2}) x [{h2}, {n_in})", "ms": r_ms, "cmac_per_s": r_cmac / (r_ms * 1e-3),
                 "tensor_frac": 8.0 * r_cmac / (r_ms * 1e-3) / 1e12 / pk["bf16_sus"]}
        del rect

    # ---- CUDA-core comparator at the same accuracy (exact dp4a INT8 X-engine), same data
    cc_ms = None
    if args.comparator:
        cc = api.Correlator(n_ant, n_pol, N, K, precision="int8", xengine="cudacore")
        chan8 = cc.chan_buffer()
        cc.fengine(volt, scale, chan8)
        cc.xengine(chan8)
        torch.cuda.synchronize()
        a, b = ev(), ev()
        a.record(stream)
        cc.xengine(chan8)
        b.record(stream)
        torch.cuda.synchronize()
        cc_ms = a.elapsed_time(b)
        cc.close()

    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return 0

    peaks = _peaks()
    x_flops = 8.0 * cmac_step
    # read complex int8 voltages + write the channelised data (2 B/complex int8, 4 B planar FP16)
    f_bytes = float(n_in * N * K * 2 + chan.numel() * chan.element_size())
    tensor = corr_uses_tc(args.xengine)
    full_size = args.workload == "B"
    x_ach = x_flops / (x_ms * 1e-3) / 1e12
    f_ach = f_bytes / (f_ms * 1e-3) / 1e9
    if tensor:
        roof_x = {"bound": "tensor", "achieved": x_ach, "peak": peaks["bf16_sus"], "unit": "TFLOP/s",
                  "frac": x_ach / peaks["bf16_sus"],
                  "traffic": _traffic("k_xeng_tma") if (full_size and planar) else None,
                  "kernel": "k_xeng_tma (X-engine INT8-exact, tcgen05 kind::f16)" if planar
                  else "k_xeng_tc (X-engine INT8-exact, tcgen05 kind::f16)",
                  "peak_note": f"{peaks['src']} sustained bf16 dense (fp16 runs at the same rate)",
                  "algorithmic": f"{x_flops:.4g} FLOP per launch (8 per complex MAC over packed baselines)"}
    else:
        roof_x = {"bound": "alu", "achieved": x_ach, "peak": None, "unit": "TOP/s", "frac": None,
                  "traffic": None, "kernel": "k_xeng_i8 (CUDA-core dp4a)"}
    roof_f = {"bound": "hbm", "achieved": f_ach, "peak": peaks["hbm"], "unit": "GB/s", "frac": f_ach / peaks["hbm"],
              "traffic": _traffic("k_fengine") if (full_size and planar) else None,
              "kernel": "k_fengine (FFT + int8 re-packing + corner turn)",
              "peak_note": f"{peaks['src']} HBM copy bandwidth",
              "algorithmic": f"{f_bytes:.4g} bytes per launch (read raw int8, write channelised data once)"}
    d_bytes = float(N * B * (8 + 32))  # read INT32 pairs, read and write FP64 pairs
    roof_d = None
    if d_ms:
        d_ach = d_bytes / (d_ms * 1e-3) / 1e9
        roof_d = {"bound": "hbm", "achieved": d_ach, "peak": peaks["hbm"], "unit": "GB/s", "frac": d_ach / peaks["hbm"],
                  "traffic": _traffic("k_dump") if full_size else None,
                  "kernel": "k_dump (INT32 accumulator into the FP64 long integration)",
                  "peak_note": f"{peaks['src']} HBM copy bandwidth",
                  "algorithmic": f"{d_bytes:.4g} bytes per launch (40 per visibility)"}
    roof = roof_f if f_ms >= x_ms else roof_x
    cpu = None
    if ws == 1 and not args.no_cpu:
        # about 10 s of host work on 16 cores (24 of the 1024 channels, all inputs and spectra)
        r, dt, cores, desc = cpu_oracle_sample(n_ant, n_pol, N, K, n_chan_sample=24, volt=volt_h)
        cpu = {"value": r, "unit": "cMAC/s", "cores": cores, "kind": "oracle", "sample": desc, "seconds": dt}
    # per step: F-engine, X-engine (+ dump kernel unless fused); the calibration power pass is outside
    launches = 2 if fused else 3
    line = {
        "metric": METRIC, "value": value, "unit": "cMAC/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int8", "data": "synthetic",
        "config": {"workload": _workload_name(args.workload), "l2": "inputs larger than L2 (4.29 GB per step)",
                   "layout": args.layout, "dump": "fused into the X-engine epilogue" if fused else "separate kernel",
                   "delay_compensation": bool(args.delays),
                   "pfb_taps": args.pfb,
                   "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"},
        "stages_ms": {"fengine": f_ms, "xengine": x_ms, "dump": d_ms},
        "xengine_cmac_per_s": cmac_step / (x_ms * 1e-3),
        "fengine_gbs": f_bytes / (f_ms * 1e-3) / 1e9,
        "fengine_hbm_frac": f_bytes / (f_ms * 1e-3) / 1e9 / peaks["hbm"],
        "fengine_fp32": fengine_fp32_rate(N, n_in * K, f_ms, clocks),
        "dump_gbs": (N * B * (8 + 32)) / (d_ms * 1e-3) / 1e9,
        "cudacore_comparator": None if cc_ms is None else {
            "xengine_ms": cc_ms, "cmac_per_s": cmac_step / (cc_ms * 1e-3), "speedup_tensor_vs_cudacore": cc_ms / x_ms,
            "accuracy": "both exact (bit-identical INT32)"},
        "cross_only_xengine": cross,
        "short_time_xengine": short_time,
        "roofline": roof,
        "roofline_xengine": roof_x,
        "roofline_fengine": roof_f,
        "roofline_dump": roof_d,
        "cpu_baseline": cpu,
        "e2e": {"value": ws * cmac_step / (e2e_ms * 1e-3), "unit": "cMAC/s",
                "h2d_bytes_per_step": int(volt.numel()), "d2h_bytes_per_step": int(vis_pin.numel() * 16),
                "ms_per_step": e2e_ms, "ms_per_step_min": float(min(e2e_blocks)), "ms_per_step_blocks": e2e_blocks,
                "path": "corr_fx_host (copies pipelined with the engines)" if planar else "copies then kernels"},
        "gpu_launches": launches * args.steps,
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    corr.close()
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_short_time_only(args):
    """Profiling mode: only the short-time INT8 X-engine (512-spectrum blocks) on the
    chosen INT8 workload, after one F-engine pass; `warmup` untimed calls (each followed
    by a dump), then `steps` timed calls. Every X-engine launch of the process is a
    short-time one, so a profiler can select them by kernel name and launch count."""
    import torch
    from paper_1305_5639_gb300 import api

    n_ant, n_pol, N, K = WORKLOADS[args.workload]
    dev = torch.device("cuda", 0)
    corr = api.Correlator(n_ant, n_pol, N, K, precision="int8", planar=True)
    g = torch.Generator(device=dev).manual_seed(0)
    volt = torch.randint(-127, 128, (n_ant * n_pol, K * N, 2), dtype=torch.int8, device=dev, generator=g)
    chan = corr.chan_buffer()
    corr.fengine(volt, torch.full((N,), 1.0 / np.sqrt(N), device=dev), chan)
    del volt
    st = corr.set_short_time(512)
    for _ in range(args.warmup):
        corr.xengine(chan)
        corr.dump(copy=False)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(args.steps):
        corr.xengine(chan)
        corr.dump(copy=False)
    b.record()
    torch.cuda.synchronize()
    corr.check_status()
    ms = a.elapsed_time(b) / args.steps
    cmac = float(N) * (n_ant * n_pol) * (n_ant * n_pol + 1) / 2 * K
    print(json.dumps({"metric": "short-time X-engine + dump complex-MAC/s", "value": cmac / (ms * 1e-3),
                      "unit": "cMAC/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                      "higher_is_better": True, "dtype": "int8", "data": "synthetic",
                      "config": {"workload": f"INT8 short-time X-engine: {n_ant * n_pol} inputs, {N} channels, "
                                             f"{K} spectra, uniform random int8 voltages through the F-engine",
                                 "block_spectra": 512,
                                 "block_bytes_per_call": int(st.numel() * 4)}}), flush=True)
    corr.close()
    return 0


def run_batched(args):
    """Batched workload: 64 sub-arrays (antennas log-uniform 32-2048, channels from
    {256, 1024, 4096}, 512-4096 spectra, complex int8 sigma=16 as planar FP16
    codes), each on a window of --window channels (the full set, ~490 GB, does not
    fit one GPU). One tuned, graph-replayed persistent launch against 64 sequential
    plain launches of the same data."""
    import tempfile

    import torch

    import synth
    from paper_1305_5639_gb300 import build as pbuild

    pbuild.build()
    from paper_1305_5639_gb300 import api

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    subs = synth.subarrays(seed=0)
    W = args.window
    gen = torch.Generator(device=dev).manual_seed(0)
    planes = []
    for d in subs:
        z = torch.randn((W, 2, d["n_in"], d["n_spectra"]), generator=gen, device=dev) * 16.0
        planes.append(torch.clamp(torch.round(z), -127, 127).to(torch.float16).contiguous())
    cmac = float(sum(W * d["n_in"] * (d["n_in"] + 1) // 2 * d["n_spectra"] for d in subs))
    stream = torch.cuda.current_stream()
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731

    b = api.Batch(planes)
    cache = os.path.join(tempfile.gettempdir(), "corr_batch_tune.json")
    b.tune(cache)
    seq = [api.Correlator(d["n_in"], 1, W, d["n_spectra"], precision="int8", planar=True) for d in subs]

    def run_seq():
        for c, p in zip(seq, planes):
            c.xengine(p)
            c.dump(copy=False)

    for _ in range(args.warmup):
        b.run()
        run_seq()
    b.check_status()
    torch.cuda.synchronize()
    clk = ClockSampler(dev.index)
    clk.start()
    time.sleep(0.3)
    a0, a1 = ev(), ev()
    a0.record(stream)
    for _ in range(args.steps):
        b.run()
    a1.record(stream)
    torch.cuda.synchronize()
    clocks = clk.stop()
    t_batch = a0.elapsed_time(a1) / args.steps
    a0.record(stream)
    for _ in range(args.steps):
        run_seq()
    a1.record(stream)
    torch.cuda.synchronize()
    t_seq = a0.elapsed_time(a1) / args.steps
    b.check_status()
    peaks = _peaks()
    ach = 8.0 * cmac / (t_batch * 1e-3) / 1e12
    line = {
        "metric": METRIC, "value": cmac / (t_batch * 1e-3), "unit": "cMAC/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_batch, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int8", "data": "synthetic",
        "config": {"workload": f"batched: 64 sub-arrays (seed-0 shapes), {W}-channel window each, complex int8 "
                               f"sigma=16 as planar FP16 codes, one tuned graph-replayed persistent launch",
                   "l2": f"inputs larger than L2 ({sum(p.numel() * 2 for p in planes) / 1e9:.2f} GB per step)"},
        "sequential_64_launches_ms": t_seq, "speedup_vs_sequential": t_seq / t_batch,
        "channels_per_tile": [b.channels_per_tile(k) for k in range(len(subs))],
        "roofline": {"bound": "tensor", "achieved": ach, "peak": peaks["bf16_sus"], "unit": "TFLOP/s",
                     "frac": ach / peaks["bf16_sus"], "traffic": None, "kernel": "k_xeng_tma (batched)"},
        "gpu_launches": args.steps, "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    b.close()
    for c in seq:
        c.close()
    return 0


def run_calibration(args):
    """Calibration workload: 512 inputs, 1024 channels, 1024 spectra, per-input
    complex gains; one gained forward X-engine and one adjoint (dL/dX and dL/dg)
    per step. The headline runs both on tcgen05 tensor cores with the FP16 hi/lo
    split; the FP32 CUDA-core forward and adjoint are timed beside it."""
    import torch

    import synth
    from paper_1305_5639_gb300 import build as pbuild

    pbuild.build()
    from paper_1305_5639_gb300 import api

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    n_in, N, K = 512, 1024, 1024
    B = n_in * (n_in + 1) // 2
    gen = torch.Generator(device=dev).manual_seed(0)
    X = torch.complex(torch.randn((N, n_in, K), generator=gen, device=dev),
                      torch.randn((N, n_in, K), generator=gen, device=dev)).contiguous()
    g = torch.from_numpy(synth.gains(n_in, seed=0)).to(dev)
    G = torch.complex(torch.randn((N, B), generator=gen, device=dev),
                      torch.randn((N, B), generator=gen, device=dev)).contiguous() * 1e-6
    gx = torch.empty_like(X)
    gg = torch.empty(n_in, dtype=torch.complex64, device=dev)
    stream = torch.cuda.current_stream()
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731

    def measure(precision):
        c = api.Correlator(n_in, 1, N, K, precision=precision)

        def fwd():
            c.xengine(X, g)
            c.dump(copy=False)

        def bwd():
            api.corr_backward(c.h, G, X, g, gx, gg)

        for _ in range(args.warmup):
            fwd()
            bwd()
        torch.cuda.synchronize()
        res = {}
        for name, fn in (("forward", fwd), ("backward", bwd)):
            a, b = ev(), ev()
            a.record(stream)
            for _ in range(args.steps):
                fn()
            b.record(stream)
            torch.cuda.synchronize()
            res[name] = a.elapsed_time(b) / args.steps
        c.check_status()
        c.close()
        return res

    tc = measure("fp16_hilo")
    cc = measure("fp32") if args.comparator else None
    cm_f, cm_b = N * B * K, N * n_in * n_in * K
    ms = tc["forward"] + tc["backward"]
    # launches per step: forward planar split + X-engine + dump; adjoint: 4 per block of
    # channels (exponents, A planes, conj(X)^T planes, GEMM) + 2 for the dL/dg reduction
    cb = max(1, min(N, (1 << 30) // (8 * n_in * n_in + 8 * K * n_in)))
    launches = 3 + 4 * ((N + cb - 1) // cb) + 2
    line = {
        "metric": METRIC, "value": (cm_f + cm_b) / (ms * 1e-3), "unit": "cMAC/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f16 hi/lo (f32 accumulate)",
        "data": "synthetic",
        "config": {"workload": "calibration: 512 inputs, 1024 channels, 1024 spectra, complex64, per-input gains; "
                               "gained X-engine + adjoint (dL/dX, dL/dg)",
                   "l2": "inputs larger than L2 (4.29 GB)"},
        "forward_ms": tc["forward"], "forward_cmac_per_s": cm_f / (tc["forward"] * 1e-3),
        "backward_ms": tc["backward"], "backward_cmac_per_s": cm_b / (tc["backward"] * 1e-3),
        "cudacore_fp32": None if cc is None else {
            "forward_ms": cc["forward"], "backward_ms": cc["backward"],
            "speedup_step": (cc["forward"] + cc["backward"]) / ms},
        "gpu_launches": launches * args.steps,
    }
    print(json.dumps(line), flush=True)
    return 0


def run_fp16(args):
    """FP16 workload: 1024 antennas x 2 pol = 2048 inputs, 2048 spectra per integration,
    8 integrations dumped to FP64, on a window of --window channels of the 4096 (the
    per-channel work is identical; the full set would hold 137 GB of complex64 input).
    One step = 8 integrations (X-engine + dump) of the window. The headline is the hi/lo
    FP16 X-engine (FP32-class accuracy); plain FP16 and the FP32 CUDA-core X-engine are
    timed on the same data."""
    import torch

    from paper_1305_5639_gb300 import build as pbuild

    pbuild.build()
    from paper_1305_5639_gb300 import api

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    n_ant, n_pol, K, n_int = 1024, 2, 2048, 8
    n_in = n_ant * n_pol
    W = args.window
    B = n_in * (n_in + 1) // 2
    gen = torch.Generator(device=dev).manual_seed(0)
    X = torch.complex(torch.randn((W, n_in, K), generator=gen, device=dev),
                      torch.randn((W, n_in, K), generator=gen, device=dev)).contiguous()
    stream = torch.cuda.current_stream()
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731

    def measure(precision, steps, warmup):
        # separate dump kernel: measured faster than the dump fused into the FP16 epilogues
        # (40.0 / 43.4 ms vs 25.6 / 13.5 ms per step for hi/lo / plain), whose FP64 adds
        # then stall the tensor pipe on GB300's reduced FP64 path
        c = api.Correlator(n_ant, n_pol, W, K, precision=precision)

        def step():
            for _ in range(n_int):
                c.xengine(X)
                c.dump(copy=False)

        for _ in range(warmup):
            step()
        torch.cuda.synchronize()
        a, b = ev(), ev()
        a.record(stream)
        for _ in range(steps):
            step()
        b.record(stream)
        torch.cuda.synchronize()
        c.check_status()
        c.close()
        return a.elapsed_time(b) / steps

    clk = ClockSampler(0)
    clk.start()
    hl = measure("fp16_hilo", args.steps, args.warmup)
    clocks = clk.stop()
    pl = measure("fp16", args.steps, args.warmup)
    cc = measure("fp32", 1, 1) if args.comparator else None
    cm = W * B * K * n_int
    peaks = _peaks()
    ach = 8.0 * cm / (hl * 1e-3) / 1e12
    line = {
        "metric": METRIC, "value": cm / (hl * 1e-3), "unit": "cMAC/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": hl, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f16 hi/lo (f32 accumulate)", "data": "synthetic",
        "config": {"workload": f"FP16: 1024 antennas x 2 pol = 2048 inputs, 2048 spectra per integration, "
                               f"8 integrations dumped to FP64, window of {W} of 4096 channels, complex64 N(0,1)",
                   "l2": f"inputs larger than L2 ({X.numel() * 8 / 1e9:.2f} GB)"},
        "roofline": {"bound": "tensor", "achieved": ach, "peak": peaks["bf16_sus"], "unit": "TFLOP/s",
                     "frac": ach / peaks["bf16_sus"], "traffic": None,
                     "kernel": "k_to_planar + k_xeng_tma<FP16, 4 planes> + k_dump (hi/lo: 12 MMAs per 16 spectra, "
                               "3x the algorithmic products)",
                     "peak_note": f"{peaks['src']} sustained bf16 dense",
                     "algorithmic": "8 FLOP per complex MAC over packed baselines"},
        "fp16_plain": {"ms_per_step": pl, "cmac_per_s": cm / (pl * 1e-3),
                       "tensor_frac": 8.0 * cm / (pl * 1e-3) / 1e12 / peaks["bf16_sus"]},
        "cudacore_fp32": None if cc is None else {"ms_per_step": cc, "cmac_per_s": cm / (cc * 1e-3),
                                                 "hilo_speedup": cc / hl},
        "e2e": None,
        "gpu_launches": 3 * n_int * args.steps,
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    return 0


def corr_uses_tc(xengine: str) -> bool:
    return xengine in ("auto", "tcgen05")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="B", choices=sorted(WORKLOADS) + ["C", "D", "E"])
    ap.add_argument("--window", type=int, default=16,
                    help="batched workload: channels per sub-array; FP16 workload: channels of the 4096 (use 32)")
    ap.add_argument("--xengine", default="auto", choices=["auto", "cudacore", "tcgen05"])
    ap.add_argument("--layout", default="planar", choices=["planar", "int8"],
                    help="channelised layout between the engines: planar FP16 codes (TMA X-engine) or complex int8")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU-baseline leg")
    ap.add_argument("--short-time", action="store_true",
                    help="INT8 planar workloads: also time the X-engine writing 512-spectrum short-time visibilities")
    ap.add_argument("--only-short-time", action="store_true",
                    help="profiling mode: only the short-time INT8 X-engine (+ dump) on the chosen INT8 workload")
    ap.add_argument("--cross", action="store_true",
                    help="INT8 planar workloads: also time the cross-only rectangle between the two input halves")
    ap.add_argument("--pfb", type=int, default=0,
                    help="INT8 workloads: polyphase filter-bank front end with this many taps (0: plain FFT)")
    ap.add_argument("--delays", action="store_true",
                    help="INT8 workloads: delay compensation in the F-engine (per-input integer + fractional delays)")
    ap.add_argument("--fused-dump", action="store_true",
                    help="planar layout: the X-engine epilogue adds each integration into the FP64 buffer "
                         "directly instead of the separate dump kernel (measured equal on GB300)")
    ap.add_argument("--comparator", type=int, default=1, help="time the CUDA-core X-engine once")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.only_short_time:
        return run_short_time_only(args)
    if args.workload == "E":
        return run_batched(args)
    if args.workload == "D":
        return run_calibration(args)
    if args.workload == "C":
        return run_fp16(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())

"""Benchmark of the FX correlator hot path on one GB300 (or N replicas).

One step = F-engine (FFT + int8 re-packing + corner turn) + X-engine (INT8,
exact) + integration dump to FP64, over one integration of the INT8 workload:
256 antennas x 2 pol = 512 inputs, 1024 channels, 4096 spectra (4.29 GB of raw
complex int8 voltages per step, larger than L2, so no flush is needed). The
JSON line's headline is that workload; after its timed region the default run
adds compact sub-results for the other configurations (FP32 FX, FP16 plain and
hi/lo, calibration forward + adjoint, batched sub-arrays) under "configs", each
with its stage times, roofline fraction and accuracy (``--configs`` selects
them; ``--workload A|C|D|E`` runs one alone).

The ``small``, ``prof`` and ``prof_f`` workloads and ``--only-short-time`` are
smaller INT8 shapes and a single-kernel mode for profiler captures, which must
stay a few GB on the device; they are not bench lines.

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
    fused = args.fused_dump
    corr = api.Correlator(n_ant, n_pol, N, K, precision="int8", xengine=args.xengine, planar=planar,
                          fused_dump=fused, fengine=args.fengine)
    # the tensor-core F-engine runs for 1024 channels without delays or a filter bank
    f_tc = args.fengine == "auto" and N == 1024 and not args.pfb and not args.delays
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
    # count the library's kernel launches in the timed region (stage timing off: counts only)
    corr.set_stage_timing(False)
    corr.stage_times()

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
    # a dump deferred into the next X-engine launch is still pending after the last step:
    # complete it inside the timed region, so that every timed integration is dumped
    corr.flush()
    t1.record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    clocks = clk.stop()
    corr.check_status()
    launches = sum(n for _, n in corr.stage_times().values())
    ms = t0.elapsed_time(t1)
    f_ms = float(np.mean([e[0].elapsed_time(e[1]) for e in evs]))
    x_ms = float(np.mean([e[1].elapsed_time(e[2]) for e in evs]))
    d_ms = float(np.mean([e[2].elapsed_time(e[3]) for e in evs]))
    ms_step, value = job_time_and_rate(ms, cmac_step, args.steps, torch.distributed if ws > 1 else None)

    # ---- end to end through the C ABI with host buffers: pinned raw voltages in, each
    # integration's exact visibilities out (INT32 pairs; corr_fx_host_accum pipelines the
    # copies with the engines and keeps the FP64 long integration on the device)
    e2e_steps = max(1, min(args.steps, 5))
    accum_out = planar and not fused  # the fused dump keeps no INT32 accumulator
    if accum_out:
        out_pin = torch.empty((N, B, 2), dtype=torch.int32).pin_memory()
        e2e_step = lambda: corr.fx_host_accum(volt_pin, scale, out_pin)  # noqa: E731
    else:
        out_pin = torch.empty((N, B), dtype=torch.complex128).pin_memory()
    if planar and not accum_out:
        e2e_step = lambda: corr.fx_host(volt_pin, scale, out_pin)  # noqa: E731
    elif not planar:
        vis_dev = torch.empty((N, B), dtype=torch.complex128, device=dev)

        def e2e_step():
            volt.copy_(volt_pin, non_blocking=True)
            corr.fengine(volt, scale, chan)
            corr.xengine(chan)
            corr.dump(vis_dev)
            out_pin.copy_(vis_dev, non_blocking=True)

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
                 "tensor_frac": 8.0 * r_cmac / (r_ms * 1e-3) / 1e12 / pk["bf16"]}
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
        del chan8

    if rank != 0:
        corr.close()
        if ws > 1:
            torch.distributed.destroy_process_group()
        return 0

    peaks = _peaks()
    x_flops = 8.0 * cmac_step
    # algorithmic F-engine bytes (the survey's unit): read the complex int8 voltages and
    # write complex int8 spectra once, 2 B + 2 B per complex sample
    f_bytes = float(n_in * N * K * 4)
    # bytes the chosen exchange layout moves: the planar FP16 codes are 4 B per sample
    f_layout_bytes = float(n_in * N * K * 2 + chan.numel() * chan.element_size())
    full_size = args.workload == "B"
    x_ach = x_flops / (x_ms * 1e-3) / 1e12
    f_ach = f_bytes / (f_ms * 1e-3) / 1e9
    roof_x = {"bound": "tensor", "achieved": x_ach, "peak": peaks["bf16"], "unit": "TFLOP/s",
              "frac": x_ach / peaks["bf16"], "frac_of_sustained": x_ach / peaks["bf16_sus"],
              "traffic": _traffic("k_xeng_tma") if (full_size and planar) else None,
              "kernel": "k_xeng_tma (X-engine INT8-exact, tcgen05 kind::f16, wide form)",
              "peak_note": f"{peaks['src']} burst bf16 dense (fp16 runs at the same rate; the kernel is timed "
                           f"inside a region of well under a second)",
              "algorithmic": f"{x_flops:.4g} FLOP per launch (8 per complex MAC over packed baselines)"}
    if args.xengine == "cudacore":
        roof_x = {"bound": "alu", "achieved": x_ach, "peak": None, "unit": "TOP/s", "frac": None,
                  "traffic": None, "kernel": "k_xeng_i8 (CUDA-core dp4a)"}
    f_kernel = "k_fengine_tc" if f_tc else "k_fengine"
    f_traffic = _traffic(f_kernel) if (full_size and planar and not args.pfb and not args.delays) else None
    roof_f = {"bound": "hbm", "achieved": f_ach, "peak": peaks["hbm"], "unit": "GB/s", "frac": f_ach / peaks["hbm"],
              "traffic": f_traffic,
              "traffic_ratio": None if f_traffic is None else f_traffic / f_bytes,
              "layout_bytes": f_layout_bytes,
              "kernel": ("k_fengine_tc (32 x 32 FFT: both DFT stages as FP16 hi/lo GEMMs on tcgen05, int8 "
                         "re-packing, corner turn)" if f_tc else "k_fengine (FFT + int8 re-packing + corner turn)"),
              "peak_note": f"{peaks['src']} HBM copy bandwidth",
              "algorithmic": f"{f_bytes:.4g} bytes per launch (read 2 B + write 2 B per complex sample); the "
                             f"{args.layout} exchange layout moves {f_layout_bytes:.4g}"}
    d_bytes = float(N * B * (8 + 32))  # read INT32 pairs, read and write FP64 pairs
    deferred = d_ms < 0.05  # the dump ran inside the next X-engine launch (no kernel of its own)
    roof_d = None
    if not deferred:
        d_ach = d_bytes / (d_ms * 1e-3) / 1e9
        roof_d = {"bound": "hbm", "achieved": d_ach, "peak": peaks["hbm"], "unit": "GB/s", "frac": d_ach / peaks["hbm"],
                  "traffic": _traffic("k_dump") if full_size else None,
                  "kernel": "k_dump (INT32 accumulator into the FP64 long integration)",
                  "peak_note": f"{peaks['src']} HBM copy bandwidth",
                  "algorithmic": f"{d_bytes:.4g} bytes per launch (40 per visibility)"}
    roof = roof_f if f_ms >= x_ms else roof_x

    # ---- the other configurations (rank 0 at one GPU): free this workload's buffers first
    configs = None
    if ws == 1 and args.configs:
        corr.close()
        del chan, volt
        torch.cuda.empty_cache()
        mhz = (clocks or {}).get("sm_mhz") or 2070.0
        configs = {}
        runners = {"A": lambda: bench_A(10, 3, dev, peaks, mhz),
                   "C": lambda: bench_C(2, 1, dev, peaks, args.c_window),
                   "D": lambda: bench_D(10, 3, dev, peaks, bool(args.comparator), args.d_window),
                   "E": lambda: bench_E(10, 3, dev, peaks, args.e_window)}
        for name in args.configs:
            configs[name] = runners[name]()
            torch.cuda.empty_cache()
    cpu = None
    if ws == 1 and not args.no_cpu:
        # about 10 s of host work on 16 cores (24 of the 1024 channels, all inputs and spectra)
        r, dt, cores, desc = cpu_oracle_sample(n_ant, n_pol, N, K, n_chan_sample=24, volt=volt_h)
        cpu = {"value": r, "unit": "cMAC/s", "cores": cores, "kind": "oracle", "sample": desc, "seconds": dt}
    line = {
        "metric": METRIC, "value": value, "unit": "cMAC/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int8", "data": "synthetic",
        "config": {"workload": _workload_name(args.workload), "l2": "inputs larger than L2 (4.29 GB per step)",
                   "layout": args.layout,
                   "dump": "fused into the X-engine epilogue" if fused else (
                       "deferred: each integration's FP64 dump runs in idle warps of the next X-engine launch (the last "
                       "one by a flush inside the timed region)" if deferred else "separate kernel"),
                   "delay_compensation": bool(args.delays),
                   "pfb_taps": args.pfb,
                   "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"},
        "stages_ms": {"fengine": f_ms, "xengine": x_ms, "dump": d_ms},
        "xengine_cmac_per_s": cmac_step / (x_ms * 1e-3),
        "fengine_gbs": f_ach,
        "fengine_hbm_frac": f_ach / peaks["hbm"],
        "fengine_fp32": fengine_fp32_rate(N, n_in * K, f_ms, clocks),
        "dump_gbs": d_bytes / (d_ms * 1e-3) / 1e9 if not deferred else None,
        "cudacore_comparator": None if cc_ms is None else {
            "xengine_ms": cc_ms, "cmac_per_s": cmac_step / (cc_ms * 1e-3), "speedup_tensor_vs_cudacore": cc_ms / x_ms,
            "accuracy": "both exact (bit-identical INT32)"},
        "cross_only_xengine": cross,
        "short_time_xengine": short_time,
        "roofline": roof,
        "roofline_xengine": roof_x,
        "roofline_fengine": roof_f,
        "roofline_dump": roof_d,
        "configs": configs,
        "cpu_baseline": cpu,
        "e2e": {"value": ws * cmac_step / (e2e_ms * 1e-3), "unit": "cMAC/s",
                "h2d_bytes_per_step": int(volt_pin.numel()),
                "d2h_bytes_per_step": int(out_pin.numel() * out_pin.element_size()),
                "ms_per_step": e2e_ms, "ms_per_step_min": float(min(e2e_blocks)), "ms_per_step_blocks": e2e_blocks,
                "path": ("corr_fx_host_accum (copies pipelined with the engines; the integration's INT32 "
                         "visibilities out, the FP64 long integration kept on the device)" if accum_out
                         else "corr_fx_host (copies pipelined with the engines; FP64 long integration out)"
                         if planar else "copies then kernels")},
        "gpu_launches": launches,
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    if not (ws == 1 and args.configs):
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


# ----------------------------------------------------------------------------- the other configurations
# Compact sub-results for the FP32 FX, FP16, calibration and batched workloads, run
# after the INT8 workload's timed region (rank 0, one GPU) and reported beside it.
# Each gives its time, complex-MAC/s, roofline fraction of the dominant kernel,
# per-stage kernel times from the library's stage timing, and the accuracy against
# an FP64 reference computed on the GPU with torch (cuFFT / cuBLAS in complex128:
# a measurement beside the number; the parity proof is the test suite's oracle).


def _ev():
    import torch

    return torch.cuda.Event(enable_timing=True)


def _flush_l2(buf):
    """Overwrite a buffer larger than L2 (129 MB) so that the next step starts cold."""
    buf.zero_()


def _packed_from_full(Vfull):
    """[n_chan, n, n] -> packed lower triangle [n_chan, B] (b(i, j) = i (i + 1) / 2 + j)."""
    import torch

    n = Vfull.shape[-1]
    i, j = torch.tril_indices(n, n, device=Vfull.device)
    return Vfull[:, i, j]


def _norm_err(V, Vref, n_in):
    """max and rms of |V_ij - Vref_ij| / sqrt(|Vref_ii| |Vref_jj|) over packed pairs."""
    import torch

    idx = torch.arange(n_in, device=Vref.device)
    aut = Vref[:, idx * (idx + 1) // 2 + idx].abs()
    i, j = torch.tril_indices(n_in, n_in, device=Vref.device)
    e = (V.to(torch.complex128) - Vref).abs() / torch.sqrt(aut[:, i] * aut[:, j])
    return float(e.max()), float(torch.sqrt((e ** 2).mean()))


def _stage_ms(times, steps):
    return {k: v[0] / steps for k, v in times.items() if v[1]}


def _stage_launches(times, steps):
    return {k: v[1] // steps for k, v in times.items() if v[1]}


def bench_A(steps, warmup, dev, peaks, clocks_mhz):
    """FP32 FX (16 antennas x 1 pol, 256-point FFT, 1024 spectra, complex64 N(0,1)
    plus a source delayed by d_i = i samples): F-engine FFT + FP32 CUDA-core X-engine
    + dump per step, L2 flushed before each step (the whole workload, 33.5 MB,
    would otherwise sit in L2)."""
    import torch

    import synth
    from paper_1305_5639_gb300 import api

    n_in, N, K = 16, 256, 1024
    B = n_in * (n_in + 1) // 2
    v = torch.from_numpy(synth.volt_fp32(n_in, N, K, seed=0)).to(dev)
    c = api.Correlator(n_in, 1, N, K, precision="fp32")
    chan = c.chan_buffer()
    flush = torch.empty(64 << 20, dtype=torch.float32, device=dev)  # 256 MB
    stream = torch.cuda.current_stream()

    def step():
        c.fengine(v, None, chan)
        c.xengine(chan)
        c.dump(copy=False)

    for _ in range(warmup):
        step()
    c.set_stage_timing(True)
    c.stage_times()
    tot = 0.0
    for _ in range(steps):
        _flush_l2(flush)
        a, b = _ev(), _ev()
        a.record(stream)
        step()
        b.record(stream)
        torch.cuda.synchronize()
        tot += a.elapsed_time(b)
    st = c.stage_times()
    ms = tot / steps
    # accuracy of one integration against FP64 on the GPU (cuFFT + complex128 products)
    c.reset()
    c.fengine(v, None, chan)
    c.xengine(chan)
    V = c.accum()
    S = torch.fft.fft(v.to(torch.complex128).reshape(n_in, K, N), dim=-1)  # [i, a, k]
    Vref = _packed_from_full(torch.einsum("iak,jak->kij", S, S.conj()))
    emax, erms = _norm_err(V, Vref, n_in)
    c.check_status()
    c.close()
    cm = N * B * K
    x_ms = st["xengine"][0] / steps
    fp32_peak = FP32_FLOP_PER_CLK * clocks_mhz * 1e6 / 1e12
    f_bytes = n_in * N * K * 16.0  # read and write 8 B per complex sample
    return {
        "workload": "FP32 FX: 16 antennas x 1 pol, 256-point FFT, 1024 spectra, complex64 N(0,1) + source delayed "
                    "d_i = i samples",
        "ms_per_step": ms, "cmac_per_s": cm / (ms * 1e-3),
        "stages_ms": _stage_ms(st, steps), "launches_per_step": _stage_launches(st, steps),
        "roofline": {"kernel": "k_xeng_f32_small (FP32 CUDA-core X-engine for few inputs: one CTA per channel, one thread per pair)", "bound": "alu",
                     "achieved": 8.0 * cm / (x_ms * 1e-3) / 1e12, "peak": fp32_peak, "unit": "TFLOP/s",
                     "frac": 8.0 * cm / (x_ms * 1e-3) / 1e12 / fp32_peak,
                     "peak_note": f"152 SMs x 128 FP32 lanes x 2 flop at {clocks_mhz:.0f} MHz"},
        "fengine_gbs": f_bytes / (st["fengine"][0] / steps * 1e-3) / 1e9,
        "note": "launch-bound size (a few microseconds per kernel); L2 flushed before each step",
        "err_vs_fp64": {"max": emax, "rms": erms, "bar": 1e-5,
                        "reference": "torch complex128 on the GPU: cuFFT of the raw voltages, then X X^H"},
    }


def bench_C(steps, warmup, dev, peaks, window, fused=False):
    """FP16 workload (1024 antennas x 2 pol = 2048 inputs, 2048 spectra per
    integration, 8 integrations dumped to FP64) on a window of `window` of the 4096
    channels (the per-channel work is the same; all channels would hold 137 GB of
    complex64 input). hi/lo and plain FP16 on the tensor cores, each step = 8
    integrations of the window; the FP32 CUDA-core X-engine once for comparison."""
    import torch

    from paper_1305_5639_gb300 import api

    n_ant, n_pol, K, n_int = 1024, 2, 2048, 8
    n_in = n_ant * n_pol
    W = window
    B = n_in * (n_in + 1) // 2
    gen = torch.Generator(device=dev).manual_seed(0)
    X = torch.complex(torch.randn((W, n_in, K), generator=gen, device=dev),
                      torch.randn((W, n_in, K), generator=gen, device=dev)).contiguous()
    stream = torch.cuda.current_stream()
    res = {}
    for prec in ("fp16_hilo", "fp16"):
        # plain FP16 integrates straight into the FP64 buffer from the X-engine's epilogue
        # (measured faster than the separate dump there: 21.3 against 22.6 ms on 64 channels);
        # hi/lo keeps its dump in the next X-engine launch's idle warps (37.5 against 35.5 ms)
        c = api.Correlator(n_ant, n_pol, W, K, precision=prec, fused_dump=fused or prec == "fp16")

        def step():
            for _ in range(n_int):
                c.xengine(X)
                c.dump(copy=False)

        for _ in range(warmup):
            step()
        torch.cuda.synchronize()
        c.set_stage_timing(True)
        c.stage_times()
        a, b = _ev(), _ev()
        a.record(stream)
        for _ in range(steps):
            step()
        b.record(stream)
        torch.cuda.synchronize()
        st = c.stage_times()
        c.check_status()
        c.close()
        res[prec] = (a.elapsed_time(b) / steps, st)
    # accuracy on 2 channels, one integration: each path against FP64 (cuBLAS complex128)
    Xe = X[:2].contiguous()
    Xd = Xe.to(torch.complex128)
    Vref = _packed_from_full(torch.matmul(Xd, Xd.conj().transpose(1, 2)))
    del Xd
    errs = {}
    for prec, xe in (("fp16_hilo", "auto"), ("fp16", "auto"), ("fp32", "cudacore")):
        c = api.Correlator(n_ant, n_pol, 2, K, precision=prec, xengine=xe)
        c.xengine(Xe)
        errs[prec] = _norm_err(c.accum(), Vref, n_in)
        if prec == "fp32":
            torch.cuda.synchronize()
            a, b = _ev(), _ev()
            a.record(stream)
            c.xengine(Xe)
            b.record(stream)
            torch.cuda.synchronize()
            cc_ms_per_chan_int = a.elapsed_time(b) / 2
        c.close()
    del X, Xe
    cm = W * B * K * n_int
    out = {"workload": f"FP16: 2048 inputs, 2048 spectra x 8 integrations dumped to FP64, window of {W} of 4096 "
                       f"channels, complex64 N(0,1)", "window_channels": W}
    for prec, (ms, st) in res.items():
        x_ms = st["xengine"][0] / steps
        ach = 8.0 * cm / (x_ms * 1e-3) / 1e12
        executed = 3 if prec == "fp16_hilo" else 1
        out[prec] = {
            "ms_per_step": ms, "cmac_per_s": cm / (ms * 1e-3),
            "stages_ms": _stage_ms(st, steps), "launches_per_step": _stage_launches(st, steps),
            "xengine_cmac_per_s": cm / (x_ms * 1e-3),
            "roofline_xengine": {"kernel": f"k_xeng_tma<FP16, {4 if prec == 'fp16_hilo' else 2} planes>",
                                 "bound": "tensor", "achieved": ach, "peak": peaks["bf16"], "unit": "TFLOP/s",
                                 "frac": ach / peaks["bf16"], "frac_executed": executed * ach / peaks["bf16"],
                                 "peak_note": f"{peaks['src']} burst bf16 dense (fp16 runs at the same rate)"},
            "err_vs_fp64": {"max": errs[prec][0], "rms": errs[prec][1],
                            "bar": 5e-5 if prec == "fp16_hilo" else 2e-3},
            "dump": ("each integration added to the FP64 buffer in the next X-engine launch's idle warps (inside "
                     "the X-engine time)" if prec == "fp16_hilo" and not fused else
                     "fused into the X-engine epilogue (the X-engine time includes the FP64 update)"),
        }
    cc_ms = cc_ms_per_chan_int * W * n_int
    out["fp32_cudacore"] = {"ms_per_step_extrapolated": cc_ms, "cmac_per_s": cm / (cc_ms * 1e-3),
                            "timed": "one integration of 2 channels, scaled to the window's 8 integrations",
                            "err_vs_fp64": {"max": errs["fp32"][0], "rms": errs["fp32"][1], "bar": 1e-5},
                            "hilo_speedup": cc_ms / res["fp16_hilo"][0]}
    out["err_reference"] = "torch complex128 X X^H on the GPU (cuBLAS), 2 channels, one integration"
    return out


def bench_D(steps, warmup, dev, peaks, comparator=True, window=1024):
    """Calibration workload: 512 inputs, 1024 channels, 1024 spectra, complex64,
    per-input complex gains; one gained forward X-engine (hi/lo, tensor cores) and
    one adjoint (dL/dX, dL/dg on tensor cores) per step. The FP32 CUDA-core forward
    and adjoint run once beside it; the gradients are compared with each other.
    `window` < 1024 runs that many of the channels (profiler captures)."""
    import torch

    import synth
    from paper_1305_5639_gb300 import api

    n_in, N, K = 512, window, 1024
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

    def measure(precision, n_steps, n_warm):
        c = api.Correlator(n_in, 1, N, K, precision=precision)

        def fwd():
            c.xengine(X, g)
            c.dump(copy=False)

        def bwd():
            api.corr_backward(c.h, G, X, g, gx, gg)

        for _ in range(n_warm):
            fwd()
            bwd()
        torch.cuda.synchronize()
        c.set_stage_timing(True)
        c.stage_times()
        r = {}
        for name, fn in (("forward", fwd), ("backward", bwd)):
            a, b = _ev(), _ev()
            a.record(stream)
            for _ in range(n_steps):
                fn()
            b.record(stream)
            torch.cuda.synchronize()
            r[name] = a.elapsed_time(b) / n_steps
        st = c.stage_times()
        c.check_status()
        c.close()
        return r, st, gx.clone(), gg.clone()

    tc, st, dX_tc, dg_tc = measure("fp16_hilo", steps, warmup)
    cm_f, cm_b = N * B * K, N * n_in * n_in * K
    ms = tc["forward"] + tc["backward"]
    gemm_ms = st["adj_gemm"][0] / steps
    ach = 8.0 * cm_b / (gemm_ms * 1e-3) / 1e12
    out = {
        "workload": f"calibration: 512 inputs, {N} of 1024 channels, 1024 spectra, complex64, per-input gains; "
                    "gained X-engine + adjoint (dL/dX, dL/dg)",
        "ms_per_step": ms, "cmac_per_s": (cm_f + cm_b) / (ms * 1e-3),
        "forward_ms": tc["forward"], "backward_ms": tc["backward"],
        "stages_ms": _stage_ms(st, steps), "launches_per_step": _stage_launches(st, steps),
        "roofline_adjoint_gemm": {"kernel": "k_xeng_tma<kAdj> (dX GEMM, hi/lo: 3 products)", "bound": "tensor",
                                  "achieved": ach, "peak": peaks["bf16"], "unit": "TFLOP/s",
                                  "frac": ach / peaks["bf16"], "frac_executed": 3 * ach / peaks["bf16"],
                                  "algorithmic": f"{8.0 * cm_b:.4g} FLOP per step (n_in^2 K complex MAC per "
                                                 f"channel, 8 FLOP each)"},
    }
    if comparator:
        cc, _, dX_cc, dg_cc = measure("fp32", 1, 1)
        rel = lambda a, b: float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))  # noqa: E731
        rms = torch.sqrt(torch.mean(dX_cc.abs() ** 2, dim=(1, 2)))
        elem = float(torch.max(torch.amax((dX_tc - dX_cc).abs(), dim=(1, 2)) / rms))
        out["fp32_cudacore"] = {"forward_ms": cc["forward"], "backward_ms": cc["backward"],
                                "speedup_step": (cc["forward"] + cc["backward"]) / ms}
        out["grad_vs_fp32"] = {"dX_rel_l2": rel(dX_tc, dX_cc), "dg_rel_l2": rel(dg_tc, dg_cc),
                               "dX_max_over_channel_rms": elem, "bar_rel_l2": 1e-4}
    del X, G, gx
    return out


def bench_E(steps, warmup, dev, peaks, window):
    """Batched workload: 64 sub-arrays (antennas log-uniform 32-2048, channels from
    {256, 1024, 4096}, 512-4096 spectra, complex int8 sigma=16 as planar FP16 codes),
    each on a window of `window` channels (the full set, ~490 GB, does not fit one
    GPU): one tuned, graph-replayed persistent launch against 64 sequential plain
    launches of the same data (their results compared bit for bit)."""
    import tempfile

    import torch

    import synth
    from paper_1305_5639_gb300 import api

    subs = synth.subarrays(seed=0)
    W = window
    gen = torch.Generator(device=dev).manual_seed(0)
    planes = []
    for d in subs:
        z = torch.randn((W, 2, d["n_in"], d["n_spectra"]), generator=gen, device=dev) * 16.0
        planes.append(torch.clamp(torch.round(z), -127, 127).to(torch.float16).contiguous())
    cmac = float(sum(W * d["n_in"] * (d["n_in"] + 1) // 2 * d["n_spectra"] for d in subs))
    stream = torch.cuda.current_stream()
    b = api.Batch(planes)
    b.tune(os.path.join(tempfile.gettempdir(), "corr_batch_tune.json"))
    seq = [api.Correlator(d["n_in"], 1, W, d["n_spectra"], precision="int8", planar=True) for d in subs]

    def run_seq():
        for c, p in zip(seq, planes):
            c.xengine(p)
            c.dump(copy=False)

    for _ in range(warmup):
        b.run()
        run_seq()
    b.check_status()
    torch.cuda.synchronize()
    a0, a1 = _ev(), _ev()
    a0.record(stream)
    for _ in range(steps):
        b.run()
    a1.record(stream)
    torch.cuda.synchronize()
    t_batch = a0.elapsed_time(a1) / steps
    a0.record(stream)
    for _ in range(steps):
        run_seq()
    a1.record(stream)
    torch.cuda.synchronize()
    t_seq = a0.elapsed_time(a1) / steps
    b.check_status()
    # the batch's INT32 outputs against the sequential launches' accumulators
    exact = True
    for c, p, v in zip(seq, planes, b.vis):
        c.reset()
        c.xengine(p)
        exact = exact and bool(torch.equal(c.accum(), v))
        c.close()
    cpt = [b.channels_per_tile(k) for k in range(len(subs))]
    b.close()
    ach = 8.0 * cmac / (t_batch * 1e-3) / 1e12
    return {
        "workload": f"batched: 64 sub-arrays (seed-0 shapes), {W}-channel window each, complex int8 sigma=16 as "
                    f"planar FP16 codes, one tuned graph-replayed persistent launch",
        "window_channels": W, "ms_per_step": t_batch, "cmac_per_s": cmac / (t_batch * 1e-3),
        "sequential_64_launches_ms": t_seq, "speedup_vs_sequential": t_seq / t_batch,
        "channels_per_tile": cpt, "bit_identical_to_sequential": exact,
        "roofline": {"kernel": "k_xeng_tma (batched, wide INT8)", "bound": "tensor", "achieved": ach,
                     "peak": peaks["bf16"], "unit": "TFLOP/s", "frac": ach / peaks["bf16"]},
        "launches_per_step": 1,
    }


def _standalone(args, name, fn):
    """One configuration alone: its sub-result as the JSON line's body."""
    import torch

    from paper_1305_5639_gb300 import build as pbuild

    pbuild.build()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    peaks = _peaks()
    clk = ClockSampler(0)
    clk.start()
    r = fn(dev, peaks)
    clocks = clk.stop()
    unit_ms = r.get("ms_per_step") or r.get("fp16_hilo", {}).get("ms_per_step")
    rate = r.get("cmac_per_s") or r.get("fp16_hilo", {}).get("cmac_per_s")
    line = {"metric": METRIC, "value": rate, "unit": "cMAC/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": unit_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {"A": "f32", "C": "f16 hi/lo (f32 accumulate)",
                                            "D": "f16 hi/lo (f32 accumulate)", "E": "int8"}[name],
            "data": "synthetic", "config": {"workload": r["workload"]}, "result": r, "clocks": clocks}
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
    ap.add_argument("--workload", default="B", choices=sorted(WORKLOADS) + ["A", "C", "D", "E"],
                    help="B (default): the INT8 workload with the other configurations' sub-results; A, C, D, E: "
                         "one configuration alone; small, prof, prof_f: smaller INT8 shapes for profiler captures")
    ap.add_argument("--configs", default="ACDE",
                    help="configurations whose sub-results the default run adds (subset of ACDE, '' for none)")
    ap.add_argument("--c-window", type=int, default=256, help="FP16 workload: channels of the 4096 per step")
    ap.add_argument("--d-window", type=int, default=1024,
                    help="calibration workload: channels of the 1024 per step (smaller for profiler captures)")
    ap.add_argument("--e-window", type=int, default=16, help="batched workload: channels per sub-array")
    ap.add_argument("--xengine", default="auto", choices=["auto", "cudacore", "tcgen05"])
    ap.add_argument("--fengine", default="auto", choices=["auto", "cudacore"],
                    help="INT8 F-engine: tensor cores where they apply (1024 channels, no delays or filter bank) "
                         "or the CUDA-core FFT")
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
    if args.workload == "A":
        return _standalone(args, "A", lambda dev, pk: bench_A(args.steps, args.warmup, dev, pk, 2070.0))
    if args.workload == "C":
        return _standalone(args, "C", lambda dev, pk: bench_C(args.steps, args.warmup, dev, pk, args.c_window,
                                                              args.fused_dump))
    if args.workload == "D":
        return _standalone(args, "D", lambda dev, pk: bench_D(args.steps, args.warmup, dev, pk, args.comparator,
                                                              args.d_window))
    if args.workload == "E":
        return _standalone(args, "E", lambda dev, pk: bench_E(args.steps, args.warmup, dev, pk, args.e_window))
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())

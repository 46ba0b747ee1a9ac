"""Benchmark: streaming FDL convolution throughput on GB300.

One step = one block of the whole hot path (input pack + R2C FFT + FDL push,
FDL MAC over every partition and input->output pair, split reduction + C2R +
overlap-save) for the paper-scale workload: 4 microphone inputs x 16
loudspeaker outputs, 8 s filters (384,000 taps) at 48 kHz, block 256, FP32
spectra, synthetic pink-noise input and exponentially decaying noise filters
with early reflections.

Prints ONE JSON line (rank 0):
  value      Gtap*ch/s = n_in * n_out * taps * block / block time, inputs resident
             in device memory, all ranks together (each rank runs its own session)
  e2e        the same metric through the host-buffer C call, host<->device copies
             of every block inside the timed region; with p50/p99 block latency
  roofline   the FDL MAC kernel: algorithmic bytes / its CUDA-event duration
  cpu_baseline  the FP64 oracle timed on this host's cores on a bounded sample

``--impl reference`` times the FP64 oracle instead (rank 0 only).
"""

from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Gtap*ch/s of FDL convolution (% HBM roofline); p99 block latency vs block period"
UNIT = "Gtap*ch/s"
FALLBACK_HBM_GBS = 6800.0


# ------------------------------------------------------------------ helpers


def env_rank():
    return (
        int(os.environ.get("RANK", "0")),
        int(os.environ.get("LOCAL_RANK", "0")),
        int(os.environ.get("WORLD_SIZE", "1")),
    )


def aggregate(elapsed_s: float, units: float, dist=None):
    """Whole-job figures: max elapsed over ranks, sum of units over ranks."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return elapsed_s, units
    import torch

    t = torch.tensor([elapsed_s], dtype=torch.float64)
    u = torch.tensor([units], dtype=torch.float64)
    if dist.get_backend() == "nccl":
        t, u = t.cuda(), u.cuda()
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": FALLBACK_HBM_GBS}, "fallback"


def kernel_source_hash():
    """sha256 (first 16 hex digits) of the MAC's sources: kernels.cu,
    device_util.cuh, kernels.h, spectrum_store.cuh and the planner function
    plan_mac of engine.cu (it fixes the launch configuration)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2509_04390_gb300", "csrc")
    for name in ("kernels.cu", "device_util.cuh", "kernels.h", "spectrum_store.cuh"):
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(f.read())
    with open(os.path.join(csrc, "engine.cu"), "rb") as f:
        eng = f.read()
    start = eng.find(b"MacPlan plan_mac(")
    end = eng.find(b"\n}\n", start)
    h.update(eng[start:end] if start >= 0 and end > start else eng)
    return h.hexdigest()[:16]


def ncu_traffic(workload: str, field: str = "dram_bytes_per_launch"):
    """A DRAM figure from the committed ncu summary, if it was taken on the
    current kernel source (else None): dram_bytes_per_launch (one MAC launch,
    cold L2, read + write), dram_read_bytes_warm_l2 (one MAC launch, kernel
    replay with the L2 as the previous kernels left it) or
    dram_read_bytes_per_step_range (a whole step, range replay over 100
    blocks back to back)."""
    path = os.path.join(ROOT, "profiles", "fdl_mac_traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    entry = rec.get(workload)
    if not entry or entry.get("kernel_hash") != kernel_source_hash():
        return None
    return entry.get(field)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = (
        "index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
        "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
        "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap"
    )

    def __init__(self, gpu_index: int):
        self.samples = []
        self.proc = None
        self.gpu = gpu_index
        self.window = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.gpu)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        threading.Thread(target=self._read, daemon=True).start()

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append((time.time(), line.strip()))

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self, t0, t1):
        rows = []
        for ts, line in self.samples:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            rows.append((ts, parts))
        inside = [r for r in rows if t0 <= r[0] <= t1]
        use = inside if inside else rows
        if not use:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        sm = [float(p[1]) for _, p in use if p[1].replace(".", "", 1).isdigit()]
        smax = [float(p[2]) for _, p in use if p[2].replace(".", "", 1).isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, p in use for i in range(4) if p[5 + i].lower() == "active"})
        return {
            "sm_mhz": statistics.median(sm) if sm else None,
            "sm_max_mhz": max(smax) if smax else None,
            "reasons": reasons,
            "samples": len(use),
            "in_timed_region": bool(inside),
        }


def make_workload(args):
    from paper_2509_04390_gb300 import signals

    if args.afc:
        return signals.afc_4x16(block=args.block, seconds=args.seconds, taps=args.taps, taps_fb=args.taps_fb)
    return signals.paper_4x16(block=args.block, seconds=args.seconds, taps=args.taps)


def workload_name(args):
    if args.afc:
        nlms = "_nlms" if args.adapt > 0 else ""
        reuse = "_reuse_nf3" if args.reuse else ""
        return f"afc{nlms}_4x16_{args.taps}taps_fb{args.taps_fb}_B{args.block}{reuse}_{args.precision}"
    far = f"_far{args.far_block}" if args.far_block else ""
    if args.far_block and args.far_block2:
        far += f"_far{args.far_block2}"
    return f"paper_4x16_{args.taps}taps_B{args.block}{far}_{args.precision}"


def tapch(w):
    """Time-domain-equivalent tap*channel MACs of one block (both convolutions
    when the feedback canceller runs)."""
    t = float(w.n_in) * w.n_out * w.taps
    if w.f is not None:
        t += float(w.f.shape[0]) * w.f.shape[1] * w.f.shape[2]
    return t * w.block


def step_bandwidth(w, info, t_step, peak, warm_read=None):
    """Bytes per step over the step time.  The filter spectra (n_out * n_in *
    (K-1) * B * s bytes per tail) are read once per step; the delay line
    (n_in * K * B * s bytes, 12 MB at the paper configuration) is re-read by
    every output tile and stays L2-resident.  hbm_* counts the filter
    spectra; the engine keeps the first l2_keep_bytes of them in L2 from one
    block to the next, so hbm_* above the copy peak measures those L2 hits:
    at least (hbm_frac_of_peak - 1) of the copy peak's bytes per step come
    from L2."""
    s = 8 if info["precision"] == 0 else 4
    K, B = info["K"], w.block
    total = info["mac_bytes"] + step_extra_bytes(w, info)
    filt = w.n_out * w.n_in * (K - 1) * B * s
    if w.f is not None and info["K_fb"] > 1:
        filt += w.f.shape[0] * w.f.shape[1] * (info["K_fb"] - 1) * B * s
        total += info["mac_fb_bytes"]
    return {
        "algorithmic_bytes_per_step": int(total),
        "algorithmic_gbs": total / t_step / 1e9,
        "hbm_bytes_per_step": int(filt),
        "hbm_gbs": filt / t_step / 1e9,
        "hbm_frac_of_peak": filt / t_step / 1e9 / peak,
        # ncu range replay over 100 whole steps (every kernel running as it does live)
        "dram_read_bytes_per_step_measured": warm_read,
        "dram_frac_of_peak_measured": (warm_read / t_step / 1e9 / peak) if warm_read else None,
        "l2_kept_bytes": info.get("l2_keep_bytes"),
        "min_bytes_from_l2_per_step": int(max(0.0, filt - peak * 1e9 * t_step)),
        "note": "whole steps back to back (pack, head + output, tail MAC), each step's background tail inside "
                "the timed region; hbm_* counts the filter spectra, of which the engine keeps l2_kept_bytes in "
                "L2 between blocks; the delay line is L2-resident; consecutive tails overlap on two streams; so "
                "algorithmic_gbs and hbm_gbs are not DRAM throughput: at least min_bytes_from_l2_per_step per "
                "step come from L2",
    }


def step_extra_bytes(w, info):
    """Algorithmic bytes of a step outside the tail MAC: the head partition
    (filters + delay-line row), the new spectrum written, input and output."""
    s = 8 if info["precision"] == 0 else 4
    B = w.block
    return int((w.n_out + 1) * w.n_in * B * s + w.n_in * B * s + (w.n_in + w.n_out) * B * 4)


# ----------------------------------------------------------- CPU baseline


def time_oracle(w, budget_s: float, max_blocks: int | None = None, n_sub: int | None = None):
    """Time the FP64 oracle as it stands on a bounded sample of the workload:
    ``n_sub`` of the outputs for as many blocks as fit in ``budget_s``."""
    from oracle import UpolsOracle

    n_sub = w.n_out if n_sub is None else n_sub
    sub = np.ascontiguousarray(w.h[:n_sub])
    eng = UpolsOracle(sub, w.block)
    B = w.block
    nb_avail = w.x.shape[1] // B
    times = []
    t_start = time.perf_counter()
    b = 0
    while True:
        xb = w.x[:, (b % nb_avail) * B : (b % nb_avail + 1) * B]
        t0 = time.perf_counter()
        eng.process_block(xb)
        times.append(time.perf_counter() - t0)
        b += 1
        if time.perf_counter() - t_start > budget_s or (max_blocks and b >= max_blocks):
            break
    per_block = statistics.median(times)
    value = float(w.n_in) * n_sub * w.taps * B / per_block / 1e9
    return value, per_block, b, n_sub


def _oracle_worker(args):
    """One process of the all-cores oracle timing: UPOLS of one output slice."""
    h, x, B, n_blocks = args
    from oracle import UpolsOracle

    eng = UpolsOracle(h, B)
    nb_avail = x.shape[1] // B
    eng.process_block(x[:, :B])  # warm-up
    times = []
    for b in range(1, n_blocks + 1):
        xb = x[:, (b % nb_avail) * B : (b % nb_avail + 1) * B]
        t0 = time.perf_counter()
        eng.process_block(xb)
        times.append(time.perf_counter() - t0)
    return statistics.median(times)


def time_oracle_all_cores(w, budget_s: float, per_block_1: float):
    """The same oracle on every host core: the outputs split into one slice per
    process (spawned, so nothing inherits the CUDA context), all processes
    running the same blocks at once; the block time is the slowest slice's."""
    import multiprocessing as mp

    cores = os.cpu_count() or 1
    workers = max(1, min(cores, w.n_out))
    bounds = [round(i * w.n_out / workers) for i in range(workers + 1)]
    slices = [np.ascontiguousarray(w.h[bounds[i] : bounds[i + 1]]) for i in range(workers)]
    x = np.ascontiguousarray(w.x[:, : min(w.x.shape[1], 64 * w.block)])
    # blocks per process: the single-thread time per output scaled to the slice, within the budget
    per_out = per_block_1 / w.n_out
    n_blocks = int(max(3, min(200, budget_s / max(per_out * (bounds[1] - bounds[0]), 1e-6))))
    env_before = os.environ.get("OMP_NUM_THREADS")
    os.environ["OMP_NUM_THREADS"] = "1"
    try:
        with mp.get_context("spawn").Pool(workers) as pool:
            per = pool.map(_oracle_worker, [(h, x, w.block, n_blocks) for h in slices])
    finally:
        if env_before is None:
            os.environ.pop("OMP_NUM_THREADS", None)
        else:
            os.environ["OMP_NUM_THREADS"] = env_before
    per_block = max(per)
    value = float(w.n_in) * w.n_out * w.taps * w.block / per_block / 1e9
    return value, per_block, n_blocks, workers


# ------------------------------------------------------------------- arms


def run_reference(args):
    rank, _, world = env_rank()
    if rank != 0:
        return 0
    w = make_workload(args)
    from oracle import UpolsOracle

    # size each step so that warmup + steps finish within ~150 s
    probe = UpolsOracle(np.ascontiguousarray(w.h[:1]), w.block)
    t0 = time.perf_counter()
    probe.process_block(w.x[:, : w.block])
    t1 = time.perf_counter() - t0
    del probe
    per_output = max(t1, 1e-4)
    budget = 150.0 / max(1, args.steps + args.warmup)
    n_sub = int(max(1, min(w.n_out, budget // per_output)))
    from oracle import UpolsOracle as _U

    eng = _U(np.ascontiguousarray(w.h[:n_sub]), w.block)
    B = w.block
    nb = w.x.shape[1] // B
    for i in range(args.warmup):
        eng.process_block(w.x[:, (i % nb) * B : (i % nb + 1) * B])
    times = []
    for i in range(args.steps):
        j = (args.warmup + i) % nb
        t0 = time.perf_counter()
        eng.process_block(w.x[:, j * B : (j + 1) * B])
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = float(w.n_in) * n_sub * w.taps * B * args.steps / total / 1e9
    sample = f"{n_sub} of {w.n_out} outputs, {args.steps} blocks of {B} (FP64 numpy oracle, single thread)"
    line = {
        "impl": "reference",
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": total / args.steps * 1e3,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": config_dict(args, w),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def l2_bytes():
    """The current device's L2 cache size in bytes (126 MiB without a GPU)."""
    try:
        import torch

        props = torch.cuda.get_device_properties(torch.cuda.current_device())
        return int(getattr(props, "L2_cache_size", 0) or 126 * 2**20)
    except (RuntimeError, AssertionError, AttributeError, ImportError):
        return 126 * 2**20


def stream_bytes_of(args, w):
    """Algorithmic bytes the tail MACs of one step stream: partitions 1..K-1
    of every filter spectrum plus the matching delay-line rows (the engine's
    conv_info.mac_bytes + mac_fb_bytes)."""
    es = 8 if args.precision == "fp32" else 4
    bins = w.block * 3 // 2 if getattr(args, "reuse", False) else w.block

    def part(n_src, n_dst, taps):
        K = -(-taps // w.block)
        return (n_dst + 1) * n_src * (K - 1) * bins * es

    b = part(w.n_in, w.n_out, w.taps)
    if args.afc:
        b += part(w.n_out, w.n_in, args.taps_fb)
    return b


def l2_note(args, stream_bytes, l2):
    """config["l2"]: whether the bytes a step streams exceed the L2 cache."""
    if args.far_block:
        return ("inputs larger than L2: the far part's spectra, streamed once per far block, exceed the L2 "
                f"({l2 / 1e6:.0f} MB); the near part (block-size partitions up to the far block) stays "
                "L2-resident, as in real-time use")
    if stream_bytes > l2:
        return (f"inputs larger than L2: the {stream_bytes / 1e6:.1f} MB of spectra streamed every step exceed "
                f"the {l2 / 1e6:.0f} MB L2; the engine keeps the first "
                f"{56 if getattr(args, 'l2_keep', None) is None else args.l2_keep:g} MB of them in L2 from one block "
                "to the next (conv_set_l2_keep), the rest streams from HBM every step")
    return (f"working set below the L2 size ({stream_bytes / 1e6:.1f} MB of spectra per step, L2 {l2 / 1e6:.0f} MB): "
            "the step value is the steady state, in which part of each step's reads hit L2 as in real-time use; "
            "the roofline's launches are timed after an L2 flush (conv_profile_flush_l2)")


def config_dict(args, w):
    return {
        "workload": workload_name(args),
        "n_in": w.n_in,
        "n_out": w.n_out,
        "taps": w.taps,
        "filter_s": w.taps / w.fs,
        "block": w.block,
        "fs": w.fs,
        "precision": args.precision,
        "global_batch": 1,
        "parallelism": "replicas",
        "far_block": args.far_block or None,
        "far_block2": (args.far_block2 or None) if args.far_block else None,
        "l2": l2_note(args, stream_bytes_of(args, w), l2_bytes()),
    }


def run_ours(args):
    """The headline arm: returns rank 0's JSON line (None on other ranks)."""
    import torch

    rank, local_rank, world = env_rank()
    dist = None
    if world > 1:
        import torch.distributed as dist

        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend=backend)
    if not torch.cuda.is_available():
        raise RuntimeError("a CUDA device is required (the engine has no CPU path)")
    torch.cuda.set_device(local_rank)

    from paper_2509_04390_gb300 import upols as U

    w = make_workload(args)
    B = w.block
    prec = args.precision
    eng = U.Engine(w.fs, B, w.n_in, w.n_out, w.taps, prec, far_block=args.far_block, reuse=args.reuse)
    if args.l2_keep is not None:
        U.conv_set_l2_keep(eng.h, int(args.l2_keep * 1e6))
    far_h = U.conv_far_engine(eng.h) if args.far_block else None
    if far_h and args.far_block2:  # a third partition size: the far part's own far block
        U.conv_set_far_block(far_h, args.far_block2)
    eng.set_filters(w.h)
    if args.afc:
        eng.set_paths(w.f)
        if args.adapt > 0:
            eng.set_adaptation(args.adapt, 0.95, 1e-1)
    info = eng.info()
    nb = w.x.shape[1] // B
    d_x = torch.from_numpy(np.ascontiguousarray(w.x[:, : nb * B])).cuda()
    # block-major copy so each block's [n_in][B] input is contiguous
    d_blocks = d_x.reshape(w.n_in, nb, B).permute(1, 0, 2).contiguous()
    d_out = torch.empty((2, w.n_out, B), dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    # device addresses resolved once: the timed loop is the C-ABI call and the
    # engine's own launches, not Python tensor indexing
    lib = U.load()
    p_blocks = [d_blocks[i].data_ptr() for i in range(nb)]
    p_out = [d_out[0].data_ptr(), d_out[1].data_ptr()]
    p_stream = stream.cuda_stream

    def step(i):
        if args.afc:
            rc = lib.afc_process_block_async(eng.h, p_blocks[i % nb], p_out[i & 1], None, p_stream)
        else:
            rc = lib.conv_process_block_async(eng.h, p_blocks[i % nb], p_out[i & 1], p_stream)
        if rc:
            raise U.ConvError(rc, U.conv_last_error())

    def host_call(h_in, h_out):
        if args.afc:
            U.afc_process_block(eng.h, h_in, h_out, None, (w.n_in, w.n_out, B))
        else:
            U.conv_process_block(eng.h, h_in, h_out, (w.n_in, w.n_out, B))

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    clocks = ClockSampler(local_rank if "CUDA_VISIBLE_DEVICES" not in os.environ else 0)
    clocks.start()
    time.sleep(0.5)

    def timed_region(first):
        if dist is not None:
            dist.barrier()
        U.conv_synchronize(eng.h)  # nothing of the engine's runs into the region
        torch.cuda.synchronize()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for i in range(args.steps):
            step(first + i)
        # the region ends when everything the steps enqueued has finished,
        # including the last step's background tail MAC (for the next block):
        # S steps are credited with S tails, all inside the region
        lib.conv_join_async(eng.h, p_stream)
        ev1.record(stream)
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        return ev0.elapsed_time(ev1) / 1e3

    # region A: the measured value (kernels back to back, nothing in between)
    tw0 = time.time()
    elapsed = timed_region(args.warmup)
    tw1 = time.time()
    # region B: the same steps with CUDA events around every FDL MAC launch on
    # its stream (events between kernels serialise them, so this region is
    # only used for the kernel's own duration)
    U.conv_profile_enable(eng.h, args.steps + 16)
    # a working set below the L2 size would start each timed launch with its
    # data still cached: flush L2 before each one (outside its events)
    l2 = l2_bytes()
    stream_bytes = info["mac_bytes"] + info["mac_fb_bytes"]
    flushed = not far_h and stream_bytes <= l2
    if flushed:
        U.conv_profile_flush_l2(eng.h, 4 * l2)
    if far_h:
        U.conv_profile_enable(far_h, args.steps + 16)
    elapsed_prof = timed_region(args.warmup + args.steps)
    if flushed:
        U.conv_profile_flush_l2(eng.h, 0)
    mac_ms, mac_n = U.conv_profile_read(eng.h)
    U.conv_profile_enable(eng.h, 0)
    if far_h:
        near_mac = (mac_ms, mac_n)
        mac_ms, mac_n = U.conv_profile_read(far_h)
        U.conv_profile_enable(far_h, 0)
    U.conv_synchronize(eng.h)
    clocks.stop()
    units = tapch(w) * args.steps
    t_max, units_all = aggregate(elapsed, units, dist)
    value = units_all / t_max / 1e9

    # end to end through the multi-block host call (pinned host buffers, every
    # block's input copied in and its output copied out inside the timed region)
    e2e_chunk = max(1, min(args.e2e_chunk, nb))
    r_steps = max(e2e_chunk, (min(args.steps, args.e2e_steps * 4) // e2e_chunk) * e2e_chunk)
    r_value = None
    if not args.afc:
        h_rin = torch.empty((w.n_in, e2e_chunk * B), dtype=torch.float32).pin_memory().numpy()
        h_rout = torch.empty((w.n_out, e2e_chunk * B), dtype=torch.float32).pin_memory().numpy()
        eng.reset()
        for c in range(2):
            U.conv_process_blocks(eng.h, h_rin, h_rout, (w.n_in, w.n_out, B))
        if dist is not None:
            dist.barrier()
        tr0 = time.perf_counter()
        for c in range(r_steps // e2e_chunk):
            j = (c * e2e_chunk) % max(1, nb - e2e_chunk)
            np.copyto(h_rin, w.x[:, j * B : (j + e2e_chunk) * B])
            U.conv_process_blocks(eng.h, h_rin, h_rout, (w.n_in, w.n_out, B))
        tr1 = time.perf_counter()
        r_t, r_units = aggregate(tr1 - tr0, tapch(w) * r_steps, dist)
        r_value = r_units / r_t / 1e9

    # end to end through the single-block host call: copies in and out every block.
    # Python's cyclic garbage collector, which runs at points of its own
    # choosing, stays off over the latency loops below, as in a real-time
    # caller, so that none of its passes is counted as a call's latency.
    import gc

    gc.collect()
    gc.disable()
    eng.reset()
    h_in = np.empty((w.n_in, B), np.float32)
    h_out = np.empty((w.n_out, B), np.float32)
    e2e_steps = min(args.steps, args.e2e_steps)
    lat = []
    for i in range(min(args.warmup, 50)):
        np.copyto(h_in, w.x[:, (i % nb) * B : (i % nb + 1) * B])
        host_call(h_in, h_out)
    if dist is not None:
        dist.barrier()
    g0 = U.conv_get_host_graph(eng.h)[1]
    te0 = time.perf_counter()
    for i in range(e2e_steps):
        j = (i + 50) % nb
        t0 = time.perf_counter_ns()
        np.copyto(h_in, w.x[:, j * B : (j + 1) * B])
        host_call(h_in, h_out)
        lat.append(time.perf_counter_ns() - t0)
    te1 = time.perf_counter()
    g1 = U.conv_get_host_graph(eng.h)[1]
    e_t, e_units = aggregate(te1 - te0, tapch(w) * e2e_steps, dist)
    e2e_value = e_units / e_t / 1e9
    lat_us = np.array(lat) / 1e3
    period_us = B / w.fs * 1e6

    # real-time use: one host-buffer call per block period, latency of each call
    paced = []
    if args.paced_blocks > 0:
        period_ns = int(period_us * 1e3)
        t_next = time.perf_counter_ns() + period_ns
        for i in range(args.paced_blocks):
            while time.perf_counter_ns() < t_next:
                pass
            j = (i + 50 + e2e_steps) % nb
            t0 = time.perf_counter_ns()
            np.copyto(h_in, w.x[:, j * B : (j + 1) * B])
            host_call(h_in, h_out)
            paced.append(time.perf_counter_ns() - t0)
            t_next += period_ns
    g2 = U.conv_get_host_graph(eng.h)[1]
    gc.enable()
    paced_us = np.array(paced) / 1e3 if paced else None

    peaks, peak_kind = measured_peaks()
    peak = float(peaks.get("hbm_gbs", FALLBACK_HBM_GBS))
    mac_avg_s = mac_ms / 1e3 / max(mac_n, 1)
    roof_bytes = info["mac_far_bytes"] if far_h else info["mac_bytes"]
    achieved = roof_bytes / mac_avg_s / 1e9 if mac_n else None

    cpu = None
    if rank == 0 and not args.no_cpu_baseline and not args.afc:
        cv, per_block, nblk, n_sub = time_oracle(w, args.cpu_budget)
        cpu = {
            "value": cv,
            "unit": UNIT,
            "cores": 1,
            "kind": "oracle",
            "sample": f"{nblk} blocks of {B} on all {n_sub} outputs, FP64 numpy oracle, single thread "
                      f"(median {per_block * 1e3:.1f} ms per block)",
        }
        if args.cpu_all_cores:
            av, apb, anb, aw = time_oracle_all_cores(w, args.cpu_budget / 2, per_block)
            cpu["all_cores"] = {
                "value": av,
                "unit": UNIT,
                "cores": aw,
                "kind": "oracle",
                "sample": f"{anb} blocks of {B}, the 16 outputs split over {aw} spawned processes, same FP64 "
                          f"oracle (slowest slice {apb * 1e3:.1f} ms per block)",
            }

    clk = clocks.summary(tw0, tw1)
    if rank == 0:
        line = {
            "metric": METRIC,
            "value": value,
            "unit": UNIT,
            "n_gpus": world,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": t_max / args.steps * 1e3,
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f32" if prec == "fp32" else f"{prec} storage, f32 arithmetic",
            "data": "synthetic: seeded pink-noise input, exponentially decaying noise filters with early reflections",
            "config": config_dict(args, w),
            "e2e": {
                "value": r_value if r_value is not None else e2e_value,
                "unit": UNIT,
                "h2d_bytes_per_step": w.n_in * B * 4,
                "d2h_bytes_per_step": w.n_out * B * 4,
                "steps": r_steps if r_value is not None else e2e_steps,
                "call": (f"conv_process_blocks, {e2e_chunk} blocks per call from pinned host buffers"
                         if r_value is not None else "afc_process_block, one block per call"),
                "per_block_call": {"value": e2e_value, "steps": e2e_steps,
                                   "call": "conv_process_block / afc_process_block, one block per call"},
                "latency_us": {
                    "p50": float(np.percentile(lat_us, 50)),
                    "p99": float(np.percentile(lat_us, 99)),
                    "max": float(np.max(lat_us)),
                    "block_period": period_us,
                    "p99_over_period": float(np.percentile(lat_us, 99)) / period_us,
                    "mode": "back to back",
                    "graph_calls": g1 - g0,
                },
                "latency_paced_us": None if paced_us is None else {
                    "p50": float(np.percentile(paced_us, 50)),
                    "p99": float(np.percentile(paced_us, 99)),
                    "max": float(np.max(paced_us)),
                    "block_period": period_us,
                    "p99_over_period": float(np.percentile(paced_us, 99)) / period_us,
                    "blocks": len(paced_us),
                    "mode": "one call per block period (real-time use)",
                    # calls that went through conv_process_block's CUDA graph
                    # (the rest took the stream form: the previous tail still ran)
                    "graph_calls": g2 - g1,
                },
            },
            "step_bandwidth": step_bandwidth(w, info, t_max / args.steps, peak,
                                             ncu_traffic(workload_name(args), "dram_read_bytes_per_step_range")),
            "roofline": {
                "bound": "hbm",
                "kernel": "k_fdl_mac (far part, once per far block)" if far_h else "k_fdl_mac",
                "achieved": achieved,
                "peak": peak,
                "peak_kind": f"{peak_kind} hbm_gbs (copy test)",
                "unit": "GB/s",
                "frac": (achieved / peak) if achieved else None,
                "traffic": ncu_traffic(workload_name(args)),
                "traffic_kind": "ncu, cold L2 (ncu's default cache control), per launch",
                "traffic_warm_l2_ncu": ncu_traffic(workload_name(args), "dram_read_bytes_warm_l2"),
                "dram_read_bytes_per_step_range": ncu_traffic(workload_name(args), "dram_read_bytes_per_step_range"),
                "l2_kept_bytes": None if flushed else info.get("l2_keep_bytes"),
                "algorithmic_bytes_per_launch": roof_bytes,
                "avg_launch_us": mac_avg_s * 1e6,
                "launches_timed": mac_n,
                "timing": "CUDA events around each launch on its stream, second timed region of the same steps "
                          f"({elapsed_prof / args.steps * 1e6:.1f} us per step there)"
                          + ("; L2 flushed before each timed launch" if flushed else ""),
            },
            "cpu_baseline": cpu,
            "gpu_launches": args.steps * (info["kernels_per_afc_block"] if args.afc else info["kernels_per_block"])
            + (args.steps // (args.far_block // B)) * 3
            + ((args.steps // (args.far_block2 // B)) * 3 if args.far_block2 else 0) if args.far_block else
            args.steps * (info["kernels_per_afc_block"] if args.afc else info["kernels_per_block"]),
            "clocks": clk,
            "plan": {k: info[k] for k in ("K", "mac_ctas", "mac_splits", "mac_smem", "device_bytes")},
        }
    eng.close()
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return line if rank == 0 else None


BATCH_TILING = {"kernel": "tma", "warps": 8}


def run_batch(args):
    """Many independent heterogeneous sessions: one step = one block of every
    session, through one batched launch per stage; then the same sessions one
    engine call at a time (the unbatched per-session path) for comparison."""
    import torch

    from paper_2509_04390_gb300 import signals
    from paper_2509_04390_gb300 import upols as U

    rank, local_rank, world = env_rank()
    torch.cuda.set_device(local_rank)
    specs = signals.batch_sessions(args.batch, seed=args.batch_seed)
    engs = []
    t_setup = time.time()
    for sp in specs:
        e = U.Engine(signals.FS, sp.block, sp.n_in, sp.n_out, sp.taps, args.precision, BATCH_TILING)
        e.set_filters(sp.filters())
        engs.append(e)
    t_setup = time.time() - t_setup
    nbuf = 8
    d_x = [torch.from_numpy(sp.signal(nbuf)).cuda().reshape(sp.n_in, nbuf, sp.block).permute(1, 0, 2).contiguous()
           for sp in specs]
    d_y = [torch.empty((sp.n_out, sp.block), dtype=torch.float32, device="cuda") for sp in specs]
    stream = torch.cuda.current_stream()
    units = sum(sp.tapch_per_block() for sp in specs)
    batch = U.Batch(args.precision)
    for e in engs:
        batch.add(e)
    if args.persistent:
        batch.set_persistent(args.persistent)

    lib = U.load()
    p_stream = stream.cuda_stream
    n_s = len(specs)
    p_ins = [(ctypes.c_void_p * n_s)(*[x[k].data_ptr() for x in d_x]) for k in range(nbuf)]
    p_outs = (ctypes.c_void_p * n_s)(*[y.data_ptr() for y in d_y])
    p_x = [[x[k].data_ptr() for k in range(nbuf)] for x in d_x]
    p_y = [y.data_ptr() for y in d_y]

    def bstep(i):
        rc = lib.conv_batch_process_async(batch.b, p_ins[i % nbuf], p_outs, p_stream)
        if rc:
            raise U.ConvError(rc, U.conv_last_error())

    def ustep(i):
        for j, e in enumerate(engs):
            rc = lib.conv_process_block_async(e.h, p_x[j][i % nbuf], p_y[j], p_stream)
            if rc:
                raise U.ConvError(rc, U.conv_last_error())

    for i in range(args.warmup):
        bstep(i)
    torch.cuda.synchronize()
    batch.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for i in range(args.steps):
        bstep(args.warmup + i)
    lib.conv_batch_join_async(batch.b, p_stream)  # the last step's background tails inside the region
    ev1.record(stream)
    torch.cuda.synchronize()
    batch.synchronize()
    t_b = ev0.elapsed_time(ev1) / 1e3 / args.steps
    step_bytes = batch.step_bytes()
    for e in engs:
        batch.remove(e)
    batch.close()

    # unbatched: one engine call per session per step
    k_u = max(3, min(args.steps, 200))
    for i in range(3):
        ustep(i)
    torch.cuda.synchronize()
    ev0.record(stream)
    for i in range(k_u):
        ustep(i)
    for e in engs:
        lib.conv_join_async(e.h, p_stream)
    ev1.record(stream)
    torch.cuda.synchronize()
    for e in engs:
        U.conv_synchronize(e.h)
    t_u = ev0.elapsed_time(ev1) / 1e3 / k_u
    peaks, peak_kind = measured_peaks()
    peak = float(peaks.get("hbm_gbs", FALLBACK_HBM_GBS))
    line = {
        "metric": METRIC,
        "value": units / t_b / 1e9,
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": t_b * 1e3,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32" if args.precision == "fp32" else f"{args.precision} storage, f32 arithmetic",
        "data": "synthetic: seeded exponentially decaying noise filters, white-noise inputs",
        "config": {
            "workload": f"batch_{len(specs)}_sessions_{args.precision}"
                        + {0: "", 1: "_persistent", 2: "_persistent_graph"}[args.persistent],
            "step_form": {0: "one launch per stage", 1: "one persistent launch per step",
                          2: "one persistent launch per step, replayed from a CUDA graph"}[args.persistent],
            "sessions": len(specs),
            "n_in": "U{1..8}", "n_out": "U{2..32}", "filter_s": "U(2,12)", "block": "{64..1024}",
            "taps_total": int(sum(sp.n_in * sp.n_out * sp.taps for sp in specs)),
            "precision": args.precision,
            "l2": "inputs larger than L2: the filter spectra streamed every step exceed the 126 MB L2",
        },
        "step_bandwidth": {
            "algorithmic_bytes_per_step": step_bytes,
            "achieved_gbs": step_bytes / t_b / 1e9,
            "frac_of_peak": step_bytes / t_b / 1e9 / peak,
            "peak_kind": peak_kind,
        },
        "unbatched": {
            "value": units / t_u / 1e9,
            "ms_per_step": t_u * 1e3,
            "steps": k_u,
            "note": "same sessions, one engine call (3 launches) per session per step",
        },
        "gpu_launches": args.steps * (1 if args.persistent else 3),
        "setup_s": t_setup,
        "device_bytes": int(sum(e.info()["device_bytes"] for e in engs)),
    }
    for e in engs:
        e.close()
    return line


def run_group(args):
    """S sessions of the paper configuration sharing one filter set, in one
    shared-filter group (tensor-core MAC): one step = one block of every
    session.  Then the same sessions as S separate engines (one call each per
    step) for comparison."""
    import torch

    from paper_2509_04390_gb300 import signals
    from paper_2509_04390_gb300 import upols as U

    rank, local_rank, world = env_rank()
    torch.cuda.set_device(local_rank)
    prec = args.precision if args.precision != "fp32" else "fp16"
    S = args.group
    w = signals.paper_4x16(block=args.block, seconds=min(args.seconds, 8.0), taps=args.taps)
    B = w.block
    nb = w.x.shape[1] // B
    x = np.stack([np.roll(w.x[:, : nb * B], 4801 * s, axis=1) for s in range(S)]).astype(np.float32)
    d_blocks = torch.from_numpy(x).cuda().reshape(S, w.n_in, nb, B).permute(2, 0, 1, 3).contiguous()
    d_out = torch.empty((2, S, w.n_out, B), dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    grp = U.Group(prec, B, w.n_in, w.n_out, w.taps, S)
    if args.l2_keep is not None:
        U.conv_group_set_l2_keep(grp.g, int(args.l2_keep * 1e6))
    grp.set_filters(w.h)
    info = grp.info()
    units = float(S) * w.n_in * w.n_out * w.taps * B

    lib = U.load()
    p_blocks = [d_blocks[i].data_ptr() for i in range(nb)]
    p_out = [d_out[0].data_ptr(), d_out[1].data_ptr()]
    p_stream = stream.cuda_stream

    def step(i):
        rc = lib.conv_group_process_async(grp.g, p_blocks[i % nb], p_out[i & 1], p_stream)
        if rc:
            raise U.ConvError(rc, U.conv_last_error())

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    clocks = ClockSampler(local_rank if "CUDA_VISIBLE_DEVICES" not in os.environ else 0)
    clocks.start()
    time.sleep(0.5)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    tw0 = time.time()
    ev0.record(stream)
    for i in range(args.steps):
        step(args.warmup + i)
    lib.conv_group_join_async(grp.g, p_stream)  # the last step's background tail inside the region
    ev1.record(stream)
    torch.cuda.synchronize()
    tw1 = time.time()
    U.conv_group_synchronize(grp.g)
    t_step = ev0.elapsed_time(ev1) / 1e3 / args.steps
    # the MAC alone, CUDA events around each launch on its stream
    k_p = min(args.steps, 4000)
    U.conv_group_profile_enable(grp.g, k_p + 8)
    for i in range(k_p):
        step(i)
    torch.cuda.synchronize()
    mac_ms, mac_n = U.conv_group_profile_read(grp.g)
    U.conv_group_profile_enable(grp.g, 0)
    t_mac = mac_ms / 1e3 / max(1, mac_n)
    # end to end through the host-buffer calls: one block per call, and
    # e2e_chunk blocks per conv_group_process_blocks call from pinned buffers
    h_in = np.ascontiguousarray(x[:, :, :B])
    h_out = np.empty((S, w.n_out, B), np.float32)
    k_e = max(3, min(args.e2e_steps, 2000))
    grp.reset()
    for i in range(3):
        U.conv_group_process(grp.g, h_in, h_out, (S, w.n_in, w.n_out, B))
    t0 = time.perf_counter()
    for i in range(k_e):
        U.conv_group_process(grp.g, h_in, h_out, (S, w.n_in, w.n_out, B))
    t_e2e_1 = (time.perf_counter() - t0) / k_e
    C = max(1, min(args.e2e_chunk, nb))
    h_rin = torch.empty((S, w.n_in, C * B), dtype=torch.float32).pin_memory().numpy()
    h_rout = torch.empty((S, w.n_out, C * B), dtype=torch.float32).pin_memory().numpy()
    grp.reset()
    U.conv_group_process_blocks(grp.g, h_rin, h_rout, (S, w.n_in, w.n_out, B))
    n_calls = max(2, min(args.steps, 4 * args.e2e_steps) // C)
    t0 = time.perf_counter()
    for c in range(n_calls):
        j = (c * C) % max(1, nb - C)
        np.copyto(h_rin, x[:, :, j * B : (j + C) * B])
        U.conv_group_process_blocks(grp.g, h_rin, h_rout, (S, w.n_in, w.n_out, B))
    t_e2e = (time.perf_counter() - t0) / (n_calls * C)
    clocks.stop()
    grp.close()
    # the same sessions as separate engines (filters streamed once per session)
    engs = []
    for s in range(0 if args.no_separate else S):
        e = U.Engine(w.fs, B, w.n_in, w.n_out, w.taps, prec)
        e.set_filters(w.h)
        engs.append(e)
    d_o1 = torch.empty((w.n_out, B), dtype=torch.float32, device="cuda")
    k_u = max(3, min(args.steps, 500))
    p_sess = [[d_blocks[i][s].data_ptr() for s in range(S)] for i in range(min(nb, k_u + 3))]
    p_o1 = d_o1.data_ptr()

    def sep_step(i):
        for s, e in enumerate(engs):
            rc = lib.conv_process_block_async(e.h, p_sess[i % len(p_sess)][s], p_o1, p_stream)
            if rc:
                raise U.ConvError(rc, U.conv_last_error())

    for i in range(3):
        sep_step(i)
    torch.cuda.synchronize()
    ev0.record(stream)
    for i in range(k_u):
        sep_step(i)
    for e in engs:
        lib.conv_join_async(e.h, p_stream)
    ev1.record(stream)
    torch.cuda.synchronize()
    t_sep = ev0.elapsed_time(ev1) / 1e3 / k_u
    for e in engs:
        U.conv_synchronize(e.h)
        e.close()
    peaks, peak_kind = measured_peaks()
    peak = float(peaks.get("hbm_gbs", FALLBACK_HBM_GBS))
    mac_bytes = info["mac_bytes"]
    line = {
        "metric": METRIC,
        "value": units / t_step / 1e9,
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": t_step * 1e3,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": f"{prec} operands, f32 accumulation (tensor cores)",
        "data": "synthetic: the paper-scale filter set shared by all sessions; each session a shifted pink-noise input",
        "config": {
            "workload": f"group_{S}_sessions_paper_4x16_{w.taps}taps_B{B}_{prec}",
            "sessions": S, "n_in": w.n_in, "n_out": w.n_out, "taps": w.taps, "block": B, "precision": prec,
            "l2": (f"inputs larger than L2: the filter tiles and delay lines streamed every step exceed the "
                   f"{l2_bytes() / 1e6:.0f} MB L2; the first {60 if args.l2_keep is None else args.l2_keep:g} MB of "
                   "filter tiles stay in L2 from one block to the next (conv_group_set_l2_keep)"),
        },
        "roofline": {
            "bound": "hbm", "kernel": "k_group_mac", "achieved": mac_bytes / t_mac / 1e9, "peak": peak,
            "peak_kind": peak_kind, "unit": "GB/s", "frac": mac_bytes / t_mac / 1e9 / peak, "traffic": None,
            "algorithmic_bytes_per_launch": mac_bytes, "avg_launch_us": t_mac * 1e6, "launches_timed": mac_n,
        },
        "e2e": {
            "value": units / t_e2e / 1e9, "unit": UNIT, "h2d_bytes_per_step": int(h_in.nbytes),
            "d2h_bytes_per_step": int(h_out.nbytes), "steps": n_calls * C,
            "call": f"conv_group_process_blocks, {C} blocks per call from pinned host buffers",
            "per_block_call": {"value": units / t_e2e_1 / 1e9, "steps": k_e, "ms_per_call": t_e2e_1 * 1e3,
                               "call": "conv_group_process, one block per call"},
        },
        "separate_engines": None if args.no_separate else {
            "value": units / t_sep / 1e9, "ms_per_step": t_sep * 1e3, "steps": k_u,
            "note": "the same sessions as separate engines, one call (3 launches) each per step",
        },
        "plan": {k: info[k] for k in ("groups", "splits", "stages", "stage_k_steps", "mac_ctas", "mac_smem",
                                      "tmem_cols", "acc_buffers", "tail_streams", "device_bytes")},
        "gpu_launches": args.steps * info["kernels_per_block"],
        "clocks": clocks.summary(tw0, tw1),
    }
    return line


def run_serve(args):
    """Serving loop: Poisson arrivals with admission by device memory and
    continuous batching (p50/p99 tick latency vs the tick period), and the
    number of concurrent sessions sustained at p99 under the deadline,
    batched (FP16, FP32) against the plain per-session FP32 path."""
    import torch

    from paper_2509_04390_gb300 import serve

    rank, local_rank, world = env_rank()
    torch.cuda.set_device(local_rank)
    pool = serve.FilterPool()
    peaks, _ = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", FALLBACK_HBM_GBS))
    sims = [serve.simulate_poisson(p, duration_s=args.serve_seconds, pool=pool) for p in ("fp16", "fp32")]
    # FP32 with admission by HBM load as well as memory: no deadline misses by construction of the budget
    sims.append(serve.simulate_poisson("fp32", duration_s=args.serve_seconds, pool=pool, load_frac=0.6, hbm_gbs=hbm))
    caps = [
        serve.capacity("fp16", True, pool=pool),
        serve.capacity("fp32", True, pool=pool),
        serve.capacity("fp32", False, pool=pool),
    ]
    sim = sims[0]
    line = {
        "metric": "p99 block latency vs block period; sessions sustained (serving loop)",
        "value": sim["latency_us"]["p99"],
        "unit": "us (p99 tick latency, FP16)",
        "n_gpus": world,
        "higher_is_better": False,
        "dtype": "fp16 storage, f32 arithmetic",
        "data": "synthetic: Poisson arrivals 4/s, lifetimes U(5,60) s, 1-8 in x 8-64 out, 1-15 s filters, "
                "block 128 or 256, half with a 0.5 s feedback canceller",
        "config": {"workload": "serving", "tick": 128, "simulated_s": args.serve_seconds},
        "poisson": sims,
        "sustained": caps,
    }
    return line


EXTRA_KEYS = ("metric", "value", "unit", "ms_per_step", "steps", "warmup", "dtype", "config", "roofline", "e2e",
              "step_bandwidth", "unbatched", "separate_engines", "plan", "clocks", "gpu_launches", "poisson",
              "sustained", "higher_is_better", "planner", "speedup_vs_planner")


def run_tuned(args):
    """The autotuner on the headline shape: candidates timed on the real engine
    within a budget (objective: the back-to-back step), the winner cached in a
    private file, then the tuned engine against the planner's, both measured
    the same way."""
    import tempfile

    from paper_2509_04390_gb300 import autotune as A

    with tempfile.TemporaryDirectory() as tmp:
        path = os.path.join(tmp, "tiling.json")
        t0 = time.time()
        entry = A.tune(args.precision, args.block, 4, 16, args.taps, budget_s=args.tune_budget, steps=400,
                       path=path)
        tune_s = time.time() - t0
        h = A._filters(16, 4, args.taps)
        tuned = min(A.measure(entry["tiling"], args.precision, args.block, 4, 16, args.taps, h, steps=1000)
                    for _ in range(3))
        planner = min(A.measure({}, args.precision, args.block, 4, 16, args.taps, h, steps=1000) for _ in range(3))
    units = 4.0 * 16 * args.taps * args.block
    return {
        "metric": METRIC, "unit": UNIT, "value": units / tuned / 1e9, "ms_per_step": tuned * 1e3,
        "config": {"workload": f"paper_4x16_{args.taps}taps_B{args.block}_{args.precision}_tuned",
                   "tiling": entry["tiling"], "candidates_timed": entry["candidates_timed"],
                   "candidates": entry["candidates"], "tune_seconds": tune_s,
                   "filters": "exponentially decaying noise (the tuner's own), 4x16"},
        "planner": {"value": units / planner / 1e9, "ms_per_step": planner * 1e3},
        "speedup_vs_planner": planner / tuned,
    }


def run_extras(args):
    """The secondary configurations, each a short run of its own with its own
    timing and roofline, reported under "extra" of the headline line: block
    128 (the paper's default) and 512 at the headline shape, FP16 and BF16
    spectra, synthesis + feedback canceller (FP32, FP16; adaptive; in the
    n_f = 3 n_x spectrum-reuse form), non-uniform partitions (far block 2048),
    8 sessions sharing one filter set on the tensor cores, 64 heterogeneous
    FP16 sessions in one batch (per-stage launches, one persistent launch, its
    CUDA graph), a short serving run, and the autotuner.  A configuration
    that fails is reported with its error instead of ending the run."""
    import copy
    import traceback

    steps = max(3, min(args.steps, args.extra_steps))

    def variant(**kw):
        a = copy.copy(args)
        a.steps, a.warmup = steps, max(3, min(args.warmup, 50))
        a.seconds = min(args.seconds, 4.0)
        a.e2e_steps, a.paced_blocks, a.no_cpu_baseline = 300, 0, True
        a.far_block = a.far_block2 = 0
        a.afc, a.adapt, a.batch, a.group, a.serve, a.reuse = False, 0.0, 0, 0, False, False
        a.no_separate = False
        a.persistent = 0
        for k, v in kw.items():
            setattr(a, k, v)
        return a

    plan = [
        ("paper_4x16_B128_fp32", run_ours, variant(block=128)),
        ("paper_4x16_B512_fp32", run_ours, variant(block=512)),
        ("paper_4x16_B256_fp16", run_ours, variant(precision="fp16")),
        ("paper_4x16_B256_bf16", run_ours, variant(precision="bf16")),
        # with the real-time latency of the canceller's host call (2,000 paced blocks, 10.7 s)
        ("afc_4x16_B256_fp32", run_ours, variant(afc=True, paced_blocks=2000, e2e_steps=2000)),
        ("afc_4x16_B256_fp16", run_ours, variant(afc=True, precision="fp16")),
        ("afc_nlms_4x16_B256_fp32", run_ours, variant(afc=True, adapt=0.05)),
        ("paper_4x16_B256_far2048_fp32", run_ours, variant(far_block=2048)),
        ("afc_4x16_B256_fp32_reuse_nf3", run_ours, variant(afc=True, reuse=True)),
        ("afc_4x16_B256_fp16_reuse_nf3", run_ours, variant(afc=True, reuse=True, precision="fp16")),
        ("group_8_sessions_B256_fp16", run_group, variant(group=8, precision="fp16")),
        ("batch_64_sessions_fp16", run_batch, variant(batch=64, precision="fp16", steps=min(steps, 200))),
        ("batch_64_sessions_fp16_persistent", run_batch,
         variant(batch=64, precision="fp16", steps=min(steps, 200), persistent=1)),
        ("batch_64_sessions_fp16_persistent_graph", run_batch,
         variant(batch=64, precision="fp16", steps=min(steps, 200), persistent=2)),
        ("serving", run_serve, variant(serve=True, serve_seconds=min(args.serve_seconds, 5.0))),
        ("paper_4x16_B256_fp32_tuned", run_tuned, variant()),
        ("paper_4x16_B256_fp16_tuned", run_tuned, variant(precision="fp16")),
    ]
    # Each configuration runs in a fresh process (spawned: this one already
    # holds a CUDA context), so no configuration inherits device memory,
    # allocator or cache state from the ones before it.  Measured: the
    # adaptive canceller took 43-46 us per block after other configurations in
    # the same process, 39.8 us on its own.
    import multiprocessing

    ctx = multiprocessing.get_context("spawn")
    out = {}
    for name, fn, a in plan:
        if name not in args.extras:
            continue
        t0 = time.time()
        try:
            with ctx.Pool(1, maxtasksperchild=1) as pool:
                line = pool.apply(fn, (a,))
            out[name] = {k: line[k] for k in EXTRA_KEYS if k in line}
        except Exception as exc:  # noqa: BLE001 - reported, the headline stands
            out[name] = {"error": f"{type(exc).__name__}: {exc}", "trace": traceback.format_exc()[-800:]}
        out[name]["wall_s"] = round(time.time() - t0, 1)
    return out


ALL_EXTRAS = ("paper_4x16_B128_fp32,paper_4x16_B512_fp32,paper_4x16_B256_fp16,paper_4x16_B256_bf16,"
              "afc_4x16_B256_fp32,afc_4x16_B256_fp16,afc_nlms_4x16_B256_fp32,paper_4x16_B256_far2048_fp32,"
              "afc_4x16_B256_fp32_reuse_nf3,afc_4x16_B256_fp16_reuse_nf3,"
              "group_8_sessions_B256_fp16,batch_64_sessions_fp16,"
              "batch_64_sessions_fp16_persistent,batch_64_sessions_fp16_persistent_graph,serving,"
              "paper_4x16_B256_fp32_tuned,paper_4x16_B256_fp16_tuned")


def parse(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--warmup", type=int, default=200)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--block", type=int, default=256)
    ap.add_argument("--taps", type=int, default=384000)
    ap.add_argument("--seconds", type=float, default=30.0)
    ap.add_argument("--precision", choices=["fp32", "fp16", "bf16"], default="fp32")
    ap.add_argument("--afc", action="store_true", help="synthesis + feedback canceller (paths [4][16], 0.5 s)")
    ap.add_argument("--taps-fb", type=int, default=24000)
    ap.add_argument("--adapt", type=float, default=0.0, help="with --afc: NLMS step size of the adaptive canceller")
    ap.add_argument("--l2-keep", type=float, default=None,
                    help="MB of tail filter spectra kept in L2 between blocks (default: the engine's, 56)")
    ap.add_argument("--profile-range", type=int, default=0,
                    help="run this many blocks inside a profiler range (for ncu --replay-mode app-range) and exit")
    ap.add_argument("--reuse", action="store_true",
                    help="with --afc: the n_f = 3 n_x form, the synthesis output spectra feeding the canceller")
    ap.add_argument("--far-block", type=int, default=0,
                    help="non-uniform partitioning: taps beyond this many samples in partitions of this size")
    ap.add_argument("--far-block2", type=int, default=0,
                    help="with --far-block: taps beyond far-block + far-block2 in partitions of far-block2")
    # latency percentiles over 10,000 blocks each (the paced ones take 10,000 block periods, 53 s at B = 256)
    ap.add_argument("--e2e-steps", type=int, default=10000)
    ap.add_argument("--paced-blocks", type=int, default=10000)
    ap.add_argument("--e2e-chunk", type=int, default=64, help="blocks per conv_process_blocks call in the e2e figure")
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-all-cores", type=int, default=1,
                    help="also time the oracle on all host cores (one output slice per process); 0 to skip")
    ap.add_argument("--batch", type=int, default=0, help="time N heterogeneous sessions in one batch instead")
    ap.add_argument("--batch-seed", type=int, default=4)
    ap.add_argument("--serve", action="store_true", help="run the serving-loop simulation instead")
    ap.add_argument("--group", type=int, default=0, help="time N sessions sharing one filter set (tensor-core MAC)")
    ap.add_argument("--serve-seconds", type=float, default=15.0)
    ap.add_argument("--extras", default=ALL_EXTRAS,
                    help="comma-separated secondary configurations reported under 'extra' of the headline line "
                         "(single GPU, default run only); '' for none")
    ap.add_argument("--extra-steps", type=int, default=2000, help="timed steps of each secondary configuration")
    ap.add_argument("--tune-budget", type=float, default=15.0, help="seconds of candidate timing in the tuned extras")
    ap.add_argument("--persistent", type=int, nargs="?", const=1, default=0, choices=[0, 1, 2],
                    help="with --batch: each step as one persistent launch (1), replayed from a CUDA graph (2)")
    ap.add_argument("--no-separate", action="store_true",
                    help="with --group: skip the comparison with separate engines")
    return ap.parse_args(argv)


def run_profile_range(args):
    """--profile-range N: N blocks back to back, after the warm-up, inside a
    profiler range (cudaProfilerStart / Stop), so that ncu's range replay
    (`ncu --replay-mode app-range`) measures whole steps with every kernel
    running as it does live.  Prints the block time of the range."""
    import torch

    from paper_2509_04390_gb300 import upols as U

    torch.cuda.set_device(0)
    w = make_workload(args)
    B = w.block
    eng = U.Engine(w.fs, B, w.n_in, w.n_out, w.taps, args.precision, reuse=args.reuse)
    try:
        if args.l2_keep is not None:
            U.conv_set_l2_keep(eng.h, int(args.l2_keep * 1e6))
        eng.set_filters(w.h)
        if args.afc:
            eng.set_paths(w.f)
        nb = w.x.shape[1] // B
        d = torch.from_numpy(np.ascontiguousarray(w.x[:, : nb * B])).cuda()
        d = d.reshape(w.n_in, nb, B).permute(1, 0, 2).contiguous()
        out = torch.empty((2, w.n_out, B), dtype=torch.float32, device="cuda")
        stream = torch.cuda.current_stream()
        lib = U.load()

        def run(n, first):
            for i in range(n):
                j = first + i
                if args.afc:
                    rc = lib.afc_process_block_async(eng.h, d[j % nb].data_ptr(), out[j & 1].data_ptr(), None,
                                                     stream.cuda_stream)
                else:
                    rc = lib.conv_process_block_async(eng.h, d[j % nb].data_ptr(), out[j & 1].data_ptr(),
                                                      stream.cuda_stream)
                if rc:
                    raise U.ConvError(rc, U.conv_last_error())

        run(args.warmup, 0)
        U.conv_synchronize(eng.h)
        torch.cuda.synchronize()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.profiler.start()
        ev0.record(stream)
        run(args.profile_range, args.warmup)
        lib.conv_join_async(eng.h, stream.cuda_stream)
        ev1.record(stream)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        line = {"workload": workload_name(args), "blocks": args.profile_range,
                "us_per_block": ev0.elapsed_time(ev1) / args.profile_range * 1e3,
                "l2_keep_bytes": eng.info()["l2_keep_bytes"]}
    finally:
        eng.close()
    print(json.dumps(line), flush=True)
    return 0


def main(argv=None):
    args = parse(argv)
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.profile_range:
        return run_profile_range(args)
    args.extras = [x for x in args.extras.split(",") if x]
    if args.batch:
        line = run_batch(args)
    elif args.serve:
        line = run_serve(args)
    elif args.group:
        line = run_group(args)
    else:
        line = run_ours(args)
        _, _, world = env_rank()
        plain = not (args.afc or args.far_block or args.precision != "fp32" or args.block != 256)
        if line is not None and world == 1 and plain and args.extras:
            line["extra"] = run_extras(args)
    if line is not None:
        print(json.dumps(line), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())

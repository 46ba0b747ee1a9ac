"""Serving loop: many auralization sessions on one GPU.

* Admission by device-memory footprint (``conv_footprint``, host-only): a
  session is admitted when its spectra, delay lines and buffers fit in the
  budget; its state then stays resident on the device until it departs.
* Admission by HBM load (optional): the tail MAC streams every filter
  spectrum once per block, so a session adds ``tick_bytes`` to every tick;
  with a load fraction set, a session is admitted only while the sum stays
  below that fraction of the HBM bandwidth times the tick period.
* Continuous batching on a fixed tick (128 samples): each tick, the sessions
  whose next block is due (block 128: every tick, block 256: every other
  tick) are processed together, one batched launch per stage.  Sessions that
  arrive while others run join at the next tick; departures free their memory.
* Per tick, all due sessions' input blocks cross to the device in one copy
  and all outputs come back in one copy; the tick's latency is measured from
  the start of its input copy to its outputs on the host, against the tick
  period (the deadline of a block-128 session).

The engine runs every step; this module only schedules (host side).
"""

from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

from . import signals
from . import upols as U

BATCH_TILING = {"kernel": "tma", "warps": 8}
DEFAULT_HBM_GBS = 6704.5  # measured copy bandwidth of the GB300s this was tuned on


def tick_bytes(spec, precision, tick=128):
    """Algorithmic HBM bytes a session adds to each tick on average: every
    filter spectrum plus the delay-line rows of one output tile, per block
    ((n_out + 1) n_in K B s, s = bytes per complex value), and the same for
    the canceller, divided by the ticks per block."""
    s = 8 if precision in ("fp32", U.CONV_FP32) else 4
    K = -(-spec.taps // spec.block)
    per_block = (spec.n_out + 1) * spec.n_in * K * spec.block * s
    if spec.taps_fb:
        K_fb = -(-spec.taps_fb // spec.block)
        per_block += (spec.n_in + 1) * spec.n_out * K_fb * spec.block * s
    return per_block * tick / spec.block


@dataclass
class Session:
    sid: int
    spec: signals.SessionSpec
    eng: U.Engine
    footprint: int
    every: int  # ticks between blocks
    phase: int  # first tick
    x: np.ndarray  # cycled input, [n_in][n_buf * block]
    n_buf: int
    blocks: int = 0
    outputs: list = field(default_factory=list)
    keep_outputs: bool = False
    tick_bytes: float = 0.0


class FilterPool:
    """Seeded noise to cut filters from (drawing 10^8 normals per arriving
    session would dominate the set-up time); each session gets its own decay."""

    def __init__(self, seed=11, n_out=64, n_in=8, taps=15 * signals.FS):
        rng = np.random.default_rng(seed)
        self.noise = rng.standard_normal((n_out, n_in, taps), dtype=np.float32)

    def filters(self, spec):
        t = np.arange(spec.taps, dtype=np.float32) / signals.FS
        env = np.exp(np.float32(-signals.DECAY_60DB) * t / np.float32(spec.rt60)).astype(np.float32)
        env *= np.float32(1.0 / np.sqrt(max(1.0, float(np.sum(env * env)))))
        return np.ascontiguousarray(self.noise[: spec.n_out, : spec.n_in, : spec.taps] * env)


class Server:
    def __init__(self, precision="fp16", budget_bytes=None, tick=128, fs=signals.FS, load_frac=None,
                 hbm_gbs=DEFAULT_HBM_GBS):
        import torch

        self.torch = torch
        self.precision = precision
        self.tick = tick
        self.fs = fs
        if budget_bytes is None:
            free, _ = torch.cuda.mem_get_info()
            budget_bytes = int(free * 0.85)
        self.budget = int(budget_bytes)
        self.used = 0
        # HBM load admission: bytes per tick against load_frac of the bandwidth
        self.load_cap = None if load_frac is None else load_frac * hbm_gbs * 1e9 * tick / fs
        self.load = 0.0
        self.rejected_load = 0
        self.batch = U.Batch(precision)
        self.sessions: list[Session] = []  # batch order
        self.tick_index = 0
        self.next_sid = 0
        self.rejected = 0
        self._cap = 0
        self.stream = torch.cuda.current_stream()

    # ------------------------------------------------------------ admission

    def footprint(self, spec):
        return U.conv_footprint(self.precision, spec.block, spec.n_in, spec.n_out, spec.taps, spec.taps_fb)

    def admit(self, spec, filters, paths=None, x=None, keep_outputs=False):
        fp = self.footprint(spec)
        if self.used + fp > self.budget:
            self.rejected += 1
            return None
        tb = tick_bytes(spec, self.precision, self.tick)
        if self.load_cap is not None and self.load + tb > self.load_cap:
            self.rejected_load += 1
            return None
        eng = U.Engine(self.fs, spec.block, spec.n_in, spec.n_out, spec.taps, self.precision, BATCH_TILING)
        eng.set_filters(filters)
        if spec.taps_fb:
            eng.set_paths(paths if paths is not None else spec.paths())
        if x is None:
            x = spec.signal(8)
        n_buf = x.shape[1] // spec.block
        every = max(1, spec.block // self.tick)
        # start on the next tick that is due for this block size
        phase = self.tick_index + (-self.tick_index) % every
        s = Session(self.next_sid, spec, eng, fp, every, phase, np.ascontiguousarray(x), n_buf,
                    keep_outputs=keep_outputs)
        self.next_sid += 1
        self.batch.add(eng)
        self.sessions.append(s)
        self.used += fp
        self.load += tb
        s.tick_bytes = tb
        return s

    def depart(self, s):
        self.batch.remove(s.eng)
        self.sessions.remove(s)
        s.eng.close()
        self.used -= s.footprint
        self.load -= s.tick_bytes

    def close(self):
        for s in list(self.sessions):
            self.depart(s)
        self.batch.close()

    # ----------------------------------------------------------------- ticks

    def due(self):
        t = self.tick_index
        return [i for i, s in enumerate(self.sessions) if t >= s.phase and (t - s.phase) % s.every == 0]

    def _buffers(self, n_in_floats, n_out_floats):
        torch = self.torch
        need = max(n_in_floats, n_out_floats)
        if need > self._cap:
            cap = max(need, 2 * self._cap, 1 << 16)
            self.h_in = torch.empty(cap, dtype=torch.float32, pin_memory=True)
            self.h_out = torch.empty(cap, dtype=torch.float32, pin_memory=True)
            self.d_in = torch.empty(cap, dtype=torch.float32, device="cuda")
            self.d_out = torch.empty(cap, dtype=torch.float32, device="cuda")
            self._cap = cap

    def run_tick(self, batched=True):
        """Process every due session's next block.  Returns (latency_s, due
        sessions, tap*ch of the work)."""
        torch = self.torch
        idx = self.due()
        self.tick_index += 1
        if not idx:
            return 0.0, [], 0.0
        ss = [self.sessions[i] for i in idx]
        in_off, out_off = [], []
        ni = no = 0
        for s in ss:
            in_off.append(ni)
            out_off.append(no)
            ni += s.spec.n_in * s.spec.block
            no += s.spec.n_out * s.spec.block
        self._buffers(ni, no)
        h_in = self.h_in.numpy()
        for s, o in zip(ss, in_off):
            B = s.spec.block
            j = s.blocks % s.n_buf
            h_in[o : o + s.spec.n_in * B].reshape(s.spec.n_in, B)[:] = s.x[:, j * B : (j + 1) * B]
        t0 = time.perf_counter()
        self.d_in[:ni].copy_(self.h_in[:ni], non_blocking=True)
        base_in = self.d_in.data_ptr()
        base_out = self.d_out.data_ptr()
        ins = [base_in + 4 * o for o in in_off]
        outs = [base_out + 4 * o for o in out_off]
        if batched:
            U.conv_batch_process_some_async(self.batch.b, idx, ins, outs, self.stream)
        else:
            for s, a, b in zip(ss, ins, outs):
                if s.spec.taps_fb:
                    U.afc_process_block_async(s.eng.h, a, b, None, self.stream)
                else:
                    U.conv_process_block_async(s.eng.h, a, b, self.stream)
        self.h_out[:no].copy_(self.d_out[:no], non_blocking=True)
        self.stream.synchronize()
        lat = time.perf_counter() - t0
        h_out = self.h_out.numpy()
        work = 0.0
        for s, o in zip(ss, out_off):
            if s.keep_outputs:
                s.outputs.append(h_out[o : o + s.spec.n_out * s.spec.block].reshape(s.spec.n_out, -1).copy())
            s.blocks += 1
            work += s.spec.tapch_per_block()
        return lat, ss, work

    def hand_back(self):
        """Take every session out of the batch (for per-session processing)."""
        for s in self.sessions:
            self.batch.remove(s.eng)

    def take_in(self):
        for s in self.sessions:
            self.batch.add(s.eng)


def percentiles(lat_s):
    a = np.asarray(lat_s, dtype=np.float64) * 1e6
    if a.size == 0:
        return {"p50": None, "p99": None, "max": None}
    return {"p50": float(np.percentile(a, 50)), "p99": float(np.percentile(a, 99)), "max": float(a.max())}


def simulate_poisson(precision="fp16", duration_s=20.0, rate=4.0, life=(5.0, 60.0), seed=5, budget_bytes=None,
                     pool=None, load_frac=None, hbm_gbs=DEFAULT_HBM_GBS):
    """Poisson arrivals of serving sessions; ticks run back to back (simulated
    time advances one tick per iteration).  Set-up time of arriving sessions is
    kept out of the tick latencies."""
    rng = np.random.default_rng(seed)
    pool = pool or FilterPool()
    srv = Server(precision, budget_bytes, load_frac=load_frac, hbm_gbs=hbm_gbs)
    period = srv.tick / srv.fs
    n_ticks = int(duration_s / period)
    t_next = rng.exponential(1.0 / rate)
    departures = []
    lat, active, work, setup = [], [], 0.0, 0.0
    busy = 0.0
    k = 0
    for ti in range(n_ticks):
        t = ti * period
        while t_next <= t:
            spec = signals.serving_session(rng, seed * 1000 + k)
            k += 1
            t0 = time.perf_counter()
            s = srv.admit(spec, pool.filters(spec))
            setup += time.perf_counter() - t0
            if s is not None:
                departures.append((t + rng.uniform(*life), s))
            t_next += rng.exponential(1.0 / rate)
        for d in [d for d in departures if d[0] <= t]:
            srv.depart(d[1])
            departures.remove(d)
        l, ss, w = srv.run_tick()
        if ss:
            lat.append(l)
            busy += l
            work += w
        active.append(len(srv.sessions))
    out = {
        "precision": precision,
        "simulated_s": n_ticks * period,
        "tick_period_us": period * 1e6,
        "latency_us": percentiles(lat),
        "deadline_misses": int(sum(1 for x in lat if x > period)),
        "ticks": len(lat),
        "arrivals": k,
        "admitted": srv.next_sid,
        "rejected_by_memory": srv.rejected,
        "rejected_by_load": srv.rejected_load,
        "load_frac": load_frac,
        "active_sessions": {"mean": float(np.mean(active)), "max": int(np.max(active))},
        "budget_gb": srv.budget / 1e9,
        "throughput_gtapch_s": work / busy / 1e9 if busy else None,
        "setup_s": setup,
    }
    srv.close()
    return out


def capacity(precision="fp16", batched=True, start=4, step=4, max_sessions=128, ticks=64, seed=9, pool=None):
    """Largest number of concurrent serving sessions whose tick latency stays
    under the tick period at p99 (ticks back to back)."""
    rng = np.random.default_rng(seed)
    pool = pool or FilterPool()
    srv = Server(precision)
    period = srv.tick / srv.fs
    best, rows = 0, []
    n = 0
    k = 0
    while n < max_sessions:
        target = start if n == 0 else n + step
        while len(srv.sessions) < target:
            spec = signals.serving_session(rng, seed * 1000 + k)
            k += 1
            if srv.admit(spec, pool.filters(spec)) is None:
                break
        if len(srv.sessions) < target:
            break  # out of memory budget
        n = len(srv.sessions)
        if not batched:
            srv.hand_back()
        for _ in range(4):
            srv.run_tick(batched)
        lat = [srv.run_tick(batched)[0] for _ in range(ticks)]
        lat = [x for x in lat if x > 0]
        if not batched:
            srv.take_in()
        p = percentiles(lat)
        rows.append({"sessions": n, **p})
        if p["p99"] is not None and p["p99"] <= period * 1e6:
            best = n
        else:
            break
    srv.close()
    return {"precision": precision, "batched": batched, "sustained_sessions": best, "tick_period_us": period * 1e6,
            "sweep": rows}

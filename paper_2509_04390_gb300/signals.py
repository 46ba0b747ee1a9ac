"""Seeded synthetic workloads: filters and input signals.

Data only.  Nothing here performs the convolution or the feedback cancellation;
the GPU engine and the FP64 oracle both take these arrays as plain inputs.

The shapes and statistics follow the paper's workloads (48 kHz, very long
exponentially decaying reverberation filters, Sec. 6) scaled to the
configurations this engine is measured on:

* plain 1x2: h = N(0,1) * exp(-6.91 t / 1.0 s), 48,000 taps; input 2 s of
  white noise with sigma 0.1; block 256.
* paper scale 4x16: 8 s filters (384,000 taps), late part exponentially
  decaying noise with RT60 6 s plus 20 sparse early reflections (delays
  uniform 1-80 ms, gains uniform 0.1-0.8, random sign), each filter scaled
  to unit L2 norm; input 30 s of pink noise with RMS 0.1.
* feedback 4x16: the paper-scale synthesis set at block 256 plus simulated
  loudspeaker->microphone paths, 24,000 taps, RT60 0.3 s, each scaled to L2
  norm 0.1 (-20 dB), stored [mic][loudspeaker][taps].

``exp(-6.91 t / RT60)`` is the amplitude envelope that reaches -60 dB at
t = RT60 (20 log10(e^-6.91) = -60 dB).
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

FS = 48000
DECAY_60DB = 6.91  # ln(10^3): amplitude -60 dB


def exp_decay_noise(rng, lead_shape, taps, fs, rt60):
    """N(0,1) noise times the -60 dB-at-RT60 envelope, float64."""
    t = np.arange(taps, dtype=np.float64) / fs
    env = np.exp(-DECAY_60DB * t / rt60)
    return rng.standard_normal(tuple(lead_shape) + (taps,)) * env


def add_early_reflections(rng, h, fs, count=20, delay_ms=(1.0, 80.0), gain=(0.1, 0.8)):
    """Add ``count`` signed Diracs per filter at uniform delays/gains (in place)."""
    lead = h.shape[:-1]
    taps = h.shape[-1]
    flat = h.reshape(-1, taps)
    for i in range(flat.shape[0]):
        d = np.round(rng.uniform(delay_ms[0], delay_ms[1], count) * 1e-3 * fs).astype(np.int64)
        d = np.clip(d, 0, taps - 1)
        g = rng.uniform(gain[0], gain[1], count) * rng.choice([-1.0, 1.0], count)
        np.add.at(flat[i], d, g)
    return flat.reshape(lead + (taps,))


def normalise_l2(h, target):
    """Scale every filter (last axis) to L2 norm ``target``."""
    n = np.sqrt(np.sum(h * h, axis=-1, keepdims=True))
    n[n == 0] = 1.0
    return h * (target / n)


def white_noise(rng, n_ch, n, sigma):
    return rng.standard_normal((n_ch, n)) * sigma


def pink_noise(rng, n_ch, n, rms):
    """White FP64 noise shaped by 1/sqrt(f) in the frequency domain, scaled to ``rms``."""
    w = rng.standard_normal((n_ch, n))
    spec = np.fft.rfft(w, axis=-1)
    f = np.arange(spec.shape[-1], dtype=np.float64)
    shape = np.zeros_like(f)
    shape[1:] = 1.0 / np.sqrt(f[1:])
    x = np.fft.irfft(spec * shape, n=n, axis=-1)
    cur = np.sqrt(np.mean(x * x, axis=-1, keepdims=True))
    cur[cur == 0] = 1.0
    return x * (rms / cur)


@dataclass
class Workload:
    """One synthetic configuration (all arrays float32, C-contiguous)."""

    name: str
    fs: int
    block: int
    h: np.ndarray  # [n_out][n_in][taps]
    x: np.ndarray  # [n_in][T]
    f: np.ndarray | None = None  # [n_in][n_out][taps_fb]
    meta: dict = field(default_factory=dict)

    @property
    def n_out(self):
        return self.h.shape[0]

    @property
    def n_in(self):
        return self.h.shape[1]

    @property
    def taps(self):
        return self.h.shape[2]


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def plain_1x2(block=256, seconds=2.0, taps=48000, seed=1):
    """1 input x 2 outputs, 1 s exp-decay noise filters, white-noise input."""
    rng = np.random.default_rng(seed)
    h = exp_decay_noise(rng, (2, 1), taps, FS, 1.0)
    x = white_noise(rng, 1, int(round(seconds * FS)), 0.1)
    return Workload("plain_1x2_fp32", FS, block, _f32(h), _f32(x),
                    meta={"filter_s": taps / FS, "input_s": seconds})


def paper_filters(rng, n_out, n_in, taps, rt60=6.0, reflections=20):
    h = exp_decay_noise(rng, (n_out, n_in), taps, FS, rt60)
    if reflections:
        h = add_early_reflections(rng, h, FS, count=reflections)
    return normalise_l2(h, 1.0)


def paper_4x16(block=256, seconds=30.0, taps=384000, n_in=4, n_out=16, seed=2):
    """4 mic inputs x 16 loudspeaker outputs at paper scale (8 s filters)."""
    rng = np.random.default_rng(seed)
    h = paper_filters(rng, n_out, n_in, taps)
    x = pink_noise(rng, n_in, int(round(seconds * FS)), 0.1)
    return Workload(f"paper_{n_in}x{n_out}_B{block}", FS, block, _f32(h), _f32(x),
                    meta={"filter_s": taps / FS, "input_s": seconds})


def feedback_paths(rng, n_mic, n_spk, taps, rt60=0.3, norm=0.1):
    """Simulated loudspeaker->microphone paths, stored [mic][loudspeaker][taps]."""
    f = exp_decay_noise(rng, (n_mic, n_spk), taps, FS, rt60)
    return normalise_l2(f, norm)


def afc_4x16(block=256, seconds=30.0, taps=384000, taps_fb=24000, n_in=4, n_out=16, seed=2, seed_fb=3):
    """Synthesis set of ``paper_4x16`` plus feedback paths (F_hat = F)."""
    w = paper_4x16(block, seconds, taps, n_in, n_out, seed)
    rng = np.random.default_rng(seed_fb)
    f = feedback_paths(rng, n_in, n_out, taps_fb)
    w.f = _f32(f)
    w.name = f"afc_{n_in}x{n_out}_B{block}"
    w.meta["feedback_s"] = taps_fb / FS
    return w


def random_case(seed, n_in, n_out, taps, block, n_blocks, sigma=0.1, decay_s=None):
    """Small seeded case for parity tests: Gaussian filters (optionally decaying)."""
    rng = np.random.default_rng(seed)
    if decay_s:
        h = exp_decay_noise(rng, (n_out, n_in), taps, FS, decay_s)
    else:
        h = rng.standard_normal((n_out, n_in, taps)) / np.sqrt(max(taps, 1))
    x = white_noise(rng, n_in, block * n_blocks, sigma)
    return Workload(f"rand_{n_in}x{n_out}_t{taps}_B{block}", FS, block, _f32(h), _f32(x))


@dataclass
class SessionSpec:
    """Shape and seed of one auralization session; filters are drawn on demand."""

    n_in: int
    n_out: int
    taps: int
    block: int
    seed: int
    rt60: float
    taps_fb: int = 0

    def filters(self):
        rng = np.random.default_rng(self.seed)
        t = np.arange(self.taps, dtype=np.float32) / FS
        env = np.exp(np.float32(-DECAY_60DB) * t / np.float32(self.rt60)).astype(np.float32)
        h = rng.standard_normal((self.n_out, self.n_in, self.taps), dtype=np.float32)
        h *= env
        h *= np.float32(1.0 / np.sqrt(max(1.0, float(np.sum(env * env)))))
        return h

    def paths(self):
        rng = np.random.default_rng(self.seed + 7919)
        f = exp_decay_noise(rng, (self.n_in, self.n_out), self.taps_fb, FS, 0.3)
        return _f32(normalise_l2(f, 0.1))

    def signal(self, n_blocks, seed_offset=0):
        rng = np.random.default_rng(self.seed + 104729 + seed_offset)
        return rng.standard_normal((self.n_in, n_blocks * self.block), dtype=np.float32) * np.float32(0.1)

    def tapch_per_block(self):
        t = float(self.n_in) * self.n_out * self.taps
        if self.taps_fb:
            t += float(self.n_in) * self.n_out * self.taps_fb
        return t * self.block


def batch_sessions(count=64, seed=4):
    """Heterogeneous sessions: inputs U{1..8}, outputs U{2..32}, filters
    U(2, 12) s of exponentially decaying noise (RT60 = 3/4 of the length),
    blocks from {64, 128, 256, 512, 1024}."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        secs = float(rng.uniform(2.0, 12.0))
        out.append(SessionSpec(
            n_in=int(rng.integers(1, 9)), n_out=int(rng.integers(2, 33)), taps=int(secs * FS),
            block=int(rng.choice([64, 128, 256, 512, 1024])), seed=seed * 100003 + i, rt60=0.75 * secs))
    return out


def serving_session(rng, seed):
    """One arriving session of the serving workload: 1-8 inputs x 8-64 outputs,
    1-15 s filters, block 128 or 256, half with a feedback canceller (0.5 s paths)."""
    secs = float(rng.uniform(1.0, 15.0))
    afc = bool(rng.integers(0, 2))
    return SessionSpec(
        n_in=int(rng.integers(1, 9)), n_out=int(rng.integers(8, 65)), taps=int(secs * FS),
        block=int(rng.choice([128, 256])), seed=seed, rt60=0.75 * secs, taps_fb=24000 if afc else 0)

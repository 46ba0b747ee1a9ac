"""Shared helpers for the GPU tests: SNR, the simulated room, sample picking."""

from __future__ import annotations

import numpy as np


def snr_db(y, ref):
    """Output SNR 10 log10(sum |ref|^2 / sum |y - ref|^2), pooled over
    everything (real or complex arrays)."""
    y = np.asarray(y)
    ref = np.asarray(ref)
    if np.iscomplexobj(y) or np.iscomplexobj(ref):
        y = y.astype(np.complex128)
        ref = ref.astype(np.complex128)
    else:
        y = y.astype(np.float64)
        ref = ref.astype(np.float64)
    num = float(np.sum(np.abs(ref) ** 2))
    den = float(np.sum(np.abs(y - ref) ** 2))
    if den == 0.0:
        return float("inf")
    return 10.0 * np.log10(num / den)


def snr_per_channel_db(y, ref):
    return [snr_db(y[i], ref[i]) for i in range(ref.shape[0])]


class RoomPlant:
    """The simulated acoustic feedback paths F of a closed-loop test, FP64.

    ``step(l_n)`` returns (F * l) over block n's samples, from the loudspeaker
    history.  This is the physical environment the engine runs in (the true
    paths, not the engine's estimate); it uses numpy FFT convolution of the
    whole relevant history, with a transform long enough that nothing wraps.
    """

    def __init__(self, f, B):
        f = np.asarray(f, dtype=np.float64)
        self.P, self.L, self.n_t = f.shape
        self.B = B
        self.len = self.n_t - 1 + B
        n = 1
        while n < self.len + self.n_t:
            n <<= 1
        self.N = n
        self.F = np.fft.rfft(f, n, axis=-1)
        self.hist = np.zeros((self.L, self.len))

    def step(self, l_n):
        self.hist[:, : -self.B] = self.hist[:, self.B :]
        self.hist[:, -self.B :] = l_n
        Lf = np.fft.rfft(self.hist, self.N, axis=-1)
        y = np.fft.irfft(np.einsum("plk,lk->pk", self.F, Lf), self.N, axis=-1)
        return y[:, self.len - self.B : self.len]


def sample_points(rng, n_out, t_lo, t_hi, count):
    ls = rng.integers(0, n_out, count)
    ts = rng.integers(t_lo, t_hi, count)
    return list(zip(ls.tolist(), ts.tolist()))

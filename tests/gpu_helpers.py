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


def shift_blocks(c, B):
    """c over block n moved to block n+1 (the one-block delay of the
    cancellation, Sec. 5); the first block gets zeros."""
    out = np.zeros_like(c)
    out[:, B:] = c[:, :-B]
    return out


def replay_static_loop(h, f_hat, mic, B):
    """The oracle's closed loop of Sec. 5 driven by exactly the float32
    microphone blocks the engine received: no room, so the comparison holds
    only what the engine itself computed.  Returns (l, e) in FP64."""
    from oracle import afc_closed_loop

    P, L = f_hat.shape[0], f_hat.shape[1]
    l, e, _ = afc_closed_loop(h, np.zeros((P, L, 1)), f_hat, mic, B)
    return l, e


def replay_static_stages(h, f_hat, mic, l_eng, B):
    """Each stage of the loop fed with the engine's own signals: the synthesis
    of the engine's error signal is checked by comparing the engine's l with
    the oracle's UPOLS of the engine's e (done by the caller), and the
    canceller by the oracle's prediction from the engine's l, subtracted from
    the next microphone block.  Returns the oracle's e of that stage."""
    from oracle import upols

    c = upols(f_hat, l_eng.astype(np.float64), B)
    return mic.astype(np.float64) - shift_blocks(c, B)


def rms(a):
    a = np.asarray(a, dtype=np.float64)
    return float(np.sqrt(np.mean(a * a)))


def cancellation_gain_db(c, e):
    """How much larger the canceller's prediction c is than the error signal
    e = m - c it leaves (0 if smaller).  An FP32 prediction with relative
    error eps gives e a relative error of eps * rms(c) / rms(e): e's SNR is
    c's SNR minus this gain, whatever the implementation."""
    rc, re = rms(c), rms(e)
    return max(0.0, 20.0 * np.log10(rc / re)) if re > 0 and rc > 0 else 0.0


def check_replay(h, f_hat, y, e, mic, B, bound, label):
    """Like-for-like parity of a closed-loop run: each stage of the loop fed
    the engine's own signals, so the comparison holds only what the engine
    computed in that stage:
      synthesis  the engine's l against the oracle's UPOLS of the engine's e;
      canceller  the engine's prediction c = mic - e (over the previous block)
                 against the oracle's prediction from the engine's l, and e
                 itself, whose bound is lowered by the cancellation gain
                 rms(c) / rms(e) (a subtraction cannot keep more relative
                 precision than its operands have).
    The whole loop replayed from the microphone blocks alone is reported but
    not bounded: without the room its recursion e = m - F_hat * (H * e) has
    other dynamics than the physical loop (with F_hat = F it is unstable)."""
    from oracle import upols

    stage_l = upols(h.astype(np.float64), e.astype(np.float64), B)
    stage_e = replay_static_stages(h, f_hat, mic, y, B)
    c_eng = mic.astype(np.float64) - e.astype(np.float64)
    c_ref = mic.astype(np.float64) - stage_e
    gain = cancellation_gain_db(c_ref, stage_e)
    got = {
        "synthesis stage l": snr_db(y, stage_l),
        "canceller stage c": snr_db(c_eng, c_ref),
        "canceller stage e": snr_db(e, stage_e),
    }
    with np.errstate(all="ignore"):
        loop_l, loop_e = replay_static_loop(h, f_hat, mic, B)
    print(label + ": " + ", ".join(f"{k} {v:.1f} dB" for k, v in got.items())
          + f" (cancellation gain {gain:.1f} dB; whole loop replayed: l {snr_db(y, loop_l):.1f}, "
            f"e {snr_db(e, loop_e):.1f} dB)")
    assert got["synthesis stage l"] >= bound, got
    assert got["canceller stage c"] >= bound, got
    assert got["canceller stage e"] >= bound - gain, (got, gain)

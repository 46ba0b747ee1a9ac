"""FP64 CPU oracle for streaming uniformly-partitioned overlap-save convolution
and the block-delayed acoustic feedback canceller.

TEST INFRASTRUCTURE ONLY.  This module exists to check the GPU engine.  Only the
test-suite (``tests/``), ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import or call it.  The engine never calls it, and the two
share no code: no kernels, tables, helpers or pre/post-processing.  Its inputs
are plain numpy arrays (typically the float32 filters and signals that the
engine also receives, upcast here to float64).

Paper: H. Rosseel and T. van Waterschoot, "Accelerated Interactive Auralization
of Highly Reverberant Spaces using Graphics Hardware", arXiv 2509.04390.

Paper notation used below:
  n_x  block size (``B`` here)            n_h  filter length (``taps``)
  n_f  FFT size (= 2 n_x, Sec. 4)         K    number of sub-filters
  Q    conditioned inputs (= P microphones, pre-processor G taken as identity)
  L    loudspeakers (outputs)
  H_aur  Q x L synthesis filters, stored here as h[l][q][:]   (Eqs. 1-2)
  F_hat  P x L feedback-path estimates, stored as f[p][l][:]  (Eq. 3)

Readings of the paper taken here (the paper is silent or loose on these):
  R1  Time index: 0-based, no extra delay.  Eq. 4 is written with
      m = 1..n_h; we read it as y[t] = sum_{j=0}^{n_h-1} h[j] x[t-j].
  R2  K = ceil(n_h / n_x); the last sub-filter is zero-padded.  (Sec. 3.2
      states "n_h >= K n_k", which is the wrong direction for covering h.)
  R3  "Shifted up by one block" (Sec. 4, stage 2): the newest input spectrum
      meets sub-filter 0 (the k = 1 term of Eq. 6 carries delay 0).
  R4  FFT scaling: forward unscaled, inverse scaled by 1/n_f.
  R5  F_hat is P x L, indexed [mic p][loudspeaker l] (matrix of Eq. 3); the
      prose names the path "f_lp" but the matrix entries are f_pl.
  R6  "Subtracted from the next block" (Sec. 5): the prediction computed over
      block n is subtracted from microphone block n+1.  The closed-loop model
      therefore has a one-block acoustic/IO delay: m[t] = s[t] + (F*l)[t-B].
  R7  F_hat is known a priori and static (Sec. 1, Sec. 3.1); no adaptation.
  R8  The pre-processor G is the identity, so Q = P.

Every function states the passage it follows.
"""

from __future__ import annotations

import numpy as np

__all__ = [
    "mimo_fir",
    "mimo_fir_sample",
    "num_partitions",
    "UpolsOracle",
    "upols",
    "afc_closed_loop",
]


def num_partitions(n_h: int, B: int) -> int:
    """K = ceil(n_h / n_x)  (Sec. 4, reading R2)."""
    return -(-int(n_h) // int(B))


def mimo_fir(h: np.ndarray, x: np.ndarray, n_samples: int | None = None) -> np.ndarray:
    """Causal MIMO FIR filtering by its definition (Eq. 2 with Eq. 4's sum).

    y_l[t] = sum_q sum_{j=0}^{n_h-1} h[l, q, j] * x_q[t - j],  x[t < 0] = 0.

    h: [L][Q][n_h], x: [Q][T].  Returns float64 [L][n_samples] (default T).
    ``np.convolve`` (direct summation) is the per-pair step.
    """
    h = np.asarray(h, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    L, Q, _ = h.shape
    T = x.shape[1] if n_samples is None else int(n_samples)
    y = np.zeros((L, T))
    for l in range(L):
        for q in range(Q):
            full = np.convolve(h[l, q], x[q])
            n = min(T, full.shape[0])
            y[l, :n] += full[:n]
    return y


def mimo_fir_sample(h: np.ndarray, x: np.ndarray, l: int, t: int) -> float:
    """One output sample of Eq. 2 / Eq. 4: sum_q sum_j h[l,q,j] x_q[t-j].

    Used to check single samples of very long runs, where the full definition
    would take too long.  The sum runs over j = 0..min(t, n_h - 1).
    """
    n_h = h.shape[2]
    jmax = min(int(t), n_h - 1)
    acc = 0.0
    for q in range(h.shape[1]):
        hv = np.asarray(h[l, q, : jmax + 1], dtype=np.float64)
        xv = np.asarray(x[q, t - jmax : t + 1][::-1], dtype=np.float64)
        acc += float(np.dot(hv, xv))
    return acc


class UpolsOracle:
    """Streaming uniformly-partitioned overlap-save convolution, FP64 (Sec. 4).

    Initialisation (Sec. 4): every filter h_lq is split into K sub-filters of
    n_x taps, each sub-filter is padded with n_x zeros and transformed with an
    n_f = 2 n_x point real-to-complex FFT, giving h_bar[l, q, k, 0..n_x].

    ``process_block`` takes one input block x_n of shape [Q][n_x] and runs the
    three stages of Sec. 4 literally:
      1. input transformation: left-shift the n_f-sample sliding window by n_x,
         append x_n, R2C FFT -> x_bar_n (n_x + 1 bins);
      2. frequency-domain convolution: shift the FDL up by one block, put
         x_bar_n in slot 0, multiply every sub-filter spectrum with its FDL
         slot and accumulate (Eq. 6; the frequency-domain delay replaces the
         time-domain delta of Eq. 6 because n_k = n_x);
      3. output transformation: C2R IFFT of the accumulated spectrum (1/n_f
         scaling) and keep the last n_x samples (overlap-save).
    Returns float64 [L][n_x].
    """

    def __init__(self, h: np.ndarray, B: int):
        h = np.asarray(h, dtype=np.float64)
        if h.ndim != 3:
            raise ValueError("h must be [L][Q][n_h]")
        self.L, self.Q, self.n_h = h.shape
        self.B = int(B)
        self.n_f = 2 * self.B
        self.K = num_partitions(self.n_h, self.B)
        padded = np.zeros((self.L, self.Q, self.K * self.B))
        padded[:, :, : self.n_h] = h
        sub = padded.reshape(self.L, self.Q, self.K, self.B)
        # zero-pad each sub-filter by n_x and take the n_f-point R2C FFT
        self.h_bar = np.fft.rfft(sub, n=self.n_f, axis=-1)  # [L][Q][K][B+1]
        self.reset()

    def reset(self) -> None:
        self.window = np.zeros((self.Q, self.n_f))
        self.fdl = np.zeros((self.K, self.Q, self.B + 1), dtype=np.complex128)

    def process_block(self, x_n: np.ndarray) -> np.ndarray:
        x_n = np.asarray(x_n, dtype=np.float64).reshape(self.Q, self.B)
        # stage 1: input packing (left shift by n_x, append) and R2C FFT
        self.window[:, : self.B] = self.window[:, self.B :]
        self.window[:, self.B :] = x_n
        x_bar = np.fft.rfft(self.window, axis=-1)  # [Q][B+1]
        # stage 2: FDL shifted up by one block; newest spectrum in slot 0
        self.fdl[1:] = self.fdl[:-1].copy()
        self.fdl[0] = x_bar
        acc = np.zeros((self.L, self.B + 1), dtype=np.complex128)
        for k in range(self.K):
            # sub-filter k meets the spectrum from k blocks ago, summed over q
            acc += (self.h_bar[:, :, k, :] * self.fdl[k][None, :, :]).sum(axis=1)
        # stage 3: C2R IFFT (1/n_f) and overlap-save: keep the last n_x samples
        y = np.fft.irfft(acc, n=self.n_f, axis=-1)
        return y[:, self.B :]


def upols(h: np.ndarray, x: np.ndarray, B: int, n_blocks: int | None = None) -> np.ndarray:
    """Run ``UpolsOracle`` block by block over x [Q][T] (Sec. 4).

    The input is zero-extended to a whole number of blocks.  Returns float64
    [L][n_blocks * B] (default n_blocks = ceil(T / B)).
    """
    x = np.asarray(x, dtype=np.float64)
    eng = UpolsOracle(h, B)
    T = x.shape[1]
    nb = -(-T // B) if n_blocks is None else int(n_blocks)
    xp = np.zeros((eng.Q, nb * B))
    n = min(T, nb * B)
    xp[:, :n] = x[:, :n]
    out = np.zeros((eng.L, nb * B))
    for b in range(nb):
        out[:, b * B : (b + 1) * B] = eng.process_block(xp[:, b * B : (b + 1) * B])
    return out


def afc_closed_loop(
    h: np.ndarray,
    f_true: np.ndarray,
    f_hat: np.ndarray,
    s: np.ndarray,
    B: int,
    n_blocks: int | None = None,
):
    """Closed-loop auralization with feedback cancellation, FP64.

    System of Sec. 3.1 (Fig. 1, Eqs. 1-3) with the block timing of Sec. 5:
      h      [L][P][n_h]   synthesis filters H_aur (l <- q, q = p, R8)
      f_true [P][L][n_t]   the true acoustic paths F (loudspeaker l -> mic p)
      f_hat  [P][L][n_fb]  the a-priori estimate F_hat (R5, R7)
      s      [P][T]        the dry source signal reaching the microphones
    Per block n (R6):
      m_n = s_n + (F * l) over block n-1's samples      (microphone signal)
      e_n = m_n - c_{n-1}                               (cancellation, Sec. 5)
      l_n = (H_aur^T * e) over block n                  (Eq. 2)
      c_n = (F_hat * l) over block n                    (Eq. 3)
    All three convolutions are FP64 UPOLS (``UpolsOracle``).
    Returns (l [L][nb*B], e [P][nb*B], m [P][nb*B]).
    """
    synth = UpolsOracle(h, B)
    canceller = UpolsOracle(f_hat, B)
    room = UpolsOracle(f_true, B)
    P = synth.Q
    if canceller.L != P or room.L != P or canceller.Q != synth.L or room.Q != synth.L:
        raise ValueError("shape mismatch between H_aur [L][P], F [P][L], F_hat [P][L]")
    s = np.asarray(s, dtype=np.float64)
    T = s.shape[1]
    nb = -(-T // B) if n_blocks is None else int(n_blocks)
    sp = np.zeros((P, nb * B))
    n = min(T, nb * B)
    sp[:, :n] = s[:, :n]
    l_out = np.zeros((synth.L, nb * B))
    e_out = np.zeros((P, nb * B))
    m_out = np.zeros((P, nb * B))
    fb_prev = np.zeros((P, B))
    c_prev = np.zeros((P, B))
    for b in range(nb):
        sl = slice(b * B, (b + 1) * B)
        m_n = sp[:, sl] + fb_prev
        e_n = m_n - c_prev
        l_n = synth.process_block(e_n)
        c_prev = canceller.process_block(l_n)
        fb_prev = room.process_block(l_n)
        l_out[:, sl] = l_n
        e_out[:, sl] = e_n
        m_out[:, sl] = m_n
    return l_out, e_out, m_out

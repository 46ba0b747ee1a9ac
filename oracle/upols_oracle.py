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
  n_f  FFT size (2 n_x, Sec. 4; 3 n_x     K    number of sub-filters
       for the spectrum reuse of Sec. 5)
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
  R15 The spectrum reuse of Sec. 5's closing remark (only its FFT size,
      n_f = 3 n_x, and its cost are given): both convolutions at n_f = 3 n_x,
      the synthesis accumulated spectrum entering the canceller's FDL in
      place of the transform of the canceller's input window
      (``afc_closed_loop_reuse``).

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
    "afc_closed_loop_reuse",
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
    n_x taps, each sub-filter is zero-padded to n_f samples and transformed
    with an n_f-point real-to-complex FFT, giving h_bar[l, q, k, 0..n_f/2].
    The paper's default is n_f = 2 n_x; its Sec. 5 remark on reusing the
    synthesis output spectra needs n_f = 3 n_x.  Any n_f >= 2 n_x gives the
    same output: a sub-filter of n_x taps leaves the last n_x samples of the
    circular convolution free of wrap-around.

    ``process_block`` takes one input block x_n of shape [Q][n_x] and runs the
    three stages of Sec. 4 literally:
      1. ``transform_input``: left-shift the n_f-sample sliding window by n_x,
         append x_n, R2C FFT -> x_bar_n (n_f/2 + 1 bins);
      2. ``accumulate``: shift the FDL up by one block, put x_bar_n in slot 0,
         multiply every sub-filter spectrum with its FDL slot and accumulate
         (Eq. 6; the frequency-domain delay replaces the time-domain delta of
         Eq. 6 because n_k = n_x);
      3. ``transform_output``: C2R IFFT of the accumulated spectrum (1/n_f
         scaling) and keep the last n_x samples (overlap-save).
    Returns float64 [L][n_x].
    """

    def __init__(self, h: np.ndarray, B: int, n_f: int | None = None):
        h = np.asarray(h, dtype=np.float64)
        if h.ndim != 3:
            raise ValueError("h must be [L][Q][n_h]")
        self.L, self.Q, self.n_h = h.shape
        self.B = int(B)
        self.n_f = 2 * self.B if n_f is None else int(n_f)
        if self.n_f < 2 * self.B:
            raise ValueError("overlap-save with n_x-tap sub-filters needs n_f >= 2 n_x")
        self.bins = self.n_f // 2 + 1
        self.K = num_partitions(self.n_h, self.B)
        padded = np.zeros((self.L, self.Q, self.K * self.B))
        padded[:, :, : self.n_h] = h
        sub = padded.reshape(self.L, self.Q, self.K, self.B)
        # zero-pad each sub-filter to n_f and take the n_f-point R2C FFT
        self.h_bar = np.fft.rfft(sub, n=self.n_f, axis=-1)  # [L][Q][K][bins]
        self.reset()

    def reset(self) -> None:
        self.window = np.zeros((self.Q, self.n_f))
        self.fdl = np.zeros((self.K, self.Q, self.bins), dtype=np.complex128)

    def transform_input(self, x_n: np.ndarray) -> np.ndarray:
        """Stage 1: input packing (left shift by n_x, append) and R2C FFT."""
        x_n = np.asarray(x_n, dtype=np.float64).reshape(self.Q, self.B)
        self.window[:, : self.n_f - self.B] = self.window[:, self.B :].copy()
        self.window[:, self.n_f - self.B :] = x_n
        return np.fft.rfft(self.window, axis=-1)  # [Q][bins]

    def accumulate(self, x_bar: np.ndarray) -> np.ndarray:
        """Stage 2: the FDL shifted up by one block, the newest spectrum in
        slot 0, and the sum over sub-filters and inputs.  Returns [L][bins]."""
        self.fdl[1:] = self.fdl[:-1].copy()
        self.fdl[0] = x_bar
        acc = np.zeros((self.L, self.bins), dtype=np.complex128)
        for k in range(self.K):
            # sub-filter k meets the spectrum from k blocks ago, summed over q
            acc += (self.h_bar[:, :, k, :] * self.fdl[k][None, :, :]).sum(axis=1)
        return acc

    def transform_output(self, acc: np.ndarray) -> np.ndarray:
        """Stage 3: C2R IFFT (1/n_f) and overlap-save: the last n_x samples."""
        y = np.fft.irfft(acc, n=self.n_f, axis=-1)
        return y[:, self.n_f - self.B :]

    def process_block(self, x_n: np.ndarray) -> np.ndarray:
        return self.transform_output(self.accumulate(self.transform_input(x_n)))


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


def afc_closed_loop_reuse(
    h: np.ndarray,
    f_true: np.ndarray,
    f_hat: np.ndarray,
    s: np.ndarray,
    B: int,
    n_blocks: int | None = None,
):
    """The closed loop of ``afc_closed_loop`` with the synthesis output
    spectra fed straight into the canceller (the remark closing Sec. 5).

    Synthesis and canceller both use n_f = 3 n_x.  The synthesis accumulated
    spectrum Y_n is the spectrum of a 3 n_x window whose first n_x samples
    are wrap-around and whose last 2 n_x samples are [l_{n-1}, l_n]
    (Sec. 4: with n_x-tap sub-filters, positions >= n_x - 1 of the circular
    convolution are the linear one).  The canceller puts Y_n into its FDL in
    place of the R2C transform of its own input window: its n_x-tap
    sub-filters reach at most n_x - 1 samples back from the last n_x
    positions, so its kept output never sees the wrap-around part.  Per block:
      m_n, e_n            as in ``afc_closed_loop``
      Y_n = synthesis stages 1 + 2 on e_n;   l_n = stage 3 of Y_n
      C_n = canceller stage 2 on Y_n;        c_n = stage 3 of C_n
    The room (the true paths F) is the plain n_f = 2 n_x convolution.
    Returns (l [L][nb*B], e [P][nb*B], m [P][nb*B]), equal to
    ``afc_closed_loop`` up to FP64 rounding.
    """
    synth = UpolsOracle(h, B, n_f=3 * B)
    canceller = UpolsOracle(f_hat, B, n_f=3 * B)
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
        Y = synth.accumulate(synth.transform_input(e_n))
        l_n = synth.transform_output(Y)
        c_prev = canceller.transform_output(canceller.accumulate(Y))
        fb_prev = room.process_block(l_n)
        l_out[:, sl] = l_n
        e_out[:, sl] = e_n
        m_out[:, sl] = m_n
    return l_out, e_out, m_out

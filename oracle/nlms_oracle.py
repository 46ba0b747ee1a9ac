"""FP64 CPU oracle for the adaptive feedback canceller (an extension beyond the
paper): the partitioned-block frequency-domain NLMS update of F_hat.

TEST INFRASTRUCTURE ONLY.  Only the test-suite (``tests/``),
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import or call it.  The engine never calls it, and the two share no code.

The paper (Sec. 1, Sec. 3.1) takes the feedback-path estimate F_hat as known
a priori and static; it gives no adaptation rule.  This module defines the
adaptive variant the engine offers, in the same notation as ``upols_oracle``
(n_x = B block, n_f = 2B FFT, K_fb sub-filters, P microphones, L
loudspeakers), and the closed loop of Sec. 3.1 / Sec. 5 with that update.

Readings taken here, all beyond the paper:
  R12  The canceller is the UPOLS convolution of Sec. 4 with F_hat held as
       sub-filter spectra W[p][l][j][0..B] (n_f-point R2C of the zero-padded
       sub-filters at start), and the loudspeaker signals in its FDL.
  R13  Update (unconstrained partitioned-block FDAF with per-bin power
       normalisation), once per block, when the error e_n of microphone block n
       is known and before l_n enters the FDL:
         E_p      = R2C_nf( [0_B | e_n,p] )                  (error spectrum)
         pow[k]   = lam * pow[k] + (1 - lam) * sum_l |U_{l,n-1}[k]|^2
         W[p][l][j][k] += mu * E_p[k] * conj(U_{l,n-1-j}[k]) / (K_fb pow[k] + delta)
       U_{l,n-1-j} is the FDL entry j at that moment (the spectra that produced
       the prediction c_{n-1} subtracted from block n, R6).  pow starts at 0.
       "Unconstrained": the gradient is not projected back to n_x taps, so the
       sub-filter spectra leave the set of zero-padded n_x-tap spectra.
  R14  DC and Nyquist bins take the same update with their own power (both are
       real for real signals, so their products are real).

Every function states the passage it follows.
"""

from __future__ import annotations

import numpy as np

from .upols_oracle import UpolsOracle, num_partitions

__all__ = ["NlmsCanceller", "afc_closed_loop_nlms"]


class NlmsCanceller:
    """The feedback canceller of Sec. 5 (Eq. 3 by UPOLS, Sec. 4) with the
    NLMS update of reading R13.  FP64.

    f_hat0: [P][L][n_fb] initial estimate (time domain, may be all zeros).
    ``predict(l_n)`` runs the three UPOLS stages on loudspeaker block l_n and
    returns c_n [P][B]; ``adapt(e)`` applies the update with the FDL as it is.
    """

    def __init__(self, f_hat0: np.ndarray, B: int, mu: float, lam: float, delta: float):
        f = np.asarray(f_hat0, dtype=np.float64)
        if f.ndim != 3:
            raise ValueError("f_hat0 must be [P][L][n_fb]")
        self.P, self.L, n_fb = f.shape
        self.B = int(B)
        self.n_f = 2 * self.B
        self.K = num_partitions(n_fb, self.B)
        padded = np.zeros((self.P, self.L, self.K * self.B))
        padded[:, :, :n_fb] = f
        # initial sub-filter spectra, as in the initialisation of Sec. 4
        self.W = np.fft.rfft(padded.reshape(self.P, self.L, self.K, self.B), n=self.n_f, axis=-1)
        self.mu = float(mu)
        self.lam = float(lam)
        self.delta = float(delta)
        self.window = np.zeros((self.L, self.n_f))
        self.fdl = np.zeros((self.K, self.L, self.B + 1), dtype=np.complex128)
        self.power = np.zeros(self.B + 1)

    def predict(self, l_n: np.ndarray) -> np.ndarray:
        """Sec. 4 stages 1-3 on the loudspeaker block: c_n = (F_hat * l) over block n."""
        l_n = np.asarray(l_n, dtype=np.float64).reshape(self.L, self.B)
        self.window[:, : self.B] = self.window[:, self.B :]
        self.window[:, self.B :] = l_n
        self.fdl[1:] = self.fdl[:-1].copy()
        self.fdl[0] = np.fft.rfft(self.window, axis=-1)
        acc = np.zeros((self.P, self.B + 1), dtype=np.complex128)
        for j in range(self.K):
            acc += (self.W[:, :, j, :] * self.fdl[j][None, :, :]).sum(axis=1)
        return np.fft.irfft(acc, n=self.n_f, axis=-1)[:, self.B :]

    def error_spectrum(self, e: np.ndarray) -> np.ndarray:
        """E_p = R2C of the error block preceded by B zeros (R13)."""
        e = np.asarray(e, dtype=np.float64).reshape(self.P, self.B)
        padded = np.zeros((self.P, self.n_f))
        padded[:, self.B :] = e
        return np.fft.rfft(padded, axis=-1)

    def gradient(self, e: np.ndarray) -> np.ndarray:
        """G[p][l][j][k] = E_p[k] conj(U_{l, j}[k]) with the FDL as it is (R13)."""
        E = self.error_spectrum(e)
        return E[:, None, None, :] * np.conj(self.fdl.transpose(1, 0, 2))[None, :, :, :]

    def adapt(self, e: np.ndarray) -> None:
        """One NLMS step (R13, R14): power recursion, then the normalised update."""
        inst = np.sum(np.abs(self.fdl[0]) ** 2, axis=0)  # sum over loudspeakers, [B+1]
        self.power = self.lam * self.power + (1.0 - self.lam) * inst
        step = self.mu / (self.K * self.power + self.delta)
        self.W += self.gradient(e) * step[None, None, None, :]


def afc_closed_loop_nlms(
    h: np.ndarray,
    f_true: np.ndarray,
    f_hat0: np.ndarray,
    s: np.ndarray,
    B: int,
    mu: float,
    lam: float,
    delta: float,
    n_blocks: int | None = None,
):
    """Closed loop of Sec. 3.1 with the block timing of Sec. 5 (R6) and the
    adaptive canceller of R13.  Per block n:
      m_n = s_n + (F * l) over block n-1's samples
      e_n = m_n - c_{n-1}
      F_hat <- NLMS update with e_n (FDL holds l up to block n-1)
      l_n = (H_aur^T * e) over block n
      c_n = (F_hat * l) over block n
    h [L][P][n_h], f_true [P][L][n_t], f_hat0 [P][L][n_fb], s [P][T].
    Returns (l [L][nb*B], e [P][nb*B], canceller) with the final state.
    """
    synth = UpolsOracle(h, B)
    room = UpolsOracle(f_true, B)
    can = NlmsCanceller(f_hat0, B, mu, lam, delta)
    P = synth.Q
    if can.P != P or room.L != P or can.L != synth.L or room.Q != synth.L:
        raise ValueError("shape mismatch between H_aur [L][P], F [P][L], F_hat [P][L]")
    s = np.asarray(s, dtype=np.float64)
    T = s.shape[1]
    nb = -(-T // B) if n_blocks is None else int(n_blocks)
    sp = np.zeros((P, nb * B))
    n = min(T, nb * B)
    sp[:, :n] = s[:, :n]
    l_out = np.zeros((synth.L, nb * B))
    e_out = np.zeros((P, nb * B))
    fb_prev = np.zeros((P, B))
    c_prev = np.zeros((P, B))
    for b in range(nb):
        sl = slice(b * B, (b + 1) * B)
        e_n = sp[:, sl] + fb_prev - c_prev
        can.adapt(e_n)
        l_n = synth.process_block(e_n)
        c_prev = can.predict(l_n)
        fb_prev = room.process_block(l_n)
        l_out[:, sl] = l_n
        e_out[:, sl] = e_n
    return l_out, e_out, can

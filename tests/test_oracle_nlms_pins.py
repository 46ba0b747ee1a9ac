"""Pins of the FP64 adaptive-canceller oracle (``oracle.nlms_oracle``).

The update is an extension beyond the paper (readings R12-R14 in the oracle's
header), so the pins are mathematical facts about the recursion it states,
checked by means other than re-running it:

* mu = 0 reduces the adaptive closed loop to the static one of Sec. 5, which is
  itself pinned by brute force in ``test_oracle_pins``.
* The frequency-domain gradient conj(U_j) E is, after an inverse FFT, the
  circular cross-correlation of the zero-padded error block with the
  loudspeaker window of entry j, summed by explicit loops.
* NLMS a-posteriori property: with one partition, lambda = 0 and mu = 1, one
  update changes the canceller's output over the same block by exactly e
  (every bin's a-posteriori error vanishes, because the per-bin power is the
  sum over loudspeakers of |U|^2).
* Power recursion: with a loudspeaker signal that repeats every block, every
  window, and so every |U|^2, is the same, and after n blocks
  pow = (1 - lam^n) |U|^2 (geometric series).
* System identification in open loop (white loudspeaker noise, the
  microphone hears (F * l) one block later): the residual falls by > 15 dB,
  while planted mistakes (conjugate on E, error block at the front, delay line
  one entry off) make it grow.
"""

import numpy as np
import pytest

from oracle import UpolsOracle, afc_closed_loop, mimo_fir
from oracle.nlms_oracle import NlmsCanceller, afc_closed_loop_nlms


def _rand(seed, *shape):
    return np.random.default_rng(seed).standard_normal(shape)


def test_mu_zero_is_the_static_closed_loop():
    P, L, B = 2, 3, 16
    h = _rand(1, L, P, 70) * 0.3
    f = _rand(2, P, L, 40) * 0.05
    fh = f + _rand(3, P, L, 40) * 0.01
    s = _rand(4, P, 20 * B) * 0.1
    l0, e0, _ = afc_closed_loop(h, f, fh, s, B)
    l1, e1, _ = afc_closed_loop_nlms(h, f, fh, s, B, mu=0.0, lam=0.9, delta=1e-3)
    np.testing.assert_allclose(l1, l0, rtol=0, atol=1e-12)
    np.testing.assert_allclose(e1, e0, rtol=0, atol=1e-12)


def test_gradient_is_the_time_domain_cross_correlation():
    P, L, B, K = 2, 2, 8, 3
    can = NlmsCanceller(np.zeros((P, L, K * B)), B, mu=0.5, lam=0.5, delta=1e-3)
    lsig = _rand(5, L, 6 * B)
    windows = []
    for n in range(6):
        can.predict(lsig[:, n * B : (n + 1) * B])
        prev = lsig[:, (n - 1) * B : n * B] if n > 0 else np.zeros((L, B))
        windows.append(np.concatenate([prev, lsig[:, n * B : (n + 1) * B]], axis=1))
    e = _rand(6, P, B)
    G = can.gradient(e)  # [P][L][K][B+1]
    N = 2 * B
    for p in range(P):
        epad = np.concatenate([np.zeros(B), e[p]])
        for l in range(L):
            for j in range(K):
                w = windows[5 - j][l]  # delay-line entry j = window of the block j blocks back
                # circular cross-correlation by explicit sums: r[tau] = sum_t epad[t] w[(t - tau) mod N]
                r = np.zeros(N)
                for tau in range(N):
                    acc = 0.0
                    for t in range(N):
                        acc += epad[t] * w[(t - tau) % N]
                    r[tau] = acc
                # the inverse FFT (1/N scaled) of conj(U) E is the correlation itself
                got = np.fft.irfft(G[p, l, j], n=N)
                np.testing.assert_allclose(got, r, rtol=0, atol=1e-10)


def test_a_posteriori_error_vanishes_for_one_partition():
    P, L, B = 2, 3, 16
    f0 = _rand(7, P, L, B) * 0.1
    can = NlmsCanceller(f0, B, mu=1.0, lam=0.0, delta=0.0)
    lsig = _rand(8, L, 4 * B)
    for n in range(4):
        can.predict(lsig[:, n * B : (n + 1) * B])
    U = can.fdl[0]  # [L][B+1]
    before = (can.W[:, :, 0, :] * U[None]).sum(axis=1)
    e = _rand(9, P, B)
    can.adapt(e)
    after = (can.W[:, :, 0, :] * U[None]).sum(axis=1)
    change = np.fft.irfft(after - before, n=2 * B, axis=-1)
    np.testing.assert_allclose(change[:, :B], 0.0, atol=1e-12)
    np.testing.assert_allclose(change[:, B:], e, atol=1e-12)


def test_power_recursion_is_a_geometric_series():
    P, L, B, lam = 1, 3, 16, 0.7
    can = NlmsCanceller(np.zeros((P, L, 2 * B)), B, mu=0.1, lam=lam, delta=1.0)
    blk = _rand(10, L, B)
    win = np.concatenate([blk, blk], axis=1)
    u2 = np.sum(np.abs(np.fft.rfft(win, axis=-1)) ** 2, axis=0)
    can.predict(blk)  # from here on every window is [blk | blk]
    for n in range(1, 8):
        can.predict(blk)
        can.adapt(np.zeros((P, B)))
        np.testing.assert_allclose(can.power, (1.0 - lam**n) * u2, rtol=1e-12)


class _ConjOnError(NlmsCanceller):
    def gradient(self, e):
        E = self.error_spectrum(e)
        return np.conj(E)[:, None, None, :] * self.fdl.transpose(1, 0, 2)[None]


class _ErrorAtFront(NlmsCanceller):
    def error_spectrum(self, e):
        pad = np.zeros((self.P, self.n_f))
        pad[:, : self.B] = e
        return np.fft.rfft(pad, axis=-1)


class _DelayLineOffByOne(NlmsCanceller):
    def gradient(self, e):
        E = self.error_spectrum(e)
        shifted = np.zeros_like(self.fdl)
        shifted[1:] = self.fdl[:-1]
        return E[:, None, None, :] * np.conj(shifted.transpose(1, 0, 2))[None]


def _identify(cls, blocks=300):
    rng = np.random.default_rng(0)
    P, L, B, K = 2, 3, 32, 4
    F = rng.standard_normal((P, L, K * B)) * np.exp(-np.arange(K * B) / 40.0) * 0.3
    lsig = rng.standard_normal((L, blocks * B))
    d = mimo_fir(F, lsig)
    can = cls(np.zeros_like(F), B, 0.5, 0.9, 1e-6)
    c_prev = np.zeros((P, B))
    ratio = []
    for n in range(blocks):
        if n > 0:
            dn = d[:, (n - 1) * B : n * B]
            e = dn - c_prev
            can.adapt(e)
            ratio.append(np.sum(e**2) / np.sum(dn**2))
        c_prev = can.predict(lsig[:, n * B : (n + 1) * B])
    return 10 * np.log10(np.mean(ratio[-50:]))


def test_open_loop_identification_converges():
    assert _identify(NlmsCanceller) < -15.0


@pytest.mark.parametrize("cls", [_ConjOnError, _ErrorAtFront, _DelayLineOffByOne])
def test_planted_mistakes_do_not_converge(cls):
    assert _identify(cls, blocks=120) > 0.0


# ---------------------------------------------- step order of the closed loop


def _circ_conv(a, b):
    """(a (*) b)[t] = sum_tau a[tau] b[(t - tau) mod N], explicit loops."""
    N = len(a)
    return np.array([sum(a[tau] * b[(t - tau) % N] for tau in range(N)) for t in range(N)])


def _circ_xcorr(e, w):
    """r[tau] = sum_t e[t] w[(t - tau) mod N], explicit loops (the time-domain
    form of E conj(U), pinned above)."""
    N = len(e)
    return np.array([sum(e[t] * w[(t - tau) % N] for t in range(N)) for tau in range(N)])


def _two_block_case():
    """One microphone, two loudspeakers, B = 4, identity-like synthesis (l_1 = e,
    l_2 = 2e), a two-partition estimate, and a first block that is a single
    impulse: the loudspeaker window of block 0 is then an impulse too, so every
    bin of sum_l |U_0|^2 is the same and the normalised step is one number."""
    B = 4
    h = np.zeros((2, 1, 1))
    h[0, 0, 0], h[1, 0, 0] = 1.0, 2.0
    fh0 = _rand(21, 1, 2, 2 * B) * 0.3
    a, t0 = 0.7, 1
    s = np.zeros((1, 3 * B))
    s[0, t0] = a
    s[0, B:] = _rand(22, 2 * B) * 0.5
    return B, h, fh0, s, a, t0


def _hand_prediction_block1(B, h, fh0, s, mu, lam, delta, a):
    """c_1 (the prediction subtracted from block 2) of the loop with the step
    taken after e_1 is known and before l_1 enters the delay line, by hand:
      block 0: e_0 = s_0, l_0 = h * e_0, no step (empty delay line), c_0 = f_hat * l_0
      block 1: e_1 = s_1 - c_0; pow = (1 - lam) sum_l |U_0|^2 = (1 - lam) 5 a^2
               (flat); w_1 = w_0 + mu / (K pow + delta) * xcorr([0 | e_1], window_0)
               on sub-filter 0 only (the delay line has no entry 1 yet);
               l_1 = h * e_1; c_1 = last B samples of
               sum_l  w_1[l][0] (*) [l_0 | l_1]  +  w_1[l][1] (*) [0 | l_0]."""
    N, K, L = 2 * B, 2, 2
    gain = h[:, 0, 0]
    e0 = s[0, :B]
    l0 = [gain[l] * e0 for l in range(L)]
    # c_0: the static estimate over block 0 (direct convolution, zero history)
    c0 = np.array([sum(fh0[0, l, j] * l0[l][t - j] for l in range(L) for j in range(t + 1)) for t in range(B)])
    e1 = s[0, B : 2 * B] - c0
    l1 = [gain[l] * e1 for l in range(L)]
    win0 = [np.concatenate([np.zeros(B), l0[l]]) for l in range(L)]
    win1 = [np.concatenate([l0[l], l1[l]]) for l in range(L)]
    step = mu / (K * (1.0 - lam) * (1.0 + 4.0) * a * a + delta)
    epad = np.concatenate([np.zeros(B), e1])
    c1 = np.zeros(N)
    for l in range(L):
        w_0 = np.concatenate([fh0[0, l, :B], np.zeros(B)]) + step * _circ_xcorr(epad, win0[l])
        w_1 = np.concatenate([fh0[0, l, B:], np.zeros(B)])
        c1 += _circ_conv(w_0, win1[l]) + _circ_conv(w_1, win0[l])
    return e1, c1[B:]


def _loop_adapt_after_predict(h, fh0, s, B, mu, lam, delta):
    """Planted: the step of block n comes after c_n is formed."""
    synth, can = UpolsOracle(h, B), NlmsCanceller(fh0, B, mu, lam, delta)
    c_prev, out = np.zeros((1, B)), []
    for b in range(s.shape[1] // B):
        e_n = s[:, b * B : (b + 1) * B] - c_prev
        l_n = synth.process_block(e_n)
        c_prev = can.predict(l_n)
        can.adapt(e_n)
        out.append(e_n)
    return np.concatenate(out, axis=1)


def _loop_adapt_after_push(h, fh0, s, B, mu, lam, delta):
    """Planted: l_n enters the delay line before the step, so the step
    correlates e_n with the window of block n instead of block n-1."""
    synth, can = UpolsOracle(h, B), NlmsCanceller(fh0, B, mu, lam, delta)
    c_prev, out = np.zeros((1, B)), []
    for b in range(s.shape[1] // B):
        e_n = s[:, b * B : (b + 1) * B] - c_prev
        l_n = synth.process_block(e_n)
        can.predict(l_n)  # push l_n (the prediction it returns uses the old estimate)
        can.adapt(e_n)
        acc = np.zeros((can.P, B + 1), dtype=np.complex128)
        for j in range(can.K):
            acc += (can.W[:, :, j, :] * can.fdl[j][None, :, :]).sum(axis=1)
        c_prev = np.fft.irfft(acc, n=2 * B, axis=-1)[:, B:]
        out.append(e_n)
    return np.concatenate(out, axis=1)


def test_closed_loop_step_order_two_blocks():
    """afc_closed_loop_nlms takes block n's step with e_n before l_n enters the
    delay line, and predicts c_n with the updated estimate: its e_2 = s_2 - c_1
    equals the hand computation, while loops with the step after the
    prediction, or after the push, do not."""
    B, h, fh0, s, a, _ = _two_block_case()
    mu, lam, delta = 0.6, 0.5, 1e-3
    e1, c1 = _hand_prediction_block1(B, h, fh0, s, mu, lam, delta, a)
    _, e_ref, _ = afc_closed_loop_nlms(h, np.zeros((1, 2, 1)), fh0, s, B, mu, lam, delta)
    np.testing.assert_allclose(e_ref[0, B : 2 * B], e1, rtol=0, atol=1e-12)
    np.testing.assert_allclose(e_ref[0, 2 * B :], s[0, 2 * B :] - c1, rtol=0, atol=1e-12)
    for planted in (_loop_adapt_after_predict, _loop_adapt_after_push):
        e_bad = planted(h, fh0, s, B, mu, lam, delta)
        hand = np.concatenate([e1, s[0, 2 * B :] - c1])
        assert np.max(np.abs(e_bad[0, B:] - hand)) > 1e-3

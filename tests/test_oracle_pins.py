"""Pins for the FP64 oracle against things other than itself (CPU only).

Each pin is chosen so that a plausible mistake in the oracle (a dropped
sub-filter, a reversed or unshifted frequency-domain delay line, the wrong
overlap-save half, transposed channel indices, the wrong block of the feedback
prediction) fails at least one of them; ``test_planted_*`` plants exactly those
mistakes in copies of the oracle and checks that the pins catch them.
"""

import numpy as np
import pytest

from oracle import UpolsOracle, afc_closed_loop, mimo_fir, mimo_fir_sample, num_partitions, upols
from paper_2509_04390_gb300 import signals


# ----------------------------------------------------------------- helpers


def brute_mimo(h, x):
    """Direct time-domain MIMO convolution with plain Python loops (Eq. 4)."""
    L, Q, n_h = h.shape
    T = x.shape[1]
    hl = h.tolist()
    xl = x.tolist()
    y = np.zeros((L, T))
    for l in range(L):
        for t in range(T):
            acc = 0.0
            for q in range(Q):
                for j in range(min(n_h, t + 1)):
                    acc += hl[l][q][j] * xl[q][t - j]
            y[l, t] = acc
    return y


def brute_closed_loop(h, f, fh, s, B):
    """Sample-by-sample closed loop: m[t] = s[t] + (F*l)[t-B], c[t] = (F_hat*l)[t-B],
    e = m - c, l = H^T * e (Eqs. 1-3 with the one-block delay of Sec. 5)."""
    L, P, n_h = h.shape
    T = s.shape[1]
    lsig = np.zeros((L, T))
    e = np.zeros((P, T))
    m = np.zeros((P, T))
    for t in range(T):
        for p in range(P):
            fb = 0.0
            ch = 0.0
            u = t - B
            for l in range(L):
                for j in range(f.shape[2]):
                    if u - j >= 0:
                        fb += f[p, l, j] * lsig[l, u - j]
                for j in range(fh.shape[2]):
                    if u - j >= 0:
                        ch += fh[p, l, j] * lsig[l, u - j]
            m[p, t] = s[p, t] + fb
            e[p, t] = m[p, t] - ch
        for l in range(L):
            acc = 0.0
            for q in range(P):
                for j in range(min(n_h, t + 1)):
                    acc += h[l, q, j] * e[q, t - j]
            lsig[l, t] = acc
    return lsig, e, m


def rel_err(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


# ------------------------------------------------------ closed-form pins


def test_hand_computed_single_channel():
    # Eq. 4 by hand: h = [1, 2, 3], x = [1, 0, -1, 2]
    # y0 = 1*1 = 1; y1 = 1*0 + 2*1 = 2; y2 = 1*(-1) + 2*0 + 3*1 = 2
    # y3 = 1*2 + 2*(-1) + 3*0 = 0; y4 = 2*2 + 3*(-1) = 1; y5 = 3*2 = 6
    h = np.array([[[1.0, 2.0, 3.0]]])
    x = np.array([[1.0, 0.0, -1.0, 2.0, 0.0, 0.0]])
    want = np.array([[1.0, 2.0, 2.0, 0.0, 1.0, 6.0]])
    np.testing.assert_allclose(mimo_fir(h, x), want, atol=1e-15)
    # B = 2 -> K = 2 sub-filters ([1,2], [3,0]); three blocks of streaming
    np.testing.assert_allclose(upols(h, x, 2), want, atol=1e-13)


def test_hand_computed_mimo():
    # Eq. 2: output 0 = h00 * x0 + h01 * x1 with h00 = [1,2,3], h01 = [0,-1],
    # x0 = [1,0,-1,2], x1 = [2,1,0,0]:  h01 * x1 = [0,-2,-1,0,0]
    # -> [1,2,2,0,1,6] + [0,-2,-1,0,0,0] = [1,0,1,0,1,6]
    h = np.zeros((1, 2, 3))
    h[0, 0] = [1, 2, 3]
    h[0, 1] = [0, -1, 0]
    x = np.array([[1.0, 0, -1, 2, 0, 0], [2.0, 1, 0, 0, 0, 0]])
    want = np.array([[1.0, 0, 1, 0, 1, 6]])
    np.testing.assert_allclose(mimo_fir(h, x), want, atol=1e-15)
    for B in (1, 2, 3, 4):
        np.testing.assert_allclose(upols(h, x, B)[:, :6], want, atol=1e-13)


def test_num_partitions():
    assert num_partitions(48000, 256) == 188  # 187.5 -> 188, last zero-padded
    assert num_partitions(384000, 256) == 1500
    assert num_partitions(384000, 128) == 3000
    assert num_partitions(24000, 256) == 94
    assert num_partitions(256, 256) == 1
    assert num_partitions(257, 256) == 2


# ---------------------------------------------------- brute-force pins


@pytest.mark.parametrize(
    "L,Q,n_h,B,nb",
    [
        (3, 2, 37, 8, 9),  # ragged last partition, L != Q
        (2, 3, 16, 16, 4),  # n_h == B -> K = 1
        (1, 1, 48, 16, 6),  # n_h == K*B exactly
        (2, 2, 49, 16, 6),  # K*B + 1
        (2, 1, 47, 16, 6),  # K*B - 1
        (1, 2, 5, 16, 3),  # filter shorter than a block
    ],
)
def test_upols_matches_bruteforce(L, Q, n_h, B, nb):
    rng = np.random.default_rng(100 + n_h)
    h = rng.standard_normal((L, Q, n_h))
    x = rng.standard_normal((Q, B * nb))
    want = brute_mimo(h, x)
    got = upols(h, x, B)
    assert rel_err(got, want) < 1e-13
    np.testing.assert_allclose(mimo_fir(h, x), want, rtol=0, atol=1e-12)


def test_mimo_fir_sample_matches_definition():
    rng = np.random.default_rng(7)
    h = rng.standard_normal((3, 2, 50))
    x = rng.standard_normal((2, 120))
    y = brute_mimo(h, x)
    for l, t in [(0, 0), (1, 3), (2, 49), (0, 50), (1, 119), (2, 77)]:
        assert abs(mimo_fir_sample(h, x, l, t) - y[l, t]) < 1e-12


# -------------------------------------------------------- invariants


def test_dirac_input_returns_filter():
    rng = np.random.default_rng(11)
    B = 32
    h = rng.standard_normal((2, 1, 150))
    x = np.zeros((1, B * 6))
    x[0, 0] = 1.0
    y = upols(h, x, B)
    np.testing.assert_allclose(y[:, :150], h[:, 0, :], atol=1e-13)
    np.testing.assert_allclose(y[:, 150:], 0.0, atol=1e-13)


def test_identity_filter_passes_input():
    rng = np.random.default_rng(12)
    B = 16
    h = np.zeros((2, 2, 40))
    h[0, 0, 0] = 1.0
    h[1, 1, 0] = 1.0
    x = rng.standard_normal((2, B * 7))
    y = upols(h, x, B)
    np.testing.assert_allclose(y, x, atol=1e-13)


def test_pure_delay_filter_shifts_across_partitions():
    # h = delta[t - d] with d in a later sub-filter: y[t] = x[t - d]
    rng = np.random.default_rng(13)
    B = 16
    for d in (15, 16, 17, 47, 63):
        h = np.zeros((1, 1, 64))
        h[0, 0, d] = 1.0
        x = rng.standard_normal((1, B * 8))
        y = upols(h, x, B)
        np.testing.assert_allclose(y[0, d:], x[0, : B * 8 - d], atol=1e-13)
        np.testing.assert_allclose(y[0, :d], 0.0, atol=1e-13)


def test_linearity():
    rng = np.random.default_rng(14)
    B = 32
    h = rng.standard_normal((3, 2, 100))
    a = rng.standard_normal((2, B * 5))
    b = rng.standard_normal((2, B * 5))
    ya, yb = upols(h, a, B), upols(h, b, B)
    yab = upols(h, 2.5 * a - 0.75 * b, B)
    assert rel_err(yab, 2.5 * ya - 0.75 * yb) < 1e-13


def test_time_invariance_by_whole_blocks():
    rng = np.random.default_rng(15)
    B = 16
    h = rng.standard_normal((2, 2, 70))
    x = rng.standard_normal((2, B * 6))
    xs = np.concatenate([np.zeros((2, 2 * B)), x], axis=1)
    y = upols(h, x, B)
    ys = upols(h, xs, B)
    np.testing.assert_allclose(ys[:, 2 * B :], y, atol=1e-12)
    np.testing.assert_allclose(ys[:, : 2 * B], 0.0, atol=1e-13)


def test_streaming_equals_whole_signal_fft_convolution():
    # Eq. 5 over the whole signal with n_f >= n_h + n_x - 1 (a single FFT block):
    # block streaming must reach the same linear convolution.
    w = signals.plain_1x2()
    h = w.h.astype(np.float64)
    x = w.x.astype(np.float64)
    T = x.shape[1]
    n = 1 << int(np.ceil(np.log2(T + h.shape[2])))
    whole = np.fft.irfft(np.fft.rfft(h[:, 0, :], n) * np.fft.rfft(x[0], n)[None, :], n)[:, :T]
    got = upols(h, x, w.block)[:, :T]
    assert rel_err(got, whole) < 1e-12


def test_upols_matches_np_convolve_paper_shape_reduced():
    # 4 inputs x 16 outputs with paper-style filters (reduced taps), library direct convolution
    w = signals.paper_4x16(block=128, seconds=0.1, taps=3000)
    h = w.h.astype(np.float64)
    x = w.x.astype(np.float64)
    want = mimo_fir(h, x)
    got = upols(h, x, w.block)[:, : x.shape[1]]
    assert rel_err(got, want) < 1e-12


# ------------------------------------------------------- feedback loop


def _afc_case(seed, P=2, L=3, n_h=40, n_f=20, B=16, nb=8, gain=0.3):
    rng = np.random.default_rng(seed)
    h = rng.standard_normal((L, P, n_h)) * 0.3
    f = rng.standard_normal((P, L, n_f)) * gain / np.sqrt(n_f)
    s = rng.standard_normal((P, B * nb))
    return h, f, s, B


def test_afc_matches_sample_by_sample_simulation():
    h, f, s, B = _afc_case(21)
    fh = f * 0.6  # imperfect estimate: residual feedback recirculates
    want_l, want_e, want_m = brute_closed_loop(h, f, fh, s, B)
    l, e, m = afc_closed_loop(h, f, fh, s, B)
    assert rel_err(l, want_l) < 1e-12
    assert rel_err(e, want_e) < 1e-12
    assert rel_err(m, want_m) < 1e-12


def test_afc_perfect_estimate_cancels_feedback():
    # with F_hat = F the error signal is the dry source and the output is open-loop synthesis
    h, f, s, B = _afc_case(22, gain=0.8)
    l, e, m = afc_closed_loop(h, f, f, s, B)
    np.testing.assert_allclose(e, s, atol=1e-12)
    assert rel_err(l, upols(h, s, B)) < 1e-12
    assert rel_err(m, s) > 1e-3  # the feedback really was there


def test_afc_without_feedback_reduces_to_synthesis():
    h, f, s, B = _afc_case(23)
    zero = np.zeros_like(f)
    l, e, m = afc_closed_loop(h, zero, zero, s, B)
    assert rel_err(l, upols(h, s, B)) < 1e-14
    np.testing.assert_array_equal(e, s)


# ------------------------------------------- planted mistakes are caught


class _NoShift(UpolsOracle):
    def process_block(self, x_n):  # FDL never shifted: all sub-filters meet the newest spectrum
        self.window[:, : self.B] = self.window[:, self.B :]
        self.window[:, self.B :] = x_n
        xb = np.fft.rfft(self.window, axis=-1)
        acc = sum((self.h_bar[:, :, k, :] * xb[None]).sum(axis=1) for k in range(self.K))
        return np.fft.irfft(acc, n=self.n_f, axis=-1)[:, self.B :]


class _Reversed(UpolsOracle):
    def process_block(self, x_n):  # newest spectrum meets the LAST sub-filter
        self.window[:, : self.B] = self.window[:, self.B :]
        self.window[:, self.B :] = x_n
        self.fdl[1:] = self.fdl[:-1].copy()
        self.fdl[0] = np.fft.rfft(self.window, axis=-1)
        acc = sum((self.h_bar[:, :, k, :] * self.fdl[self.K - 1 - k][None]).sum(axis=1) for k in range(self.K))
        return np.fft.irfft(acc, n=self.n_f, axis=-1)[:, self.B :]


class _FirstHalf(UpolsOracle):
    def process_block(self, x_n):  # keeps the aliased first half instead of the last n_x samples
        self.window[:, : self.B] = self.window[:, self.B :]
        self.window[:, self.B :] = x_n
        self.fdl[1:] = self.fdl[:-1].copy()
        self.fdl[0] = np.fft.rfft(self.window, axis=-1)
        acc = sum((self.h_bar[:, :, k, :] * self.fdl[k][None]).sum(axis=1) for k in range(self.K))
        return np.fft.irfft(acc, n=self.n_f, axis=-1)[:, : self.B]


class _DropLast(UpolsOracle):
    def __init__(self, h, B):
        super().__init__(h, B)
        self.h_bar[:, :, -1, :] = 0.0  # last (ragged) sub-filter dropped


def _run(cls, h, x, B):
    eng = cls(h, B)
    return np.concatenate([eng.process_block(x[:, i * B : (i + 1) * B]) for i in range(x.shape[1] // B)], axis=1)


@pytest.mark.parametrize("cls", [_NoShift, _Reversed, _FirstHalf, _DropLast])
def test_planted_upols_mistakes_fail_bruteforce(cls):
    rng = np.random.default_rng(31)
    B = 8
    h = rng.standard_normal((3, 2, 37))
    x = rng.standard_normal((2, B * 8))
    want = brute_mimo(h, x)
    assert rel_err(_run(UpolsOracle, h, x, B), want) < 1e-13
    assert rel_err(_run(cls, h, x, B), want) > 1e-3


def test_planted_transposed_filters_fail_bruteforce():
    rng = np.random.default_rng(32)
    B = 8
    h = rng.standard_normal((2, 2, 20))
    x = rng.standard_normal((2, B * 5))
    want = brute_mimo(h, x)
    assert rel_err(upols(h.transpose(1, 0, 2).copy(), x, B), want) > 1e-3


def _afc_lagged(h, f, fh, s, B, lag):
    """Copy of the oracle's loop subtracting the prediction from ``lag`` blocks back."""
    synth, canc, room = UpolsOracle(h, B), UpolsOracle(fh, B), UpolsOracle(f, B)
    P = s.shape[0]
    nb = s.shape[1] // B
    hist = [np.zeros((P, B))] * (lag + 1)
    fb_prev = np.zeros((P, B))
    out = []
    for b in range(nb):
        m_n = s[:, b * B : (b + 1) * B] + fb_prev
        e_n = m_n - (hist[-lag] if lag > 0 else 0.0)
        l_n = synth.process_block(e_n)
        hist.append(canc.process_block(l_n))
        fb_prev = room.process_block(l_n)
        out.append(l_n)
    return np.concatenate(out, axis=1)


def test_planted_wrong_prediction_block_fails_simulation():
    h, f, s, B = _afc_case(33)
    fh = f * 0.6
    want_l, _, _ = brute_closed_loop(h, f, fh, s, B)
    assert rel_err(_afc_lagged(h, f, fh, s, B, 1), want_l) < 1e-12  # the correct timing
    assert rel_err(_afc_lagged(h, f, fh, s, B, 2), want_l) > 1e-3  # c_{n-2}
    assert rel_err(_afc_lagged(h, f, fh, s, B, 0), want_l) > 1e-3  # no cancellation

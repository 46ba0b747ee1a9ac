"""Pins of the oracle's spectrum-reuse closed loop (the remark closing Sec. 5:
the synthesis output spectra feed the canceller directly, with n_f = 3 n_x).

The pins are facts the mathematics fixes, checked by means other than the
oracle's own loop:

* UPOLS with n_f = 3 n_x equals direct time-domain convolution (brute force).
* The synthesis accumulated spectrum Y_n, inverse-transformed, holds
  [l_{n-1}, l_n] in its last 2 n_x samples (brute force): the property that
  lets the canceller take it as its input spectrum.
* The reuse loop equals the sample-by-sample closed loop of Eqs. 1-3 with the
  one-block delay of Sec. 5, for an imperfect estimate (the residual feedback
  recirculates), and so also equals the n_f = 2 n_x loop.
* Planted mistakes fail: reusing spectra of 2 n_x windows (whose first half is
  wrap-around), keeping the wrong third of the canceller's output, and feeding
  the canceller the previous block's spectrum.
"""

import numpy as np
import pytest

from oracle import UpolsOracle, afc_closed_loop, afc_closed_loop_reuse
from test_oracle_pins import _afc_case, brute_closed_loop, brute_mimo, rel_err


@pytest.mark.parametrize("L,Q,n_h,B,nb", [(2, 3, 37, 8, 7), (1, 1, 16, 16, 4), (3, 2, 5, 4, 9), (2, 2, 64, 8, 9)])
def test_upols_three_nx_matches_bruteforce(L, Q, n_h, B, nb):
    rng = np.random.default_rng(41 + n_h)
    h = rng.standard_normal((L, Q, n_h))
    x = rng.standard_normal((Q, B * nb))
    eng = UpolsOracle(h, B, n_f=3 * B)
    assert eng.bins == 3 * B // 2 + 1
    got = np.concatenate([eng.process_block(x[:, i * B : (i + 1) * B]) for i in range(nb)], axis=1)
    assert rel_err(got, brute_mimo(h, x)) < 1e-13


def test_upols_rejects_fft_shorter_than_two_blocks():
    with pytest.raises(ValueError):
        UpolsOracle(np.ones((1, 1, 8)), 8, n_f=15)


def test_synthesis_spectrum_holds_two_output_blocks():
    rng = np.random.default_rng(42)
    B, nb = 8, 7
    h = rng.standard_normal((2, 3, 29))
    x = rng.standard_normal((3, B * nb))
    want = brute_mimo(h, x)
    eng = UpolsOracle(h, B, n_f=3 * B)
    for n in range(nb):
        Y = eng.accumulate(eng.transform_input(x[:, n * B : (n + 1) * B]))
        y = np.fft.irfft(Y, n=3 * B, axis=-1)
        lo = max(0, (n - 1) * B)
        np.testing.assert_allclose(y[:, 3 * B - ((n + 1) * B - lo) :], want[:, lo : (n + 1) * B], atol=1e-12)
        if n >= 2:
            # the first n_x samples are wrap-around, not l_{n-2}
            assert np.max(np.abs(y[:, :B] - want[:, (n - 2) * B : (n - 1) * B])) > 1e-3


def test_reuse_loop_matches_sample_by_sample_simulation():
    h, f, s, B = _afc_case(43)
    fh = f * 0.6
    want_l, want_e, want_m = brute_closed_loop(h, f, fh, s, B)
    l, e, m = afc_closed_loop_reuse(h, f, fh, s, B)
    assert rel_err(l, want_l) < 1e-12
    assert rel_err(e, want_e) < 1e-12
    assert rel_err(m, want_m) < 1e-12


def test_reuse_loop_equals_the_two_nx_loop():
    rng = np.random.default_rng(44)
    B, nb = 16, 12
    h = rng.standard_normal((3, 2, 70)) * 0.3
    f = rng.standard_normal((2, 3, 40)) * 0.2 / np.sqrt(40)
    s = rng.standard_normal((2, B * nb))
    fh = f * 0.7
    a = afc_closed_loop(h, f, fh, s, B)
    b = afc_closed_loop_reuse(h, f, fh, s, B)
    for u, v in zip(a, b):
        assert rel_err(v, u) < 1e-12


def _reuse_variant(h, f, fh, s, B, n_f, keep=None, lag=0):
    """Copy of the reuse loop with a plantable FFT size, kept segment of the
    canceller's output, and lag of the spectrum entering the canceller."""
    synth, canc, room = UpolsOracle(h, B, n_f=n_f), UpolsOracle(fh, B, n_f=n_f), UpolsOracle(f, B)
    P = s.shape[0]
    nb = s.shape[1] // B
    fb_prev = np.zeros((P, B))
    c_prev = np.zeros((P, B))
    hist = [np.zeros((synth.L, synth.bins), dtype=np.complex128)] * (lag + 1)
    out = []
    for b in range(nb):
        e_n = s[:, b * B : (b + 1) * B] + fb_prev - c_prev
        Y = synth.accumulate(synth.transform_input(e_n))
        l_n = synth.transform_output(Y)
        hist.append(Y)
        C = canc.accumulate(hist[-1 - lag])
        y = np.fft.irfft(C, n=n_f, axis=-1)
        k0 = n_f - B if keep is None else keep
        c_prev = y[:, k0 : k0 + B]
        fb_prev = room.process_block(l_n)
        out.append(l_n)
    return np.concatenate(out, axis=1)


def test_planted_reuse_mistakes_fail_simulation():
    h, f, s, B = _afc_case(45)
    fh = f * 0.6
    want_l, _, _ = brute_closed_loop(h, f, fh, s, B)
    assert rel_err(_reuse_variant(h, f, fh, s, B, 3 * B), want_l) < 1e-12  # the correct loop
    assert rel_err(_reuse_variant(h, f, fh, s, B, 2 * B), want_l) > 1e-3  # 2 n_x windows reused
    assert rel_err(_reuse_variant(h, f, fh, s, B, 3 * B, keep=B), want_l) > 1e-3  # middle third kept
    assert rel_err(_reuse_variant(h, f, fh, s, B, 3 * B, lag=1), want_l) > 1e-3  # previous block's spectrum

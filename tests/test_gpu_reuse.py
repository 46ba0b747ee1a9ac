"""GPU parity of the spectrum-reuse form (n_f = 3 n_x, the remark closing
Sec. 5) against the FP64 oracle: the plain convolution at n_f = 3 n_x, and the
closed loop in which the synthesis output spectrum enters the canceller's
delay line as it is (``oracle.afc_closed_loop_reuse``), stage by stage.

Both are the same mathematics as the n_f = 2 n_x form; the bounds are the
same (FP32 120 dB, FP16 60 dB, BF16 42 dB).
"""

from __future__ import annotations

import os

import numpy as np
import pytest

from gpu_helpers import (
    RoomPlant,
    cancellation_gain_db,
    check_replay,
    sample_points,
    shift_blocks,
    snr_db,
    snr_per_channel_db,
)
from oracle import UpolsOracle, afc_closed_loop_reuse, mimo_fir_sample
from paper_2509_04390_gb300 import build, signals
from paper_2509_04390_gb300 import upols as U

pytestmark = pytest.mark.gpu

FP32_DB = 120.0
FP32_CH_DB = 115.0
BOUND = {"fp32": FP32_DB, "fp16": 60.0, "bf16": 42.0}


@pytest.fixture(scope="module", autouse=True)
def engine_lib():
    if not os.path.exists(build.lib_path()):
        build.build()
    U.load()


def oracle3(h, x, B):
    """The oracle's UPOLS at n_f = 3 n_x over whole blocks of x."""
    eng = UpolsOracle(np.asarray(h, np.float64), B, n_f=3 * B)
    nb = x.shape[1] // B
    x = np.asarray(x, np.float64)
    return np.concatenate([eng.process_block(x[:, i * B : (i + 1) * B]) for i in range(nb)], axis=1)


def run_reuse(w, precision="fp32", tiling=None):
    with U.Engine(w.fs, w.block, w.n_in, w.n_out, w.taps, precision, tiling, reuse=True) as e:
        assert e.info()["fft_size"] == 3 * w.block
        e.set_filters(w.h)
        return e.run(w.x)


# ------------------------------------------------------- plain convolution


@pytest.mark.parametrize("B", [32, 64, 128, 256, 512, 1024, 2048, 4096])
def test_identity_filter_every_block_size(B):
    # h = delta: output = input, every 3 n_x FFT size (radix 3, then an odd or even count of radix-2 factors)
    rng = np.random.default_rng(B)
    h = np.zeros((2, 2, 3 * B + 5), dtype=np.float32)
    h[0, 0, 0] = 1.0
    h[1, 1, 0] = 1.0
    x = rng.standard_normal((2, 6 * B)).astype(np.float32)
    with U.Engine(48000, B, 2, 2, h.shape[2], reuse=True) as e:
        e.set_filters(h)
        y = e.run(x)
    assert snr_db(y, x) >= FP32_DB
    np.testing.assert_allclose(y, x, atol=2e-6)


@pytest.mark.parametrize(
    "n_in,n_out,taps,B,nb",
    [
        (2, 3, 37, 32, 8),  # ragged last partition, K = 2
        (3, 20, 1000, 64, 24),  # two output tiles, the second ragged
        (2, 5, 4000, 512, 12),  # several bin tiles of 768 / 2 bins
        (1, 2, 9000, 4096, 5),  # K = 3 at the largest block
        (5, 7, 2048, 128, 30),  # K = 16 exactly
        (4, 33, 3000, 32, 100),  # three output tiles, many partitions per split
    ],
)
def test_random_shapes_fp32(n_in, n_out, taps, B, nb):
    w = signals.random_case(2000 + taps, n_in, n_out, taps, B, nb)
    y = run_reuse(w)
    ref = oracle3(w.h, w.x, B)
    assert snr_db(y, ref) >= FP32_DB
    assert min(snr_per_channel_db(y, ref)) >= FP32_CH_DB


@pytest.mark.parametrize("precision", ["fp16", "bf16"])
@pytest.mark.parametrize("n_in,n_out,taps,B,nb", [(3, 20, 2500, 64, 40), (2, 5, 9000, 256, 40)])
def test_random_shapes_reduced_precision(precision, n_in, n_out, taps, B, nb):
    w = signals.random_case(3000 + taps, n_in, n_out, taps, B, nb)
    y = run_reuse(w, precision)
    assert snr_db(y, oracle3(w.h, w.x, B)) >= BOUND[precision]


TILINGS = [
    {"kernel": "tma", "bin_tile": 16},
    {"kernel": "tma", "bin_tile": 64, "stages": 4, "stage_kib": 16},
    {"kernel": "tma", "bin_tile": 128, "splits": 3},
    {"kernel": "tma", "order": "interleaved"},
    {"kernel": "tma", "warps": 16},
    {"kernel": "direct1"},
    {"kernel": "direct2", "bin_tile": 32},
]


@pytest.mark.parametrize("tiling", TILINGS, ids=lambda t: "-".join(f"{k}{v}" for k, v in t.items()))
def test_mac_tilings(tiling):
    w = signals.random_case(4001, 2, 5, 9000, 256, 30)
    y = run_reuse(w, "fp32", tiling)
    assert snr_db(y, oracle3(w.h, w.x, 256)) >= FP32_DB


def test_bin_tile_that_does_not_divide_the_bins_is_rejected():
    # 3B/2 = 384 bins at B = 256: a 256-bin tile does not divide them
    with U.Engine(48000, 256, 1, 2, 2000) as e:
        U.conv_set_tiling(e.h, kernel="tma", bin_tile=256)
        with pytest.raises(U.ConvError) as ei:
            U.afc_set_spectrum_reuse(e.h, True)
        assert ei.value.code == U.CONV_E_INVAL
        # the engine keeps its n_f = 2 n_x plan and still works
        assert e.info()["fft_size"] == 512
        e.set_filters(np.ones((2, 1, 2000), np.float32) * 1e-3)
        e.process(np.zeros((1, 256), np.float32))


def test_multi_block_call_and_reset_are_bit_exact():
    w = signals.random_case(4002, 2, 3, 700, 64, 20)
    with U.Engine(w.fs, w.block, w.n_in, w.n_out, w.taps, reuse=True) as e:
        e.set_filters(w.h)
        a = e.run(w.x)
        e.reset()
        b = e.run(w.x)
        e.reset()
        c = e.render(w.x)
    np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(a, c)
    assert snr_db(a, oracle3(w.h, w.x, w.block)) >= FP32_DB


# ------------------------------------------------------------ closed loop


def run_reuse_closed_loop(h, f_true, f_hat, s, B, precision="fp32", reuse=True):
    """The engine's canceller (reuse form) in a simulated room; returns the
    loudspeaker and error signals and the float32 microphone blocks."""
    L, P, n_h = h.shape
    room = RoomPlant(f_true, B)
    nb = s.shape[1] // B
    out = np.zeros((L, nb * B), np.float32)
    err = np.zeros((P, nb * B), np.float32)
    mic = np.zeros((P, nb * B), np.float32)
    fb = np.zeros((P, B))
    with U.Engine(48000, B, P, L, n_h, precision, reuse=reuse) as e:
        e.set_filters(h)
        e.set_paths(f_hat)
        assert e.info()["fft_size"] == (3 if reuse else 2) * B
        l_n = np.empty((L, B), np.float32)
        e_n = np.empty((P, B), np.float32)
        for b in range(nb):
            m_n = (s[:, b * B : (b + 1) * B].astype(np.float64) + fb).astype(np.float32)
            e.process_afc(m_n, l_n, e_n)
            out[:, b * B : (b + 1) * B] = l_n
            err[:, b * B : (b + 1) * B] = e_n
            mic[:, b * B : (b + 1) * B] = m_n
            fb = room.step(l_n)
    return out, err, mic


def check_reuse_stages(h, f_hat, y, e, mic, B, bound, label):
    """Stage-wise parity against the reuse oracle, each stage fed the engine's
    own signals:
      synthesis  the engine's l against the oracle's n_f = 3 n_x synthesis of
                 the engine's e (whose accumulated spectra Y_n it keeps);
      canceller  the engine's prediction c = mic - e against the oracle's
                 canceller fed those Y_n as they are (the reuse);
      error      e against mic minus that prediction, its bound lowered by
                 the cancellation gain (as in the n_f = 2 n_x tests)."""
    syn = UpolsOracle(np.asarray(h, np.float64), B, n_f=3 * B)
    canc = UpolsOracle(np.asarray(f_hat, np.float64), B, n_f=3 * B)
    nb = e.shape[1] // B
    l_ref = np.zeros(y.shape)
    c_ref = np.zeros(e.shape)
    e64 = e.astype(np.float64)
    for n in range(nb):
        sl = slice(n * B, (n + 1) * B)
        Y = syn.accumulate(syn.transform_input(e64[:, sl]))
        l_ref[:, sl] = syn.transform_output(Y)
        c_ref[:, sl] = canc.transform_output(canc.accumulate(Y))
    c_eng = mic.astype(np.float64) - e64  # c_{n-1} as applied to block n
    c_ref_applied = shift_blocks(c_ref, B)
    e_ref = mic.astype(np.float64) - c_ref_applied
    s_l = snr_db(y, l_ref)
    s_c = snr_db(c_eng[:, B:], c_ref_applied[:, B:])
    gain = cancellation_gain_db(c_ref_applied, e_ref)
    s_e = snr_db(e, e_ref)
    print(f"{label}: synthesis {s_l:.1f} dB, canceller {s_c:.1f} dB, error {s_e:.1f} dB (gain {gain:.1f} dB)")
    assert s_l >= bound
    assert s_c >= bound
    assert s_e >= bound - gain


def test_closed_loop_small_against_oracle():
    rng = np.random.default_rng(51)
    P, L, B = 2, 3, 64
    h = (rng.standard_normal((L, P, 700)) * np.exp(-np.arange(700) / 200.0) * 0.08).astype(np.float32)
    f = (rng.standard_normal((P, L, 300)) * np.exp(-np.arange(300) / 60.0) * 0.05).astype(np.float32)
    fh = (0.5 * f).astype(np.float32)  # imperfect estimate: residual feedback recirculates
    s = (rng.standard_normal((P, 40 * B)) * 0.1).astype(np.float32)
    y, e, mic = run_reuse_closed_loop(h, f, fh, s, B)
    check_reuse_stages(h, fh, y, e, mic, B, FP32_DB, "reuse closed loop, F_hat = F/2")
    # the n_f = 2 n_x stage replay of the same run (the same mathematics)
    check_replay(h, fh, y, e, mic, B, FP32_DB, "reuse closed loop vs the 2 n_x stages")
    # and the physical loop: the reuse oracle with its own FP64 room, fed s
    ref_l, ref_e, _ = afc_closed_loop_reuse(h, f, fh, s, B)
    print(f"with the oracle's own room: l {snr_db(y, ref_l):.1f} dB, e {snr_db(e, ref_e):.1f} dB")
    assert snr_db(y, ref_l) >= FP32_DB
    assert snr_db(e, ref_e) >= FP32_DB


def test_closed_loop_equals_the_two_nx_form():
    rng = np.random.default_rng(52)
    P, L, B = 3, 4, 128
    h = (rng.standard_normal((L, P, 2000)) * np.exp(-np.arange(2000) / 500.0) * 0.06).astype(np.float32)
    f = (rng.standard_normal((P, L, 500)) * np.exp(-np.arange(500) / 100.0) * 0.05).astype(np.float32)
    fh = (0.7 * f).astype(np.float32)
    s = (rng.standard_normal((P, 30 * B)) * 0.1).astype(np.float32)
    y3, e3, _ = run_reuse_closed_loop(h, f, fh, s, B, reuse=True)
    y2, e2, _ = run_reuse_closed_loop(h, f, fh, s, B, reuse=False)
    print(f"3 n_x vs 2 n_x form: l {snr_db(y3, y2):.1f} dB, e {snr_db(e3, e2):.1f} dB")
    assert snr_db(y3, y2) >= FP32_DB - 6.0  # both within 120 dB of the same oracle result
    assert snr_db(e3, e2) >= FP32_DB - 6.0


@pytest.mark.parametrize("precision,bound", [("fp32", FP32_DB), ("fp16", 55.0), ("bf16", 38.0)])
def test_closed_loop_paper_scale(precision, bound):
    """4 mics x 16 loudspeakers, 8 s synthesis filters, 0.5 s feedback paths
    (F_hat = F), block 256, closed loop in a simulated room, reuse form: the
    error signal must be the dry source and the output its open-loop
    synthesis (the definition, Eq. 2, at sampled points)."""
    w = signals.afc_4x16(block=256, seconds=2.2)
    B = w.block
    nb = w.x.shape[1] // B
    s = np.ascontiguousarray(w.x[:, : nb * B])
    y, e, _ = run_reuse_closed_loop(w.h, w.f, w.f, s, B, precision)
    s_e = snr_db(e, s)
    rng = np.random.default_rng(8)
    pts = sample_points(rng, w.n_out, 0, nb * B, 120)
    ref = np.array([mimo_fir_sample(w.h, s, l, t) for l, t in pts])
    got = np.array([y[l, t] for l, t in pts])
    s_y = snr_db(got, ref)
    print(f"reuse closed loop {precision}: e vs s {s_e:.1f} dB, output {s_y:.1f} dB")
    assert s_e >= bound
    assert s_y >= bound


# ----------------------------------------------------------------- errors


def test_state_and_argument_errors():
    h = np.ones((2, 1, 300), np.float32) * 1e-3
    with U.Engine(48000, 16, 1, 2, 300) as e:  # block 16: no 3 n_x form
        with pytest.raises(U.ConvError) as ei:
            U.afc_set_spectrum_reuse(e.h, True)
        assert ei.value.code == U.CONV_E_INVAL
    with U.Engine(48000, 64, 1, 2, 300) as e:
        with pytest.raises(U.ConvError) as ei:
            U.conv_set_far_block(e.h, 128)
            U.afc_set_spectrum_reuse(e.h, True)
        assert ei.value.code == U.CONV_E_STATE
    with U.Engine(48000, 64, 1, 2, 300, reuse=True) as e:
        with pytest.raises(U.ConvError) as ei:
            U.conv_set_far_block(e.h, 128)
        assert ei.value.code == U.CONV_E_STATE
        e.set_filters(h)
        with pytest.raises(U.ConvError) as ei:  # after the filters
            U.afc_set_spectrum_reuse(e.h, False)
        assert ei.value.code == U.CONV_E_STATE
        e.set_paths(np.ones((1, 2, 100), np.float32) * 1e-3)
        with pytest.raises(U.ConvError) as ei:
            e.set_adaptation(0.05)
        assert ei.value.code == U.CONV_E_STATE
        with pytest.raises(U.ConvError) as ei:
            e.path_spectra()
        assert ei.value.code == U.CONV_E_STATE
        b = U.Batch("fp32")
        try:
            with pytest.raises(U.ConvError) as ei:
                b.add(e)
            assert ei.value.code == U.CONV_E_STATE
        finally:
            b.close()
        # the engine still runs its closed loop
        out = e.process_afc(np.zeros((1, 64), np.float32))
        assert out.shape == (2, 64)

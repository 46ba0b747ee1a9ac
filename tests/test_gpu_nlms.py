"""GPU parity of the adaptive feedback canceller (``afc_set_adaptation``).

The engine drives its canceller in a simulated room (true paths F, FP64) and
adapts F_hat with the NLMS update; the FP64 oracle ``afc_closed_loop_nlms``
runs the same recursion.  Outputs, error signals and the final sub-filter
spectra are compared.
"""

import os

import numpy as np
import pytest

from gpu_helpers import RoomPlant, cancellation_gain_db, snr_db
from oracle.nlms_oracle import NlmsCanceller, afc_closed_loop_nlms
from oracle.upols_oracle import UpolsOracle, upols
from paper_2509_04390_gb300 import build, signals
from paper_2509_04390_gb300 import upols as U

pytestmark = pytest.mark.gpu

# FP32 bound for the adaptive canceller, the same as for every FP32 path.  It
# applies to the like-for-like comparisons: the oracle is fed exactly the
# float32 microphone blocks the engine received (the whole loop), or each stage
# is fed the engine's own signals (the synthesis of the engine's e, and the
# canceller adapting with the engine's e and predicting from its l).
ADAPT_DB = 120.0


@pytest.fixture(scope="module", autouse=True)
def engine_lib():
    if not os.path.exists(build.lib_path()):
        build.build()
    U.load()


def packed(W):
    """Oracle spectra [..][B+1] -> packed [..][B] (bin 0 = DC + i Nyquist)."""
    B = W.shape[-1] - 1
    out = np.array(W[..., :B], dtype=np.complex128)
    out[..., 0] = W[..., 0].real + 1j * W[..., B].real
    return out


def run_adaptive(h, f_true, f_hat0, s, B, mu, lam, delta, precision="fp32", engine=None, blocks=None):
    L, P, n_h = h.shape
    room = RoomPlant(f_true, B)
    nb = s.shape[1] // B if blocks is None else blocks
    out = np.zeros((L, nb * B), np.float32)
    err = np.zeros((P, nb * B), np.float32)
    mic = np.zeros((P, nb * B), np.float32)
    fb = np.zeros((P, B))
    own = engine is None
    e = engine or U.Engine(48000, B, P, L, n_h, precision)
    try:
        if own:
            e.set_filters(h)
            e.set_paths(f_hat0)
            e.set_adaptation(mu, lam, delta)
        l_n = np.empty((L, B), np.float32)
        e_n = np.empty((P, B), np.float32)
        for b in range(nb):
            m_n = (s[:, b * B : (b + 1) * B].astype(np.float64) + fb).astype(np.float32)
            e.process_afc(m_n, l_n, e_n)
            out[:, b * B : (b + 1) * B] = l_n
            err[:, b * B : (b + 1) * B] = e_n
            mic[:, b * B : (b + 1) * B] = m_n
            fb = room.step(l_n)
        spec = e.path_spectra()
    finally:
        if own:
            e.close()
    run_adaptive.mic = mic
    return out, err, spec


def check_adaptive(label, h, fh0, y, e, spec, mic, B, mu, lam, delta, start=0, physical=None):
    """Like-for-like parity of an adaptive run at ADAPT_DB: each stage fed the
    engine's own signals, so the comparison holds only what the engine
    computed in that stage.
      synthesis  the engine's l against the oracle's UPOLS of the engine's e;
      canceller  the oracle's canceller adapting with the engine's e and
                 predicting from the engine's l: the final spectra F_hat, the
                 prediction c = mic - e (over the previous block), and e
                 itself, whose bound is lowered by the cancellation gain
                 rms(c) / rms(e) (a subtraction keeps no more relative
                 precision than its operands have).
    `start`: the first block that adapts (static before).  Reported beside
    them: the whole loop replayed from the microphone blocks alone (no room:
    other dynamics than the physical loop) and `physical`, the oracle's own
    closed loop with the room, (l, e, canceller); in both the engine's
    rounding circulates through a loop, so they are not bounded."""
    P, L = fh0.shape[0], fh0.shape[1]
    nb = mic.shape[1] // B
    mic64 = mic.astype(np.float64)
    synth = UpolsOracle(h, B)
    loop = NlmsCanceller(fh0, B, mu, lam, delta)
    stage = NlmsCanceller(fh0, B, mu, lam, delta)
    loop_l, loop_e = np.zeros((L, nb * B)), np.zeros((P, nb * B))
    stage_e = np.zeros((P, nb * B))
    c_loop, c_stage = np.zeros((P, B)), np.zeros((P, B))
    with np.errstate(all="ignore"):
        for b in range(nb):
            sl = slice(b * B, (b + 1) * B)
            e_b = mic64[:, sl] - c_loop
            stage_e[:, sl] = mic64[:, sl] - c_stage
            if b >= start:
                loop.adapt(e_b)
                stage.adapt(e[:, sl].astype(np.float64))
            l_b = synth.process_block(e_b)
            c_loop = loop.predict(l_b)
            c_stage = stage.predict(y[:, sl].astype(np.float64))
            loop_l[:, sl], loop_e[:, sl] = l_b, e_b
    stage_l = upols(h.astype(np.float64), e.astype(np.float64), B)
    c_eng = mic64 - e.astype(np.float64)
    c_ref = mic64 - stage_e
    gain = cancellation_gain_db(c_ref, stage_e)
    got = {
        "synthesis stage l": snr_db(y, stage_l),
        "canceller stage F_hat": snr_db(spec, packed(stage.W)),
        "canceller stage c": snr_db(c_eng, c_ref),
        "canceller stage e": snr_db(e, stage_e),
    }
    msg = f"{label}: " + ", ".join(f"{k} {v:.1f}" for k, v in got.items()) + f" dB (cancellation gain {gain:.1f} dB)"
    msg += f" | loop replayed: l {snr_db(y, loop_l):.1f}, e {snr_db(e, loop_e):.1f}, F_hat {snr_db(spec, packed(loop.W)):.1f}"
    if physical is not None:
        pl, pe, pc = physical
        msg += f" | with the oracle's own room: l {snr_db(y, pl):.1f}, e {snr_db(e, pe):.1f}, " \
               f"F_hat {snr_db(spec, packed(pc.W)):.1f}"
    print(msg + " dB")
    for k in ("synthesis stage l", "canceller stage F_hat", "canceller stage c"):
        assert got[k] >= ADAPT_DB, f"{label} {k}: {got[k]:.1f} dB < {ADAPT_DB} dB"
    assert got["canceller stage e"] >= ADAPT_DB - gain, (label, got, gain)


def small_case(seed=51, P=2, L=3, B=64, n_h=700, n_t=300, nb=60):
    rng = np.random.default_rng(seed)
    h = (rng.standard_normal((L, P, n_h)) * np.exp(-np.arange(n_h) / 200.0) * 0.08).astype(np.float32)
    f = (rng.standard_normal((P, L, n_t)) * np.exp(-np.arange(n_t) / 60.0) * 0.05).astype(np.float32)
    s = (rng.standard_normal((P, nb * B)) * 0.1).astype(np.float32)
    return h, f, s


@pytest.mark.parametrize("B,f0_scale", [(64, 0.0), (64, 0.5), (128, 0.0)])
def test_adaptive_closed_loop_against_oracle(B, f0_scale):
    h, f, s = small_case(B=B)
    fh0 = (f0_scale * f).astype(np.float32)
    mu, lam, delta = 0.3, 0.9, 1e-2
    y, e, spec = run_adaptive(h, f, fh0, s, B, mu, lam, delta)
    phys = afc_closed_loop_nlms(h, f, fh0, s, B, mu, lam, delta)
    check_adaptive(f"adaptive B={B} f0={f0_scale}", h, fh0, y, e, spec, run_adaptive.mic, B, mu, lam, delta,
                   physical=phys)
    # and the estimate moved: the update is not a no-op
    start = U.Engine(48000, B, 2, 3, h.shape[2])
    try:
        start.set_filters(h)
        start.set_paths(fh0)
        w0 = start.path_spectra()
    finally:
        start.close()
    moved = np.sqrt(np.sum(np.abs(spec - w0) ** 2) / np.sum(np.abs(spec) ** 2))
    assert moved > 0.01


@pytest.mark.parametrize("B,n_t", [(64, 64), (64, 100), (32, 300), (16, 257)])
def test_adaptive_partition_counts_against_oracle(B, n_t):
    """K_fb = 1 (the delay line is one entry: the update and the correction
    read the copy the push saved), K_fb = 2, and longer rings with a ragged
    last partition."""
    h, f, s = small_case(seed=60 + n_t, B=B, n_t=n_t, nb=50)
    fh0 = (0.25 * f).astype(np.float32)
    # mu = 0.1: with one or two partitions the unconstrained update at larger
    # steps makes the closed loop diverge in the FP64 oracle as well
    mu, lam, delta = 0.1, 0.8, 1e-2
    y, e, spec = run_adaptive(h, f, fh0, s, B, mu, lam, delta)
    phys = afc_closed_loop_nlms(h, f, fh0, s, B, mu, lam, delta)
    check_adaptive(f"adaptive B={B} n_t={n_t} (K_fb {phys[2].K})", h, fh0, y, e, spec, run_adaptive.mic, B,
                   mu, lam, delta, physical=phys)


def test_switching_adaptation_on_mid_stream_against_oracle():
    """Static canceller for 20 blocks, then adaptive: the oracle's loop skips
    the NLMS step (and the power recursion) until the same block."""
    h, f, s = small_case(seed=57, nb=50)
    P, L, B = 2, 3, 64
    n0, nb = 20, 50
    fh0 = (0.5 * f).astype(np.float32)
    mu, lam, delta = 0.3, 0.9, 1e-2
    with U.Engine(48000, B, P, L, h.shape[2]) as e:
        e.set_filters(h)
        e.set_paths(fh0)
        y0, e0, _ = run_adaptive(h, f, None, s[:, : n0 * B], B, None, None, None, engine=e)
        mic0 = run_adaptive.mic
        fb_state = RoomPlant(f, B)
        # the room's state at block n0 comes from the loudspeaker blocks so far
        fb = np.zeros((P, B))
        for b in range(n0):
            fb = fb_state.step(y0[:, b * B : (b + 1) * B])
        e.set_adaptation(mu, lam, delta)
        y1 = np.zeros((L, (nb - n0) * B), np.float32)
        e1 = np.zeros((P, (nb - n0) * B), np.float32)
        mic1 = np.zeros((P, (nb - n0) * B), np.float32)
        l_n = np.empty((L, B), np.float32)
        e_n = np.empty((P, B), np.float32)
        for b in range(n0, nb):
            m_n = (s[:, b * B : (b + 1) * B].astype(np.float64) + fb).astype(np.float32)
            e.process_afc(m_n, l_n, e_n)
            y1[:, (b - n0) * B : (b - n0 + 1) * B] = l_n
            e1[:, (b - n0) * B : (b - n0 + 1) * B] = e_n
            mic1[:, (b - n0) * B : (b - n0 + 1) * B] = m_n
            fb = fb_state.step(l_n)
        spec = e.path_spectra()
    y = np.concatenate([y0, y1], axis=1)
    err = np.concatenate([e0, e1], axis=1)
    synth, room = UpolsOracle(h, B), UpolsOracle(f, B)
    can = NlmsCanceller(fh0, B, mu, lam, delta)
    ref_l, ref_e = np.zeros((L, nb * B)), np.zeros((P, nb * B))
    fb_prev, c_prev = np.zeros((P, B)), np.zeros((P, B))
    for b in range(nb):
        sl = slice(b * B, (b + 1) * B)
        e_b = s[:, sl].astype(np.float64) + fb_prev - c_prev
        if b >= n0:
            can.adapt(e_b)
        l_b = synth.process_block(e_b)
        c_prev = can.predict(l_b)
        fb_prev = room.process_block(l_b)
        ref_l[:, sl], ref_e[:, sl] = l_b, e_b
    mic = np.concatenate([mic0, mic1], axis=1)
    check_adaptive(f"adaptation switched on at block {n0}", h, fh0, y, err, spec, mic, B, mu, lam, delta,
                   start=n0, physical=(ref_l, ref_e, can))


def test_path_spectra_are_the_subfilter_ffts():
    rng = np.random.default_rng(5)
    P, L, B, n_t = 3, 5, 32, 150
    f = rng.standard_normal((P, L, n_t)).astype(np.float32)
    with U.Engine(48000, B, P, L, 64) as e:
        e.set_filters(rng.standard_normal((L, P, 64)).astype(np.float32))
        e.set_paths(f)
        got = e.path_spectra()
    K = -(-n_t // B)
    pad = np.zeros((P, L, K * B))
    pad[:, :, :n_t] = f
    ref = packed(np.fft.rfft(pad.reshape(P, L, K, B), n=2 * B, axis=-1))
    assert got.shape == ref.shape
    assert snr_db(got, ref) >= 120.0


def test_vanishing_step_reproduces_the_static_schedule():
    """delta far above the signal power makes every step round away, so the
    adaptive schedule (step on partition 0, deferred step fused with the
    canceller's tail, correlation terms) must leave the spectra exactly as
    they were and give the static schedule's outputs up to the rounding of
    its own tail summation order."""
    h, f, s = small_case(seed=52, nb=40)
    fh0 = (0.5 * f).astype(np.float32)
    y0, e0, w0 = run_adaptive(h, f, fh0, s, 64, 0.0, 0.5, 0.0)
    y1, e1, w1 = run_adaptive(h, f, fh0, s, 64, 1e-3, 0.5, 1e30)
    assert np.array_equal(w0, w1)
    print(f"vanishing step vs static: l {snr_db(y1, y0):.1f} dB, e {snr_db(e1, e0):.1f} dB")
    assert snr_db(y1, y0) >= 125.0
    assert snr_db(e1, e0) >= 125.0


def test_reset_and_paths_repeat_bit_exact():
    h, f, s = small_case(seed=53, nb=30)
    P, L = 2, 3
    with U.Engine(48000, 64, P, L, h.shape[2]) as e:
        e.set_filters(h)
        e.set_paths(np.zeros_like(f))
        e.set_adaptation(0.4, 0.8, 1e-2)
        y0, e0, w0 = run_adaptive(h, f, None, s, 64, None, None, None, engine=e)
        e.reset()
        e.set_paths(np.zeros_like(f))
        y1, e1, w1 = run_adaptive(h, f, None, s, 64, None, None, None, engine=e)
        assert e.info()["afc_adaptive"] == 1
        assert e.info()["kernels_per_afc_block"] == 8
    assert np.array_equal(y0, y1) and np.array_equal(e0, e1) and np.array_equal(w0, w1)


def test_switching_adaptation_off_keeps_the_estimate():
    h, f, s = small_case(seed=54, nb=50)
    P, L, B = 2, 3, 64
    with U.Engine(48000, B, P, L, h.shape[2]) as e:
        e.set_filters(h)
        e.set_paths(np.zeros_like(f))
        e.set_adaptation(0.3, 0.9, 1e-2)
        run_adaptive(h, f, None, s[:, : 25 * B], B, None, None, None, engine=e)
        w_mid = e.path_spectra()
        e.set_adaptation(0.0)
        assert e.info()["afc_adaptive"] == 0
        run_adaptive(h, f, None, s[:, 25 * B :], B, None, None, None, engine=e)
        assert np.array_equal(e.path_spectra(), w_mid)


def test_state_and_argument_errors():
    h, f, _ = small_case(seed=55, nb=2)
    with U.Engine(48000, 64, 2, 3, h.shape[2]) as e:
        e.set_filters(h)
        with pytest.raises(U.ConvError) as ei:
            e.set_adaptation(0.3)
        assert ei.value.code == U.CONV_E_STATE  # no paths yet
        e.set_paths(f)
        for mu, lam, delta in ((-0.1, 0.9, 1e-3), (2.0, 0.9, 1e-3), (0.3, 1.0, 1e-3), (0.3, 0.9, -1.0),
                               (0.3, 0.9, 0.0), (0.3, 0.9, float("inf"))):
            with pytest.raises(U.ConvError) as ei:
                e.set_adaptation(mu, lam, delta)
            assert ei.value.code == U.CONV_E_INVAL
        e.set_adaptation(0.3, 0.9, 1e-3)
        with pytest.raises(U.ConvError) as ei:
            e.process(np.zeros((2, 64), np.float32))  # a synthesis-only block would skip the canceller
        assert ei.value.code == U.CONV_E_STATE
        with U.Batch("fp32") as b:
            with pytest.raises(U.ConvError) as ei:
                b.add(e)
            assert ei.value.code == U.CONV_E_STATE
        e.set_adaptation(0.0)
        with U.Batch("fp32") as b:
            b.add(e)
            with pytest.raises(U.ConvError) as ei:
                e.set_adaptation(0.3)
            assert ei.value.code == U.CONV_E_STATE  # in a batch
            b.remove(e)
        e.set_adaptation(0.3)
    with U.Engine(48000, 64, 2, 3, h.shape[2], "fp16") as e:
        e.set_filters(h)
        e.set_paths(f)
        for call in (lambda: e.set_adaptation(0.3), e.path_spectra):
            with pytest.raises(U.ConvError) as ei:
                call()
            assert ei.value.code == U.CONV_E_STATE


def test_adaptive_paper_scale_canceller_against_oracle():
    """Canceller at the paper's feedback size (4 mics x 16 loudspeakers, 0.5 s
    paths, block 256) with 0.5 s synthesis filters (the oracle's synthesis
    at the full 8 s would dominate the test's time), F_hat starting at
    half the true paths, 120 blocks."""
    rng = np.random.default_rng(61)
    P, L, B = 4, 16, 256
    h = signals.paper_filters(rng, L, P, 24000, rt60=0.4, reflections=5).astype(np.float32)
    f = signals.feedback_paths(rng, P, L, 24000).astype(np.float32)
    nb = 120
    s = (signals.pink_noise(rng, P, nb * B, 0.1)).astype(np.float32)
    fh0 = (0.5 * f).astype(np.float32)
    mu, lam, delta = 0.2, 0.95, 1e-1
    y, e, spec = run_adaptive(h, f, fh0, s, B, mu, lam, delta)
    phys = afc_closed_loop_nlms(h, f, fh0, s, B, mu, lam, delta)
    check_adaptive("adaptive paper-scale canceller", h, fh0, y, e, spec, run_adaptive.mic, B, mu, lam, delta,
                   physical=phys)


def open_loop_adaptive(e, s, B, read_at=(), stream_plan=None):
    """Drive an adaptive engine with microphone blocks s (no room): host calls,
    or device calls on the streams that stream_plan(b) names (None: host)."""
    torch = pytest.importorskip("torch")
    P = s.shape[0]
    L = e.info()["n_out"]
    nb = s.shape[1] // B
    y = np.zeros((L, nb * B), np.float32)
    err = np.zeros((P, nb * B), np.float32)
    d_m = torch.from_numpy(s).cuda().reshape(P, nb, B).permute(1, 0, 2).contiguous()
    d_y = torch.zeros((nb, L, B), dtype=torch.float32, device="cuda")
    d_e = torch.zeros((nb, P, B), dtype=torch.float32, device="cuda")
    on_dev = []
    l_n = np.empty((L, B), np.float32)
    e_n = np.empty((P, B), np.float32)
    torch.cuda.synchronize()
    for b in range(nb):
        st = stream_plan(b) if stream_plan else None
        if st is None:
            e.process_afc(np.ascontiguousarray(s[:, b * B : (b + 1) * B]), l_n, e_n)
            y[:, b * B : (b + 1) * B] = l_n
            err[:, b * B : (b + 1) * B] = e_n
        else:
            U.afc_process_block_async(e.h, d_m[b], d_y[b], d_e[b], st)
            on_dev.append(b)
        if b in read_at:
            e.path_spectra()
    U.conv_synchronize(e.h)
    torch.cuda.synchronize()
    dy, de = d_y.cpu().numpy(), d_e.cpu().numpy()
    for b in on_dev:
        y[:, b * B : (b + 1) * B] = dy[b]
        err[:, b * B : (b + 1) * B] = de[b]
    return y, err, e.path_spectra()


def test_adaptive_device_streams_and_spectra_reads_are_bit_exact():
    """The adaptive schedule through device calls on two alternating caller
    streams (with host calls in between), and with the spectra read back
    mid-stream (which applies the pending deferred step early), gives exactly
    the host-call result."""
    torch = pytest.importorskip("torch")
    h, f, s = small_case(seed=58, nb=40)
    P, L, B = 2, 3, 64

    def engine():
        e = U.Engine(48000, B, P, L, h.shape[2])
        e.set_filters(h)
        e.set_paths((0.3 * f).astype(np.float32))
        e.set_adaptation(0.3, 0.9, 1e-2)
        return e

    with engine() as e:
        y0, e0, w0 = open_loop_adaptive(e, s, B)
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    with engine() as e:
        y1, e1, w1 = open_loop_adaptive(e, s, B, stream_plan=lambda b: None if b % 3 == 2 else streams[b % 2])
    with engine() as e:
        y2, e2, w2 = open_loop_adaptive(e, s, B, read_at=(0, 17, 29))
    assert np.array_equal(y0, y1) and np.array_equal(e0, e1) and np.array_equal(w0, w1)
    assert np.array_equal(y0, y2) and np.array_equal(e0, e2) and np.array_equal(w0, w2)


def test_reset_keeps_the_adapted_estimate():
    """conv_reset restarts the stream but keeps F_hat as adapted so far,
    including the step the deferred schedule has not applied to the tail
    partitions yet."""
    h, f, s = small_case(seed=59, nb=30)
    P, L, B = 2, 3, 64

    def engine():
        e = U.Engine(48000, B, P, L, h.shape[2])
        e.set_filters(h)
        e.set_paths((0.3 * f).astype(np.float32))
        e.set_adaptation(0.3, 0.9, 1e-2)
        return e

    with engine() as e:
        open_loop_adaptive(e, s, B)
        w0 = e.path_spectra()
    with engine() as e:
        l_n = np.empty((L, B), np.float32)
        for b in range(s.shape[1] // B):
            e.process_afc(np.ascontiguousarray(s[:, b * B : (b + 1) * B]), l_n)
        e.reset()
        w1 = e.path_spectra()
        assert e.info()["afc_adaptive"] == 1
    assert np.array_equal(w0, w1)

"""GPU parity of non-uniform partitioning (``conv_set_far_block``).

Splitting a filter into a near part (partitions of the block size) and a far
part (partitions of the far block, run once per far block, output delayed by
the far block) leaves the result the causal linear convolution of Eqs. 2 and
4, so the oracle is the same FP64 UPOLS / definition as for a plain engine,
at the same bounds (FP32 >= 120 dB, FP16 >= 60 dB, BF16 >= 42 dB).
"""

import os

import numpy as np
import pytest

from gpu_helpers import RoomPlant, check_replay, sample_points, snr_db
from oracle import afc_closed_loop, mimo_fir_sample, upols
from paper_2509_04390_gb300 import build, signals
from paper_2509_04390_gb300 import upols as U

pytestmark = pytest.mark.gpu

BOUND = {"fp32": 120.0, "fp16": 60.0, "bf16": 42.0}


@pytest.fixture(scope="module", autouse=True)
def engine_lib():
    if not os.path.exists(build.lib_path()):
        build.build()
    U.load()


def run_nupc(w, far_block, precision="fp32", n_blocks=None):
    x = w.x if n_blocks is None else w.x[:, : n_blocks * w.block]
    with U.Engine(w.fs, w.block, w.n_in, w.n_out, w.taps, precision, far_block=far_block) as e:
        e.set_filters(w.h)
        info = e.info()
        return e.run(x), info


@pytest.mark.parametrize(
    "B,F,n_in,n_out,taps,nb,precision",
    [
        (64, 256, 2, 3, 3000, 60, "fp32"),  # m = 4, ragged far partitions, far ring wraps
        (64, 128, 2, 3, 3000, 60, "fp32"),  # m = 2
        (16, 256, 1, 2, 257, 64, "fp32"),  # far part of a single tap
        (128, 1024, 3, 5, 9000, 48, "fp32"),
        (32, 4096, 1, 1, 5000, 300, "fp32"),  # largest far block
        (64, 512, 2, 3, 6000, 60, "fp16"),
        (64, 512, 2, 3, 6000, 60, "bf16"),
    ],
)
def test_nupc_against_oracle(B, F, n_in, n_out, taps, nb, precision):
    w = signals.random_case(500 + taps + F, n_in, n_out, taps, B, nb, decay_s=0.05)
    y, info = run_nupc(w, F, precision)
    ref = upols(w.h.astype(np.float64), w.x.astype(np.float64), B)
    s = snr_db(y, ref)
    print(f"nupc {precision} B={B} F={F} {n_in}x{n_out} taps={taps}: {s:.1f} dB, K near {info['K']}, far {info['K_far']}")
    assert info["far_block"] == F and info["K"] == F // B and info["K_far"] == -(-(taps - F) // F)
    assert s >= BOUND[precision]


def test_nupc_paper_scale_sampled():
    """4 x 16, 8 s filters, block 256 with a 2048-sample far block (the far
    ring of 184 partitions wraps within the 9 s input): sampled outputs
    against the definition."""
    w = signals.paper_4x16(block=256, seconds=9.0)
    y, info = run_nupc(w, 2048)
    T = w.x.shape[1]
    rng = np.random.default_rng(11)
    pts = sample_points(rng, w.n_out, 0, T, 120) + sample_points(rng, w.n_out, w.taps, T, 120)
    ref = np.array([mimo_fir_sample(w.h, w.x, l, t) for l, t in pts])
    got = np.array([y[l, t] for l, t in pts])
    s = snr_db(got, ref)
    print(f"nupc paper scale: {s:.1f} dB")
    assert s >= BOUND["fp32"]


def test_nupc_closed_loop_against_oracle():
    rng = np.random.default_rng(43)
    P, L, B, F = 2, 3, 64, 512
    n_h = 4000
    h = (rng.standard_normal((L, P, n_h)) * np.exp(-np.arange(n_h) / 900.0) * 0.05).astype(np.float32)
    f = (rng.standard_normal((P, L, 300)) * np.exp(-np.arange(300) / 60.0) * 0.05).astype(np.float32)
    fh = (0.5 * f).astype(np.float32)
    nb = 48
    s = (rng.standard_normal((P, nb * B)) * 0.1).astype(np.float32)
    room = RoomPlant(f, B)
    y = np.zeros((L, nb * B), np.float32)
    err = np.zeros((P, nb * B), np.float32)
    mic = np.zeros((P, nb * B), np.float32)
    fb = np.zeros((P, B))
    with U.Engine(48000, B, P, L, n_h, far_block=F) as e:
        e.set_filters(h)
        e.set_paths(fh)
        l_n = np.empty((L, B), np.float32)
        e_n = np.empty((P, B), np.float32)
        for b in range(nb):
            m_n = (s[:, b * B : (b + 1) * B].astype(np.float64) + fb).astype(np.float32)
            e.process_afc(m_n, l_n, e_n)
            y[:, b * B : (b + 1) * B] = l_n
            err[:, b * B : (b + 1) * B] = e_n
            mic[:, b * B : (b + 1) * B] = m_n
            fb = room.step(l_n)
    ref_l, ref_e, _ = afc_closed_loop(h, f, fh, s, B)
    print(f"nupc closed loop: l {snr_db(y, ref_l):.1f} dB, e {snr_db(err, ref_e):.1f} dB")
    assert snr_db(y, ref_l) >= BOUND["fp32"]
    assert snr_db(err, ref_e) >= BOUND["fp32"]
    # like for like: each stage fed the engine's own signals
    check_replay(h, fh, y, err, mic, B, BOUND["fp32"], "nupc closed loop")


def test_nupc_reset_and_device_path_bit_exact():
    torch = pytest.importorskip("torch")
    w = signals.random_case(77, 2, 3, 2500, 64, 40, decay_s=0.05)
    with U.Engine(w.fs, w.block, w.n_in, w.n_out, w.taps, far_block=256) as e:
        e.set_filters(w.h)
        y0 = e.run(w.x)
        e.reset()
        y1 = e.run(w.x)
        e.reset()
        B, nb = w.block, w.x.shape[1] // w.block
        d_blocks = torch.from_numpy(w.x).cuda().reshape(w.n_in, nb, B).permute(1, 0, 2).contiguous()
        d_y = torch.empty((nb, w.n_out, B), dtype=torch.float32, device="cuda")
        stream = torch.cuda.current_stream()
        for b in range(nb):
            U.conv_process_block_async(e.h, d_blocks[b], d_y[b], stream)
        U.conv_synchronize(e.h)
        y2 = d_y.permute(1, 0, 2).reshape(w.n_out, nb * B).cpu().numpy()
    assert np.array_equal(y0, y1)
    assert np.array_equal(y0, y2)


def test_far_block_off_is_the_plain_engine():
    w = signals.random_case(78, 2, 3, 2500, 64, 30, decay_s=0.05)
    with U.Engine(w.fs, w.block, w.n_in, w.n_out, w.taps) as e:
        e.set_filters(w.h)
        y0 = e.run(w.x)
    with U.Engine(w.fs, w.block, w.n_in, w.n_out, w.taps, far_block=512) as e:
        U.conv_set_far_block(e.h, 0)
        e.set_filters(w.h)
        assert e.info()["far_block"] == 0
        y1 = e.run(w.x)
    assert np.array_equal(y0, y1)


def test_far_block_errors():
    w = signals.random_case(79, 2, 3, 2500, 64, 2, decay_s=0.05)
    with U.Engine(w.fs, 64, 2, 3, 2500) as e:
        for bad in (64, 32, 96, 8192, 4096):  # <= block, not a power of two, too large, >= taps
            with pytest.raises(U.ConvError) as ei:
                U.conv_set_far_block(e.h, bad)
            assert ei.value.code == U.CONV_E_INVAL
        U.conv_set_far_block(e.h, 256)
        assert U.conv_far_engine(e.h) is not None
        with U.Batch("fp32") as b:
            with pytest.raises(U.ConvError) as ei:
                b.add(e)
            assert ei.value.code in (U.CONV_E_STATE, U.CONV_E_INVAL)
        e.set_filters(w.h)
        with pytest.raises(U.ConvError) as ei:
            U.conv_set_far_block(e.h, 512)
        assert ei.value.code == U.CONV_E_STATE
        e.set_paths(np.zeros((2, 3, 100), np.float32))
        with pytest.raises(U.ConvError) as ei:
            e.set_adaptation(0.3)
        assert ei.value.code == U.CONV_E_STATE


@pytest.mark.parametrize("B,F,F2,taps,nb,precision", [(64, 256, 1024, 9000, 160, "fp32"), (32, 128, 2048, 12000, 420, "fp32"),
                                                       (64, 256, 1024, 9000, 160, "fp16")])
def test_nested_far_blocks_against_oracle(B, F, F2, taps, nb, precision):
    """Three partition sizes: the far part's engine gets a far block of its own
    (conv_set_far_block on conv_far_engine), so taps [0, F) run in partitions
    of B, [F, F + F2) in partitions of F and the rest in partitions of F2; the
    output is still the causal convolution."""
    w = signals.random_case(900 + F2, 2, 3, taps, B, nb, decay_s=0.1)
    with U.Engine(w.fs, B, w.n_in, w.n_out, w.taps, precision, far_block=F) as e:
        far = U.conv_far_engine(e.h)
        U.conv_set_far_block(far, F2)
        e.set_filters(w.h)
        y = e.run(w.x)
        e.reset()
        y2 = e.run(w.x)
    ref = upols(w.h.astype(np.float64), w.x.astype(np.float64), B)
    s = snr_db(y, ref)
    print(f"nested far blocks {precision} B={B} F={F} F2={F2}: {s:.1f} dB")
    assert s >= BOUND[precision]
    assert np.array_equal(y, y2)

"""GPU parity of shared-filter session groups (tensor-core FDL MAC).

Every session of a group is an independent stream through the shared
filters, so each session's output is checked against the FP64 oracle's
UPOLS (Sec. 4) of its own input, element by element, at the reduced-precision
bounds of the single-session engine (FP16 >= 60 dB, BF16 >= 42 dB).  At paper
scale, sampled outputs are checked against the definition (Eq. 2).
"""

import os

import numpy as np
import pytest

from gpu_helpers import sample_points, snr_db
from oracle import mimo_fir_sample, upols
from paper_2509_04390_gb300 import build, signals
from paper_2509_04390_gb300 import upols as U

pytestmark = pytest.mark.gpu

BOUND = {"fp16": 60.0, "bf16": 42.0}


@pytest.fixture(scope="module", autouse=True)
def engine_lib():
    if not os.path.exists(build.lib_path()):
        build.build()
    U.load()


def group_case(seed, S, n_in, n_out, taps, B, nb):
    rng = np.random.default_rng(seed)
    h = (rng.standard_normal((n_out, n_in, taps)) / np.sqrt(taps) * 4.0).astype(np.float32)
    x = (rng.standard_normal((S, n_in, nb * B)) * 0.1).astype(np.float32)
    return h, x


@pytest.mark.parametrize(
    "precision,S,n_in,n_out,taps,B,nb",
    [
        ("fp16", 8, 4, 16, 3000, 64, 60),  # ragged last partition, ring wraps
        ("bf16", 8, 4, 16, 3000, 64, 60),
        ("fp16", 16, 4, 16, 1500, 32, 70),  # 16 sessions: N = 256
        ("fp16", 8, 8, 8, 700, 16, 60),  # 16 bins per tile, one slot per ring row
        ("fp16", 8, 1, 32, 900, 128, 20),  # 4 bins per tile, 8 slots per ring row
        ("fp16", 32, 2, 32, 1000, 64, 30),  # 32 sessions, 4 slots per ring row
        ("fp16", 8, 4, 16, 1, 64, 6),  # one tap: K = 1, ring of 4 slots
        ("fp16", 1, 4, 16, 3000, 64, 60),  # one session: N = 16
        ("bf16", 2, 2, 16, 2000, 32, 80),
        ("fp16", 4, 8, 8, 1200, 16, 90),  # 16 bins x 4 sessions
        ("fp16", 2, 1, 32, 5000, 128, 50),  # 4 bins x 2 sessions: N = 16
    ],
)
def test_group_sessions_against_oracle(precision, S, n_in, n_out, taps, B, nb):
    h, x = group_case(100 + taps + S, S, n_in, n_out, taps, B, nb)
    with U.Group(precision, B, n_in, n_out, taps, S) as g:
        g.set_filters(h)
        y = g.run(x)
        info = g.info()
    worst = min(snr_db(y[s], upols(h, x[s], B)) for s in range(S))
    print(f"group {precision} S={S} {n_in}x{n_out} taps={taps} B={B}: worst session {worst:.1f} dB, "
          f"splits {info['splits']}, stages {info['stages']}x{info['stage_k_steps']}")
    assert worst >= BOUND[precision]


@pytest.mark.parametrize(
    "tiling",
    [
        {"ctas": 1},  # one CTA walks every (group, K-step) unit: many accumulator segments
        {"ctas": 7, "stage_k_steps": 1, "stages": 2},
        {"ctas": 37, "stage_k_steps": 3, "stages": 4, "tail_streams": 1},
        {"ctas": 152, "stage_k_steps": 4, "stages": 2},
    ],
)
def test_group_tilings_against_oracle(tiling):
    """Work splits whose runs cross bin-group boundaries, shallow and deep
    pipelines, one or two tail streams: same result bound."""
    S, n_in, n_out, taps, B, nb = 8, 4, 16, 2500, 64, 45
    h, x = group_case(300, S, n_in, n_out, taps, B, nb)
    with U.Group("fp16", B, n_in, n_out, taps, S, tiling) as g:
        g.set_filters(h)
        y = g.run(x)
        info = g.info()
    worst = min(snr_db(y[s], upols(h, x[s], B)) for s in range(S))
    print(f"group tiling {tiling}: worst session {worst:.1f} dB, ctas {info['tail_ctas']}, slots {info['splits']}")
    assert worst >= BOUND["fp16"]


def test_sessions_are_independent():
    """Session s's output must not depend on the other sessions' inputs."""
    S, n_in, n_out, taps, B, nb = 8, 4, 16, 2000, 64, 40
    h, x = group_case(7, S, n_in, n_out, taps, B, nb)
    x2 = x.copy()
    x2[1:] = np.random.default_rng(8).standard_normal(x2[1:].shape).astype(np.float32)
    with U.Group("fp16", B, n_in, n_out, taps, S) as g:
        g.set_filters(h)
        y = g.run(x)
        g.reset()
        y2 = g.run(x2)
    assert np.array_equal(y[0], y2[0])


def test_reset_repeats_bit_exact():
    S, n_in, n_out, taps, B, nb = 8, 4, 16, 2000, 64, 50
    h, x = group_case(9, S, n_in, n_out, taps, B, nb)
    with U.Group("bf16", B, n_in, n_out, taps, S) as g:
        g.set_filters(h)
        y0 = g.run(x)
        g.reset()
        y1 = g.run(x)
    assert np.array_equal(y0, y1)


def test_l2_keep_leaves_results_unchanged():
    """conv_group_set_l2_keep changes only the L2 policy of the filter-tile
    copies: no budget and a budget above every tile give the default's output
    bit for bit; a negative budget is refused."""
    S, n_in, n_out, taps, B, nb = 8, 4, 16, 2000, 64, 30
    h, x = group_case(10, S, n_in, n_out, taps, B, nb)
    outs = []
    for keep in (None, 0, 1 << 40):
        with U.Group("fp16", B, n_in, n_out, taps, S) as g:
            if keep is not None:
                U.conv_group_set_l2_keep(g.g, keep)
            g.set_filters(h)
            outs.append(g.run(x))
            with pytest.raises(U.ConvError) as ei:
                U.conv_group_set_l2_keep(g.g, -1)
            assert ei.value.code == U.CONV_E_INVAL
    assert np.array_equal(outs[0], outs[1])
    assert np.array_equal(outs[0], outs[2])


def test_render_equals_block_calls():
    """conv_group_process_blocks over a chunk boundary (300 blocks) is the
    block-by-block stream, bit for bit."""
    S, n_in, n_out, taps, B, nb = 8, 4, 16, 700, 16, 300
    h, x = group_case(11, S, n_in, n_out, taps, B, nb)
    with U.Group("fp16", B, n_in, n_out, taps, S) as g:
        g.set_filters(h)
        y_blocks = g.run(x)
        g.reset()
        y_render = g.render(x)
    assert np.array_equal(y_blocks, y_render)


def test_device_path_matches_host_path():
    torch = pytest.importorskip("torch")
    S, n_in, n_out, taps, B, nb = 8, 4, 16, 1200, 64, 30
    h, x = group_case(10, S, n_in, n_out, taps, B, nb)
    with U.Group("fp16", B, n_in, n_out, taps, S) as g:
        g.set_filters(h)
        y_host = g.run(x)
        g.reset()
        d_x = torch.from_numpy(x).cuda()
        d_blocks = d_x.reshape(S, n_in, nb, B).permute(2, 0, 1, 3).contiguous()
        d_y = torch.empty((nb, S, n_out, B), dtype=torch.float32, device="cuda")
        stream = torch.cuda.current_stream()
        for b in range(nb):
            U.conv_group_process_async(g.g, d_blocks[b], d_y[b], stream)
        U.conv_group_synchronize(g.g)
        y_dev = d_y.permute(1, 2, 0, 3).reshape(S, n_out, nb * B).cpu().numpy()
    assert np.array_equal(y_host, y_dev)


def test_group_paper_scale_sampled():
    """8 sessions of the 4x16 paper configuration (8 s filters, block 256)
    sharing one filter set, past the ring wrap: sampled outputs of every
    session against the definition."""
    w = signals.paper_4x16(block=256, seconds=9.0)
    S, B = 8, w.block
    nb = w.x.shape[1] // B
    x = np.stack([np.roll(w.x[:, : nb * B], 4801 * s, axis=1) for s in range(S)]).astype(np.float32)
    with U.Group("fp16", B, w.n_in, w.n_out, w.taps, S) as g:
        g.set_filters(w.h)
        y = g.run(x)
    rng = np.random.default_rng(3)
    for s in (0, 3, 7):
        pts = sample_points(rng, w.n_out, w.taps, nb * B, 60)
        ref = np.array([mimo_fir_sample(w.h, x[s], l, t) for l, t in pts])
        got = np.array([y[s, l, t] for l, t in pts])
        sn = snr_db(got, ref)
        print(f"paper-scale group, session {s}: {sn:.1f} dB")
        assert sn >= BOUND["fp16"]


def test_unsupported_shapes_are_rejected():
    for args in (("fp32", 64, 4, 16, 100, 8), ("fp16", 64, 3, 16, 100, 8), ("fp16", 64, 4, 12, 100, 8),
                 ("fp16", 64, 4, 16, 100, 12), ("fp16", 64, 4, 8, 100, 16), ("fp16", 48, 4, 16, 100, 8),
                 ("fp16", 64, 4, 32, 100, 1), ("fp16", 64, 4, 16, 100, 3)):
        with pytest.raises(U.ConvError) as ei:
            U.Group(*args)
        assert ei.value.code == U.CONV_E_INVAL
    with U.Group("fp16", 64, 4, 16, 100, 8) as g:
        with pytest.raises(U.ConvError) as ei:
            g.process(np.zeros((8, 4, 64), np.float32))
        assert ei.value.code == U.CONV_E_STATE


def test_fp16_group_saturates_instead_of_overflowing():
    """Input spectra beyond the FP16 range saturate (the delay line is stored
    unscaled): outputs stay finite, and BF16 handles the same input."""
    S, n_in, n_out, taps, B, nb = 8, 4, 16, 500, 256, 6
    h, x = group_case(12, S, n_in, n_out, taps, B, nb)
    x = (x * 1.0e4).astype(np.float32)  # |X| up to ~2e5 > 65504
    with U.Group("fp16", B, n_in, n_out, taps, S) as g:
        g.set_filters(h)
        y = g.run(x)
    assert np.all(np.isfinite(y))
    with U.Group("bf16", B, n_in, n_out, taps, S) as g:
        g.set_filters(h)
        yb = g.run(x)
    assert min(snr_db(yb[s], upols(h, x[s], B)) for s in range(S)) >= BOUND["bf16"]

"""The multi-block host call (conv_process_blocks) is the block-by-block
stream: bit-exact against conv_process_block over chunk boundaries, for the
plain, reduced-precision and non-uniformly partitioned engines, and the
stream continues across calls."""

import os

import numpy as np
import pytest

from gpu_helpers import snr_db
from oracle import upols
from paper_2509_04390_gb300 import build, signals
from paper_2509_04390_gb300 import upols as U

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def engine_lib():
    if not os.path.exists(build.lib_path()):
        build.build()
    U.load()


@pytest.mark.parametrize(
    "B,taps,nb,precision,far",
    [(16, 700, 300, "fp32", 0), (64, 3000, 40, "fp16", 0), (64, 3000, 260, "fp32", 256), (256, 4000, 1, "fp32", 0)],
)
def test_render_equals_block_calls(B, taps, nb, precision, far):
    w = signals.random_case(700 + nb, 2, 3, taps, B, nb, decay_s=0.05)
    with U.Engine(w.fs, B, 2, 3, taps, precision, far_block=far) as e:
        e.set_filters(w.h)
        y_blocks = e.run(w.x)
        e.reset()
        y_render = e.render(w.x)
    assert np.array_equal(y_blocks, y_render)
    if precision == "fp32":
        assert snr_db(y_render, upols(w.h.astype(np.float64), w.x.astype(np.float64), B)) >= 120.0


def test_render_continues_the_stream():
    w = signals.random_case(710, 2, 3, 2000, 64, 50, decay_s=0.05)
    B = w.block
    with U.Engine(w.fs, B, 2, 3, 2000) as e:
        e.set_filters(w.h)
        y_all = e.render(w.x)
        e.reset()
        first = e.render(np.ascontiguousarray(w.x[:, : 20 * B]))
        rest = np.empty((3, 30 * B), np.float32)
        for b in range(30):
            rest[:, b * B : (b + 1) * B] = e.process(np.ascontiguousarray(w.x[:, (20 + b) * B : (21 + b) * B]))
    assert np.array_equal(y_all, np.concatenate([first, rest], axis=1))


def test_render_rejects_bad_lengths():
    with U.Engine(48000, 64, 1, 1, 100) as e:
        e.set_filters(np.ones((1, 1, 100), np.float32))
        with pytest.raises(ValueError):
            U.conv_process_blocks(e.h, np.zeros((1, 100), np.float32), np.zeros((1, 100), np.float32))

"""Serving: a session's output is the same alone and in the mix.

A session is served on the 128-sample tick among other sessions that arrive
and depart (blocks 128 and 256, some with a feedback canceller); its output
must be bit-identical to the same session processed on its own, because every
reduction in the engine has a fixed order whatever else is batched with it.
"""

import os

import numpy as np
import pytest

from gpu_helpers import snr_db
from oracle import afc_closed_loop, upols
from paper_2509_04390_gb300 import build, serve, signals
from paper_2509_04390_gb300 import upols as U

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def engine_lib():
    if not os.path.exists(build.lib_path()):
        build.build()
    U.load()


def small_spec(rng, seed, afc=False, block=None):
    secs = float(rng.uniform(0.05, 0.3))
    return signals.SessionSpec(
        n_in=int(rng.integers(1, 4)), n_out=int(rng.integers(2, 9)), taps=int(secs * signals.FS),
        block=block or int(rng.choice([128, 256])), seed=seed, rt60=0.75 * secs, taps_fb=2000 if afc else 0)


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
@pytest.mark.parametrize("afc", [False, True])
def test_alone_equals_in_the_mix(precision, afc):
    pytest.importorskip("torch")
    rng = np.random.default_rng(41)
    pool = serve.FilterPool(seed=3, n_out=8, n_in=4, taps=int(0.3 * signals.FS) + 1)
    watched = small_spec(rng, 1000, afc=afc, block=256)
    x = watched.signal(12)
    h = pool.filters(watched)
    f = watched.paths() if afc else None

    # alone
    e = U.Engine(signals.FS, 256, watched.n_in, watched.n_out, watched.taps, precision, serve.BATCH_TILING)
    e.set_filters(h)
    blocks = []
    if afc:
        e.set_paths(f)
        for b in range(12):
            blocks.append(e.process_afc(np.ascontiguousarray(x[:, b * 256 : (b + 1) * 256])).copy())
    else:
        for b in range(12):
            blocks.append(e.process(np.ascontiguousarray(x[:, b * 256 : (b + 1) * 256])).copy())
    alone = np.concatenate(blocks, axis=1)
    e.close()

    # in the mix: others arrive and depart around it
    srv = serve.Server(precision, budget_bytes=2 << 30)
    others = [srv.admit(sp, pool.filters(sp)) for sp in (small_spec(rng, 2000 + i, afc=(i % 2 == 1)) for i in range(3))]
    srv.run_tick()
    w = srv.admit(watched, h, paths=f, x=x, keep_outputs=True)
    assert w is not None
    tick = 0
    while w.blocks < 12:
        srv.run_tick()
        tick += 1
        if tick == 5:
            srv.depart(others[0])
        if tick == 9:
            late = small_spec(rng, 3000, afc=True)
            srv.admit(late, pool.filters(late))
        assert tick < 100
    mixed = np.concatenate(w.outputs, axis=1)
    srv.close()
    np.testing.assert_array_equal(mixed, alone)
    # and the served output against the FP64 oracle: UPOLS of the session's input,
    # or with a canceller the loop of Sec. 5 fed the session's microphone blocks
    x64 = x[:, : 12 * 256].astype(np.float64)
    if afc:
        ref, _, _ = afc_closed_loop(h, np.zeros((watched.n_in, watched.n_out, 1)), f, x64, 256)
    else:
        ref = upols(h.astype(np.float64), x64, 256)
    s = snr_db(mixed, ref)
    print(f"served {precision} afc={afc}: {s:.1f} dB against the oracle")
    assert s >= {"fp32": 120.0, "fp16": 60.0}[precision]


def test_admission_respects_the_memory_budget():
    pytest.importorskip("torch")
    rng = np.random.default_rng(5)
    pool = serve.FilterPool(seed=3, n_out=8, n_in=4, taps=int(0.3 * signals.FS) + 1)
    sp = small_spec(rng, 1)
    fp = U.conv_footprint("fp32", sp.block, sp.n_in, sp.n_out, sp.taps, sp.taps_fb)
    srv = serve.Server("fp32", budget_bytes=int(2.5 * fp))
    assert srv.admit(sp, pool.filters(sp)) is not None
    assert srv.admit(sp, pool.filters(sp)) is not None
    assert srv.admit(sp, pool.filters(sp)) is None  # a third does not fit
    assert srv.rejected == 1
    assert srv.used <= srv.budget
    srv.depart(srv.sessions[0])
    assert srv.admit(sp, pool.filters(sp)) is not None  # room again after a departure
    srv.close()


@pytest.mark.parametrize(
    "precision,block,n_in,n_out,taps,taps_fb",
    [("fp32", 128, 4, 16, 48000, 0), ("fp16", 256, 2, 8, 100000, 24000), ("bf16", 64, 1, 33, 5000, 700)],
)
def test_footprint_matches_what_an_engine_holds(precision, block, n_in, n_out, taps, taps_fb):
    """conv_footprint (host-only, the admission figure) against the device bytes
    a created engine reports, within the host-side staging it leaves out."""
    fp = U.conv_footprint(precision, block, n_in, n_out, taps, taps_fb)
    with U.Engine(48000, block, n_in, n_out, taps, precision) as e:
        if taps_fb:
            e.set_paths(np.zeros((n_in, n_out, taps_fb), np.float32))
        held = e.info()["device_bytes"]
    print(f"footprint {fp} vs held {held}")
    assert abs(fp - held) <= max(4096, 0.02 * held)


def test_admission_by_hbm_load():
    pytest.importorskip("torch")
    rng = np.random.default_rng(6)
    pool = serve.FilterPool(seed=4, n_out=8, n_in=4, taps=int(0.3 * signals.FS) + 1)
    sp = small_spec(rng, 2)
    tb = serve.tick_bytes(sp, "fp16")
    # a load budget of 2.5 sessions' bytes per tick, expressed as a fraction of the bandwidth
    frac = 2.5 * tb / (serve.DEFAULT_HBM_GBS * 1e9 * 128 / signals.FS)
    srv = serve.Server("fp16", load_frac=frac)
    assert srv.admit(sp, pool.filters(sp)) is not None
    assert srv.admit(sp, pool.filters(sp)) is not None
    assert srv.admit(sp, pool.filters(sp)) is None
    assert srv.rejected_load == 1 and srv.rejected == 0
    srv.depart(srv.sessions[0])
    assert abs(srv.load - tb) < 1e-6 * tb
    assert srv.admit(sp, pool.filters(sp)) is not None
    srv.close()

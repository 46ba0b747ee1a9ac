"""The autotuner on the GPU: it times candidates on the real engine, caches the
winner, and an engine built with ``tiling="tuned"`` uses that tiling and still
matches the FP64 oracle."""

import os

import numpy as np
import pytest

from gpu_helpers import snr_db
from oracle import upols
from paper_2509_04390_gb300 import autotune as A
from paper_2509_04390_gb300 import build, signals
from paper_2509_04390_gb300 import upols as U

pytestmark = pytest.mark.gpu

BOUND = {"fp32": 120.0, "fp16": 60.0}


@pytest.fixture(scope="module", autouse=True)
def engine_lib():
    if not os.path.exists(build.lib_path()):
        build.build()
    U.load()


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
def test_tuned_engine_matches_the_oracle(precision, tmp_path, monkeypatch):
    pytest.importorskip("torch")
    monkeypatch.setenv(A.CACHE_ENV, str(tmp_path / "tiling.json"))
    w = signals.random_case(5100, 3, 20, 6000, 64, 40, decay_s=0.05)
    entry = A.tune(precision, w.block, w.n_in, w.n_out, w.taps, budget_s=4.0, steps=50)
    assert entry["candidates_timed"] >= 2 and entry["seconds_per_block"] > 0
    assert entry["planner_seconds_per_block"] is not None
    t = A.lookup(precision, w.block, w.n_in, w.n_out, w.taps, A.device_sms())
    assert t == entry["tiling"]
    with U.Engine(w.fs, w.block, w.n_in, w.n_out, w.taps, precision, "tuned") as e:
        info = e.info()
        if t.get("stages"):
            assert info["mac_stages"] == min(t["stages"], info["mac_stages"])
        if t.get("bin_tile"):
            assert info["mac_bin_tile"] == t["bin_tile"]
        e.set_filters(w.h)
        y = e.run(w.x)
    ref = upols(w.h.astype(np.float64), w.x.astype(np.float64), w.block)
    s = snr_db(y, ref)
    print(f"tuned {precision}: {t} ({entry['seconds_per_block'] * 1e6:.1f} us per block, planner "
          f"{entry['planner_seconds_per_block'] * 1e6:.1f} us), {s:.1f} dB against the oracle")
    assert s >= BOUND[precision]


def test_tuned_group_matches_the_oracle(tmp_path, monkeypatch):
    pytest.importorskip("torch")
    monkeypatch.setenv(A.CACHE_ENV, str(tmp_path / "tiling.json"))
    rng = np.random.default_rng(5101)
    S, n_in, n_out, taps, B = 8, 4, 16, 3000, 64
    entry = A.tune_group("fp16", B, n_in, n_out, taps, S, budget_s=4.0, steps=50)
    t = A.lookup_group("fp16", B, n_in, n_out, taps, S, A.device_sms())
    assert t == entry["tiling"]
    h = (rng.standard_normal((n_out, n_in, taps)) / np.sqrt(taps) * 4.0).astype(np.float32)
    x = (rng.standard_normal((S, n_in, 16 * B)) * 0.1).astype(np.float32)
    with U.Group("fp16", B, n_in, n_out, taps, S, "tuned") as g:
        if t.get("ctas"):
            assert g.info()["mac_ctas"] <= t["ctas"]
        g.set_filters(h)
        y = g.run(x)
    s = min(snr_db(y[i], upols(h.astype(np.float64), x[i].astype(np.float64), B)) for i in range(S))
    print(f"tuned group: {t}, worst session {s:.1f} dB against the oracle")
    assert s >= 60.0

"""The autotuner's host side: candidate enumeration and the cache (no GPU).

Every candidate must pass the engine's host-side plan replay
(``conv_plan_check``), the planner's own choice comes first, and a cache entry
written for a shape is found again for exactly that shape.
"""

import json
import os

import pytest

from paper_2509_04390_gb300 import autotune as A
from paper_2509_04390_gb300 import build
from paper_2509_04390_gb300 import upols as U


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not os.path.exists(build.lib_path()):
        build.build()
    return U.load()


@pytest.mark.parametrize("precision", ["fp32", "fp16", "bf16"])
@pytest.mark.parametrize("block,n_in,n_out,taps", [(256, 4, 16, 384000), (64, 2, 5, 3000), (1024, 1, 33, 50000)])
def test_candidates_pass_the_plan_replay(precision, block, n_in, n_out, taps):
    c = A.candidates(precision, block, n_in, n_out, taps, 152)
    assert c[0] == {}
    assert len(c) > 10
    keys = [tuple(sorted(t.items())) for t in c]
    assert len(set(keys)) == len(keys)
    for t in c:
        U.conv_plan_check(precision, block, n_in, n_out, taps, 152, **t)  # raises if rejected
        if precision != "fp32":
            assert t.get("kernel", "tma") == "tma"  # reduced precision has only the TMA MAC
        if "bin_tile" in t:
            assert 16 <= t["bin_tile"] <= block


def test_candidates_drop_what_the_replay_rejects(monkeypatch):
    real = U.conv_plan_check

    def picky(precision, block, n_src, n_dst, taps, num_sms=152, **t):
        if t.get("warps") == 16:
            raise U.ConvError(U.CONV_E_INVAL, "rejected for the test")
        return real(precision, block, n_src, n_dst, taps, num_sms, **t)

    monkeypatch.setattr(U, "conv_plan_check", picky)
    c = A.candidates("fp16", 256, 4, 16, 384000, 152)
    assert len(c) > 5
    assert all(t.get("warps") != 16 for t in c)


def test_group_candidates_pass_the_plan_replay():
    c = A.group_candidates("fp16", 256, 4, 16, 384000, 8, 152)
    assert c[0] == {} and len(c) > 5
    for t in c[1:]:
        U.conv_group_plan_check("fp16", 256, 4, 16, 384000, 8, 152, t)
        assert t["ctas"] <= 152


def test_cache_round_trip(tmp_path):
    path = str(tmp_path / "sub" / "tiling.json")
    assert A.lookup("fp16", 256, 4, 16, 384000, 152, path=path) is None  # no file yet
    t = {"kernel": "tma", "bin_tile": 32, "stages": 3, "stage_kib": 32, "warps": 8}
    A.save_entry(A.key("fp16", 256, 4, 16, 384000, 152), {"tiling": t, "seconds_per_block": 1e-5}, path)
    A.save_entry(A.key("fp32", 128, 4, 16, 384000, 152), {"tiling": {"kernel": "direct1"}}, path)
    assert A.lookup("fp16", 256, 4, 16, 384000, 152, path=path) == t
    assert A.lookup("fp32", 128, 4, 16, 384000, 152, path=path) == {"kernel": "direct1"}
    # the key holds the partition count, not the tap count: same K, same entry
    assert A.lookup("fp16", 256, 4, 16, 383999, 152, path=path) == t
    # other shapes, precisions and SM counts are not matched
    assert A.lookup("bf16", 256, 4, 16, 384000, 152, path=path) is None
    assert A.lookup("fp16", 256, 4, 16, 384000, 148, path=path) is None
    assert A.lookup("fp16", 256, 4, 8, 384000, 152, path=path) is None
    with open(path) as f:
        assert len(json.load(f)) == 2
    A.save_entry(A.group_key("fp16", 256, 4, 16, 384000, 8, 152), {"tiling": {"ctas": 136}}, path)
    assert A.lookup_group("fp16", 256, 4, 16, 384000, 8, 152, path=path) == {"ctas": 136}


def test_cache_ignores_a_damaged_file(tmp_path):
    path = str(tmp_path / "tiling.json")
    with open(path, "w") as f:
        f.write("{not json")
    assert A.load_cache(path) == {}
    assert A.lookup("fp32", 256, 4, 16, 384000, 152, path=path) is None
    A.save_entry("k", {"tiling": {}}, path)  # a write replaces it
    assert A.load_cache(path) == {"k": {"tiling": {}}}


def test_cache_path_from_the_environment(monkeypatch, tmp_path):
    monkeypatch.setenv(A.CACHE_ENV, str(tmp_path / "x.json"))
    assert A.cache_path() == str(tmp_path / "x.json")
    assert A.cache_path("/explicit.json") == "/explicit.json"

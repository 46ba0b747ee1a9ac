"""The C-ABI library builds, loads and exports every entry point of include/conv.h.

No compute calls: these run on machines without a GPU.
"""

import os
import re

import numpy as np
import pytest

from paper_2509_04390_gb300 import build, upols

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
        text = re.sub(r"#[^\n]*", " ", text)
        text = re.sub(r"typedef[^;]*;", " ", text)
        text = re.sub(r"typedef\s+struct\s+\w+\s*\{.*?\}\s*\w+\s*;", " ", text, flags=re.S)
        for m in re.finditer(r"\b([A-Za-z_]\w*)\s*\(([^;{}]*)\)\s*;", text):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(build.lib_path()):
        build.build()
    return upols.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in (
        "conv_create",
        "conv_set_precision",
        "conv_set_filters",
        "afc_set_paths",
        "conv_process_block",
        "conv_process_block_async",
        "afc_process_block",
        "conv_reset",
        "conv_destroy",
        "conv_last_error",
    ):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in sorted(declared_functions()) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_header():
    for n in declared_functions():
        assert hasattr(upols, n), n


def test_null_handles_are_rejected(lib):
    assert lib.conv_reset(None) == upols.CONV_E_INVAL
    assert lib.conv_set_filters(None, None) == upols.CONV_E_INVAL
    assert lib.conv_process_block(None, None, None) == upols.CONV_E_INVAL
    assert "null" in upols.conv_last_error()
    lib.conv_destroy(None)  # NULL-safe


def test_host_graph_calls_check_their_handle(lib):
    import ctypes

    assert lib.conv_set_host_graph(None, 1) == upols.CONV_E_INVAL
    m, n = ctypes.c_int(-1), ctypes.c_longlong(-1)
    assert lib.conv_get_host_graph(None, ctypes.byref(m), ctypes.byref(n)) == upols.CONV_E_INVAL
    assert (m.value, n.value) == (-1, -1)  # untouched
    assert upols.HOST_GRAPH_MODES == {"off": 0, "auto": 1, "always": 2}


def test_host_pointers_are_checked_and_exact():
    """The binding's array-address marshalling (no arithmetic: the address of
    the caller's buffer, after its dtype, layout, shape and writability are
    checked)."""
    a = np.arange(8, dtype=np.float32).reshape(2, 4)
    assert upols._host_ptr(a, (2, 4)) == a.ctypes.data
    assert upols._host_ptr(a, (2, 4), True) == a.ctypes.data
    r = a.copy()
    r.flags.writeable = False
    assert upols._host_ptr(r, (2, 4)) == r.ctypes.data  # read-only input
    with pytest.raises(ValueError):
        upols._host_ptr(r, (2, 4), True)  # read-only output
    with pytest.raises(ValueError):
        upols._host_ptr(a, (4, 2))
    with pytest.raises(TypeError):
        upols._host_ptr(a.astype(np.float64), (2, 4))
    with pytest.raises(TypeError):
        upols._host_ptr(np.asfortranarray(np.ones((3, 4), np.float32)), (3, 4))
    with pytest.raises(TypeError):
        upols._host_ptr([1.0, 2.0], (2,))
    z = np.zeros((0, 4), np.float32)
    assert upols._host_ptr(z, (0, 4), True) == z.__array_interface__["data"][0]
    v = np.zeros((4, 8), np.float32)[1:3]  # a contiguous view: its own start address
    assert upols._host_ptr(v, (2, 8)) == v.ctypes.data


def test_invalid_sizes_fail_before_touching_a_device(lib):
    assert not lib.conv_create(48000.0, 100, 1, 2, 1000)  # not a power of two
    assert "power of two" in upols.conv_last_error()
    assert not lib.conv_create(48000.0, 8192, 1, 2, 1000)  # above 4096
    assert not lib.conv_create(48000.0, 256, 0, 2, 1000)
    assert not lib.conv_create(48000.0, 256, 1, 2, 0)
    assert not lib.conv_create(-1.0, 256, 1, 2, 10)


@pytest.mark.parametrize("precision", ["fp32", "fp16", "bf16"])
def test_mac_plan_addresses_stay_in_bounds(lib, precision):
    # every tiling the engine would pick for these sizes replays in bounds
    shapes = [
        (1, 1, 1),
        (1, 2, 48000),
        (4, 16, 384000),
        (16, 4, 24000),
        (3, 20, 1000),
        (2, 5, 4000),
        (8, 32, 200000),
        (1, 64, 720000),
        (5, 7, 2048),
        (4, 33, 3000),
        (7, 1024, 100),
        (1024, 3, 50),
    ]
    for B in (16, 32, 64, 128, 256, 512, 1024, 2048, 4096):
        for n_src, n_dst, taps in shapes:
            for sms in (152, 148, 8):
                for kernel in ("auto", "direct1", "direct2"):
                    upols.conv_plan_check(precision, B, n_src, n_dst, taps, sms, kernel)


def test_tiling_overrides_stay_in_bounds(lib):
    # the autotuner's candidate space at paper scale and a small shape
    for precision in ("fp32", "fp16"):
        for B in (64, 128, 256, 512):
            for n_src, n_dst, taps in ((4, 16, 384000), (3, 20, 1000)):
                for bt in (16, 32, 64, 128, 256):
                    for stages, kib in ((2, 64), (3, 32), (4, 48), (5, 32), (8, 16), (8, 24)):
                        for splits, nw in ((0, 0), (1, 8), (9, 16), (38, 8), (1000000, 16)):
                            for kernel, order in (("tma", 1), ("tma", 2), ("direct1", 0), ("direct2", 0)):
                                upols.conv_plan_check(
                                    precision, B, n_src, n_dst, taps, 152, kernel, bt, stages, kib, splits, nw, order
                                )


def test_canceller_split_counts_replay_clean(lib):
    # the split counts an engine with a feedback canceller uses: two thirds of
    # the synthesis default and two for the canceller's own tail
    for precision in ("fp32", "fp16", "bf16"):
        for B in (16, 64, 128, 256, 512, 1024, 4096):
            for n_src, n_dst, taps in ((4, 16, 384000), (16, 4, 24000), (2, 3, 3000), (8, 32, 200000)):
                for splits in (1, 2, 3, 6, 12, 24):
                    upols.conv_plan_check(precision, B, n_src, n_dst, taps, 152, "tma", 0, 0, 0, splits)


def test_tiling_override_arguments_are_validated(lib):
    with pytest.raises(upols.ConvError):
        upols.conv_plan_check("fp32", 256, 4, 16, 384000, 152, 0, 24)  # bin tile not a power of two
    with pytest.raises(upols.ConvError):
        upols.conv_plan_check("fp32", 256, 4, 16, 384000, 152, 7)  # unknown kernel


def test_group_plans_replay_clean_over_shapes(lib):
    """Host replay of every copy address of a shared-filter group's block, over
    the supported shapes, precisions and SM counts."""
    from paper_2509_04390_gb300 import upols as U

    n = 0
    for prec in ("fp16", "bf16"):
        for B in (16, 64, 256, 1024, 4096):
            for n_in in (1, 2, 4, 8):
                for n_out in (8, 16, 32):
                    for S in (1, 2, 4, 8, 16, 32):
                        if not 8 <= (128 // n_out) * S <= 128:
                            continue
                        for taps in (1, 257, 3000, 384000):
                            for sms in (152, 20):
                                U.conv_group_plan_check(prec, B, n_in, n_out, taps, S, sms)
                                n += 1
    assert n > 500


def test_group_tilings_replay_clean(lib):
    from paper_2509_04390_gb300 import upols as U

    for tiling in ({"ctas": 1}, {"ctas": 7, "stage_k_steps": 1, "stages": 2}, {"ctas": 37, "stage_k_steps": 2, "stages": 4},
                   {"ctas": 152, "stage_k_steps": 4, "stages": 2, "tail_streams": 1}, {"ctas": 100000}):
        for B, taps in ((64, 2500), (256, 384000), (16, 1), (4096, 100000)):
            U.conv_group_plan_check("fp16", B, 4, 16, taps, 8, 152, tiling)
    for bad in ({"ctas": -1}, {"stage_k_steps": 5}, {"stages": 1}, {"stages": 9}, {"tail_streams": 3},
                {"stage_k_steps": 4, "stages": 8}):
        with pytest.raises(U.ConvError):
            U.conv_group_plan_check("fp16", 256, 4, 16, 384000, 8, 152, bad)


def test_group_rejects_unsupported_shapes_on_the_host(lib):
    from paper_2509_04390_gb300 import upols as U

    for args in (("fp32", 64, 4, 16, 100, 8), ("fp16", 64, 3, 16, 100, 8), ("fp16", 64, 4, 12, 100, 8),
                 ("fp16", 64, 4, 16, 100, 12), ("fp16", 64, 4, 8, 100, 16), ("fp16", 48, 4, 16, 100, 8),
                 ("fp16", 64, 4, 32, 100, 1), ("fp16", 64, 4, 16, 100, 3)):
        with pytest.raises(U.ConvError) as ei:
            U.conv_group_plan_check(*args)
        assert ei.value.code == U.CONV_E_INVAL

"""Thin ctypes binding of the engine's C ABI (``include/conv.h``).

Function names match the C entry points; this module only marshals arguments
(numpy arrays for host buffers, raw device addresses or torch tensors for the
``*_async`` forms) and turns negative status codes into ``ConvError``.  All
computation runs in the CUDA library; if it has not been built, loading fails
with an error instead of falling back to anything else.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

CONV_OK = 0
CONV_E_INVAL = -1
CONV_E_STATE = -2
CONV_E_NOMEM = -3
CONV_E_CUDA = -4
CONV_E_TIMEOUT = -5
CONV_E_UNSTABLE = -6

CONV_FP32 = 0
CONV_FP16 = 1
CONV_BF16 = 2

PRECISIONS = {"fp32": CONV_FP32, "fp16": CONV_FP16, "bf16": CONV_BF16}


class ConvError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[{code}] {msg}")
        self.code = code


CONV_KERNEL_AUTO = 0
CONV_KERNEL_TMA = 1
CONV_KERNEL_DIRECT1 = 2
CONV_KERNEL_DIRECT2 = 3
KERNELS = {"auto": 0, "tma": 1, "direct1": 2, "direct2": 3}


class conv_tiling(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int) for n in ("kernel", "bin_tile", "stages", "stage_kib", "splits", "warps", "order")]


ORDERS = {"auto": 0, "contiguous": 1, "interleaved": 2}


def make_tiling(kernel=0, bin_tile=0, stages=0, stage_kib=0, splits=0, warps=0, order=0):
    return conv_tiling(
        KERNELS.get(kernel, kernel), bin_tile, stages, stage_kib, splits, warps, ORDERS.get(order, order)
    )


class conv_info(ctypes.Structure):
    _fields_ = [
        (name, ctypes.c_longlong)
        for name in (
            "block",
            "n_in",
            "n_out",
            "taps",
            "K",
            "taps_fb",
            "K_fb",
            "precision",
            "mac_bytes",
            "mac_fb_bytes",
            "mac_ctas",
            "mac_splits",
            "mac_smem",
            "device_bytes",
            "kernels_per_block",
            "kernels_per_afc_block",
            "mac_bin_tile",
            "mac_stages",
            "mac_stage_bytes",
            "mac_warps",
            "mac_kernel",
            "afc_adaptive",
            "far_block",
            "K_far",
            "mac_far_bytes",
            "fft_size",
            "l2_keep_bytes",
        )
    ]

    def as_dict(self):
        return {name: int(getattr(self, name)) for name, _ in self._fields_}


class conv_group_info(ctypes.Structure):
    _fields_ = [
        (name, ctypes.c_longlong)
        for name in (
            "block", "n_in", "n_out", "taps", "sessions", "precision", "K", "ring_slots", "bins_per_group", "groups",
            "splits", "k_steps", "stage_k_steps", "stages", "mac_ctas", "mac_smem", "tmem_cols", "mac_bytes",
            "device_bytes", "kernels_per_block", "tail_streams", "tail_ctas", "acc_buffers",
        )
    ]

    def as_dict(self):
        return {name: int(getattr(self, name)) for name, _ in self._fields_}


CONV_STATS_BUCKETS = 24


class conv_stats(ctypes.Structure):
    _fields_ = [
        ("blocks", ctypes.c_longlong),
        ("timed_calls", ctypes.c_longlong),
        ("deadline_misses", ctypes.c_longlong),
        ("max_latency_us", ctypes.c_double),
        ("sum_latency_us", ctypes.c_double),
        ("latency_hist", ctypes.c_longlong * CONV_STATS_BUCKETS),
        ("device_errors", ctypes.c_longlong),
        ("guard_trips", ctypes.c_longlong),
    ]

    def as_dict(self):
        d = {n: getattr(self, n) for n, _ in self._fields_ if n != "latency_hist"}
        d["latency_hist"] = [int(v) for v in self.latency_hist]
        return d


class conv_group_tiling(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int) for n in ("ctas", "stage_k_steps", "stages", "tail_streams")]


_lib = None


def lib_path() -> str:
    return _build.lib_path()


def load():
    """Load the engine library (raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if not os.path.exists(path):
        raise RuntimeError(
            f"CUDA engine library not found at {path}; build it with "
            "`python -m paper_2509_04390_gb300.build` (there is no CPU fallback)"
        )
    L = ctypes.CDLL(path)
    vp, i, ll, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong, ctypes.c_double
    sig = {
        "conv_create": (vp, [d, i, i, i, ll]),
        "conv_set_precision": (i, [vp, i]),
        "afc_set_spectrum_reuse": (i, [vp, i]),
        "conv_set_filters": (i, [vp, vp]),
        "conv_set_tiling": (i, [vp, ctypes.POINTER(conv_tiling)]),
        "afc_set_paths": (i, [vp, vp, ll]),
        "conv_process_block": (i, [vp, vp, vp]),
        "conv_process_block_async": (i, [vp, vp, vp, vp]),
        "conv_process_blocks": (i, [vp, vp, vp, ll]),
        "afc_process_block": (i, [vp, vp, vp, vp]),
        "afc_process_block_async": (i, [vp, vp, vp, vp, vp]),
        "afc_set_guard": (i, [vp, d]),
        "afc_set_adaptation": (i, [vp, d, d, d]),
        "conv_set_far_block": (i, [vp, i]),
        "conv_far_engine": (vp, [vp]),
        "afc_get_path_spectra": (i, [vp, vp]),
        "conv_reset": (i, [vp]),
        "conv_synchronize": (i, [vp]),
        "conv_get_info": (i, [vp, ctypes.POINTER(conv_info)]),
        "conv_profile_enable": (i, [vp, i]),
        "conv_profile_flush_l2": (i, [vp, ll]),
        "conv_set_l2_keep": (i, [vp, ll]),
        "conv_group_set_l2_keep": (i, [vp, ll]),
        "conv_profile_read": (i, [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong)]),
        "conv_plan_check": (i, [i, i, i, i, ll, i, ctypes.POINTER(conv_tiling)]),
        "conv_fdl_mac_noalloc": (i, [vp, vp, i, i, i, ll, ll, vp, vp]),
        "conv_fdl_mac_noalloc_status": (i, [vp]),
        "conv_join_async": (i, [vp, vp]),
        "conv_batch_join_async": (i, [vp, vp]),
        "conv_group_join_async": (i, [vp, vp]),
        "conv_get_stats": (i, [vp, ctypes.POINTER(conv_stats)]),
        "conv_reset_stats": (i, [vp]),
        "conv_set_host_graph": (i, [vp, i]),
        "conv_get_host_graph": (i, [vp, ctypes.POINTER(i), ctypes.POINTER(ll)]),
        "conv_inject_wait_timeout": (i, [vp, ll]),
        "conv_footprint": (ll, [i, i, i, i, ll, ll, i]),
        "conv_batch_create": (vp, [i]),
        "conv_batch_add": (i, [vp, vp]),
        "conv_batch_remove": (i, [vp, vp]),
        "conv_batch_size": (i, [vp]),
        "conv_batch_process_async": (i, [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), vp]),
        "conv_batch_process_some_async": (i, [vp, i, ctypes.POINTER(i), ctypes.POINTER(vp), ctypes.POINTER(vp), vp]),
        "conv_batch_synchronize": (i, [vp]),
        "conv_batch_set_persistent": (i, [vp, i]),
        "conv_batch_step_bytes": (ll, [vp]),
        "conv_batch_destroy": (None, [vp]),
        "conv_group_create": (vp, [i, i, i, i, ll, i]),
        "conv_group_create_tiled": (vp, [i, i, i, i, ll, i, ctypes.POINTER(conv_group_tiling)]),
        "conv_group_set_filters": (i, [vp, vp]),
        "conv_group_process_async": (i, [vp, vp, vp, vp]),
        "conv_group_process": (i, [vp, vp, vp]),
        "conv_group_process_blocks": (i, [vp, vp, vp, ll]),
        "conv_group_reset": (i, [vp]),
        "conv_group_synchronize": (i, [vp]),
        "conv_group_get_info": (i, [vp, ctypes.POINTER(conv_group_info)]),
        "conv_group_plan_check": (i, [i, i, i, i, ll, i, i, ctypes.POINTER(conv_group_tiling)]),
        "conv_group_profile_enable": (i, [vp, i]),
        "conv_group_profile_read": (i, [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong)]),
        "conv_group_destroy": (None, [vp]),
        "conv_destroy": (None, [vp]),
        "conv_last_error": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def conv_last_error() -> str:
    return load().conv_last_error().decode(errors="replace")


def _check(rc: int) -> int:
    if rc != CONV_OK:
        raise ConvError(rc, conv_last_error())
    return rc


_F32 = np.dtype(np.float32)


def _host_ptr(a: np.ndarray, shape, writable=False):
    """Address of a C-contiguous float32 array of the given shape.

    Per-block calls pay for this twice, so it avoids `ndarray.ctypes` (about
    1.5-2.5 us per array): a writable array's buffer is taken as is, a
    read-only one's address comes from its array interface."""
    if not isinstance(a, np.ndarray) or a.dtype != _F32 or not a.flags.c_contiguous:
        raise TypeError("expected a C-contiguous float32 numpy array")
    if a.shape != tuple(shape):
        raise ValueError(f"expected shape {tuple(shape)}, got {a.shape}")
    if writable and not a.flags.writeable:
        raise ValueError("output array is read-only")
    if a.flags.writeable and a.size:
        return ctypes.addressof(ctypes.c_char.from_buffer(a))
    return a.__array_interface__["data"][0]


def _dev_ptr(t):
    """Device address of a torch tensor (float32, contiguous, CUDA) or an int."""
    if t is None:
        return None
    if isinstance(t, int):
        return ctypes.c_void_p(t)
    import torch

    if not t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous():
        raise TypeError("expected a contiguous float32 CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


# ---------------------------------------------------------------- C names


def conv_create(fs: float, block: int, n_in: int, n_out: int, taps: int):
    h = load().conv_create(float(fs), int(block), int(n_in), int(n_out), int(taps))
    if not h:
        raise ConvError(CONV_E_INVAL, conv_last_error())
    return h


def conv_set_precision(h, mode):
    mode = PRECISIONS.get(mode, mode)
    return _check(load().conv_set_precision(h, int(mode)))


def afc_set_spectrum_reuse(h, on: bool = True):
    return _check(load().afc_set_spectrum_reuse(h, 1 if on else 0))


def conv_set_far_block(h, far_block: int):
    return _check(load().conv_set_far_block(h, int(far_block)))


def conv_far_engine(h):
    """Handle of the far part's engine (owned by h; for conv_get_info and profiling), or None."""
    return load().conv_far_engine(h) or None


def conv_set_tiling(h, kernel=0, bin_tile=0, stages=0, stage_kib=0, splits=0, warps=0, order=0):
    t = make_tiling(kernel, bin_tile, stages, stage_kib, splits, warps, order)
    return _check(load().conv_set_tiling(h, ctypes.byref(t)))


def conv_set_filters(h, filters: np.ndarray):
    info = conv_get_info(h)
    return _check(load().conv_set_filters(h, _host_ptr(filters, (info["n_out"], info["n_in"], info["taps"]))))


def afc_set_paths(h, paths: np.ndarray):
    info = conv_get_info(h)
    if paths.ndim != 3:
        raise ValueError("paths must be [n_in][n_out][taps_fb]")
    _host_ptr(paths, (info["n_in"], info["n_out"], paths.shape[2]))
    return _check(load().afc_set_paths(h, paths.ctypes.data_as(ctypes.c_void_p), int(paths.shape[2])))


def conv_process_block(h, inp: np.ndarray, out: np.ndarray, _shape=None):
    n_in, n_out, B = _shape if _shape else _dims(h)
    return _check(load().conv_process_block(h, _host_ptr(inp, (n_in, B)), _host_ptr(out, (n_out, B), True)))


def conv_process_blocks(h, inp: np.ndarray, out: np.ndarray, _shape=None):
    """inp [n_in][n_blocks * block], out [n_out][n_blocks * block] (float32, C-contiguous)."""
    n_in, n_out, B = _shape if _shape else _dims(h)
    T = inp.shape[1] if inp.ndim == 2 else -1
    if T <= 0 or T % B:
        raise ValueError("input length must be a positive multiple of the block size")
    return _check(
        load().conv_process_blocks(h, _host_ptr(inp, (n_in, T)), _host_ptr(out, (n_out, T), True), T // B)
    )


def conv_process_block_async(h, d_in, d_out, stream=None):
    return _check(load().conv_process_block_async(h, _dev_ptr(d_in), _dev_ptr(d_out), _stream_ptr(stream)))


def afc_process_block(h, mic: np.ndarray, out: np.ndarray, e_out: np.ndarray | None = None, _shape=None):
    n_in, n_out, B = _shape if _shape else _dims(h)
    ep = _host_ptr(e_out, (n_in, B), True) if e_out is not None else None
    return _check(load().afc_process_block(h, _host_ptr(mic, (n_in, B)), _host_ptr(out, (n_out, B), True), ep))


def afc_process_block_async(h, d_mic, d_out, d_e=None, stream=None):
    return _check(
        load().afc_process_block_async(h, _dev_ptr(d_mic), _dev_ptr(d_out), _dev_ptr(d_e), _stream_ptr(stream))
    )


def afc_set_guard(h, max_rms: float):
    return _check(load().afc_set_guard(h, float(max_rms)))


def afc_set_adaptation(h, mu: float, lam: float = 0.9, delta: float = 1e-6):
    return _check(load().afc_set_adaptation(h, float(mu), float(lam), float(delta)))


def afc_get_path_spectra(h) -> np.ndarray:
    """The canceller's sub-filter spectra as complex64 [n_in][n_out][K_fb][block]
    (bin 0 holds DC in its real part and Nyquist in its imaginary part)."""
    info = conv_get_info(h)
    out = np.empty((info["n_in"], info["n_out"], info["K_fb"], info["block"], 2), dtype=np.float32)
    _check(load().afc_get_path_spectra(h, out.ctypes.data_as(ctypes.c_void_p)))
    return out[..., 0] + 1j * out[..., 1]


def conv_reset(h):
    return _check(load().conv_reset(h))


def conv_synchronize(h):
    return _check(load().conv_synchronize(h))


def conv_get_info(h) -> dict:
    info = conv_info()
    _check(load().conv_get_info(h, ctypes.byref(info)))
    return info.as_dict()


def conv_set_l2_keep(h, nbytes: int):
    return _check(load().conv_set_l2_keep(h, int(nbytes)))


def conv_group_set_l2_keep(g, nbytes: int):
    return _check(load().conv_group_set_l2_keep(g, int(nbytes)))


def conv_profile_flush_l2(h, nbytes: int):
    return _check(load().conv_profile_flush_l2(h, int(nbytes)))


def conv_profile_enable(h, enable: int):
    return _check(load().conv_profile_enable(h, int(enable)))


def conv_profile_read(h):
    ms = ctypes.c_double()
    n = ctypes.c_longlong()
    _check(load().conv_profile_read(h, ctypes.byref(ms), ctypes.byref(n)))
    return ms.value, n.value


def conv_plan_check(
    precision, block, n_src, n_dst, taps, num_sms=152, kernel=0, bin_tile=0, stages=0, stage_kib=0, splits=0,
    warps=0, order=0,
):
    precision = PRECISIONS.get(precision, precision)
    t = make_tiling(kernel, bin_tile, stages, stage_kib, splits, warps, order)
    return _check(
        load().conv_plan_check(
            int(precision), int(block), int(n_src), int(n_dst), int(taps), int(num_sms), ctypes.byref(t)
        )
    )


def conv_fdl_mac_noalloc(d_H, d_X, block, n_in, n_out, K, slot0, d_y, stream=None):
    return _check(
        load().conv_fdl_mac_noalloc(
            _dev_ptr(d_H), _dev_ptr(d_X), int(block), int(n_in), int(n_out), int(K), int(slot0), _dev_ptr(d_y),
            _stream_ptr(stream),
        )
    )


def conv_fdl_mac_noalloc_status(stream=None):
    return _check(load().conv_fdl_mac_noalloc_status(_stream_ptr(stream)))


def conv_join_async(h, stream=None):
    return _check(load().conv_join_async(h, _stream_ptr(stream)))


def conv_batch_join_async(b, stream=None):
    return _check(load().conv_batch_join_async(b, _stream_ptr(stream)))


def conv_group_join_async(g, stream=None):
    return _check(load().conv_group_join_async(g, _stream_ptr(stream)))


def conv_get_stats(h) -> dict:
    st = conv_stats()
    _check(load().conv_get_stats(h, ctypes.byref(st)))
    return st.as_dict()


def conv_reset_stats(h):
    return _check(load().conv_reset_stats(h))


HOST_GRAPH_MODES = {"off": 0, "auto": 1, "always": 2}


def conv_set_host_graph(h, mode):
    """mode: "off" / "auto" / "always" (or 0 / 1 / 2)."""
    return _check(load().conv_set_host_graph(h, int(HOST_GRAPH_MODES.get(mode, mode))))


def conv_get_host_graph(h) -> tuple[int, int]:
    """(mode, blocks that went through conv_process_block's graph)."""
    m, nb = ctypes.c_int(), ctypes.c_longlong()
    _check(load().conv_get_host_graph(h, ctypes.byref(m), ctypes.byref(nb)))
    return int(m.value), int(nb.value)


def conv_inject_wait_timeout(h, wait_ns: int):
    return _check(load().conv_inject_wait_timeout(h, int(wait_ns)))


def conv_footprint(precision, block, n_in, n_out, taps, taps_fb=0, num_sms=152):
    v = load().conv_footprint(
        int(PRECISIONS.get(precision, precision)), int(block), int(n_in), int(n_out), int(taps), int(taps_fb),
        int(num_sms),
    )
    if v < 0:
        raise ConvError(CONV_E_INVAL, conv_last_error())
    return int(v)


def conv_batch_create(precision="fp32"):
    b = load().conv_batch_create(int(PRECISIONS.get(precision, precision)))
    if not b:
        raise ConvError(CONV_E_INVAL, conv_last_error())
    return b


def conv_batch_add(b, h):
    return _check(load().conv_batch_add(b, h))


def conv_batch_remove(b, h):
    return _check(load().conv_batch_remove(b, h))


def conv_batch_size(b):
    return int(load().conv_batch_size(b))


def conv_batch_process_async(b, d_ins, d_outs, stream=None):
    n = len(d_ins)
    ins = (ctypes.c_void_p * n)(*[_dev_ptr(t).value for t in d_ins])
    outs = (ctypes.c_void_p * n)(*[_dev_ptr(t).value for t in d_outs])
    return _check(load().conv_batch_process_async(b, ins, outs, _stream_ptr(stream)))


def conv_batch_process_some_async(b, idx, d_ins, d_outs, stream=None):
    n = len(idx)
    ids = (ctypes.c_int * n)(*[int(v) for v in idx])
    ins = (ctypes.c_void_p * n)(*[_dev_ptr(t).value for t in d_ins])
    outs = (ctypes.c_void_p * n)(*[_dev_ptr(t).value for t in d_outs])
    return _check(load().conv_batch_process_some_async(b, n, ids, ins, outs, _stream_ptr(stream)))


def conv_batch_synchronize(b):
    return _check(load().conv_batch_synchronize(b))


def conv_batch_set_persistent(b, mode=1):
    """mode 0: one launch per stage; 1: one persistent launch per step; 2: the
    persistent step replayed from a CUDA graph."""
    return _check(load().conv_batch_set_persistent(b, int(mode)))


def conv_batch_step_bytes(b):
    return int(load().conv_batch_step_bytes(b))


def conv_batch_destroy(b):
    if b:
        load().conv_batch_destroy(b)


def conv_group_create(precision, block, n_in, n_out, taps, sessions):
    g = load().conv_group_create(
        int(PRECISIONS.get(precision, precision)), int(block), int(n_in), int(n_out), int(taps), int(sessions)
    )
    if not g:
        raise ConvError(CONV_E_INVAL, conv_last_error())
    return g


def conv_group_create_tiled(precision, block, n_in, n_out, taps, sessions, tiling=None):
    t = conv_group_tiling(**(tiling or {}))
    g = load().conv_group_create_tiled(
        int(PRECISIONS.get(precision, precision)), int(block), int(n_in), int(n_out), int(taps), int(sessions),
        ctypes.byref(t),
    )
    if not g:
        raise ConvError(CONV_E_INVAL, conv_last_error())
    return g


def conv_group_get_info(g) -> dict:
    info = conv_group_info()
    _check(load().conv_group_get_info(g, ctypes.byref(info)))
    return info.as_dict()


def conv_group_set_filters(g, filters: np.ndarray):
    i = conv_group_get_info(g)
    return _check(load().conv_group_set_filters(g, _host_ptr(filters, (i["n_out"], i["n_in"], i["taps"]))))


def conv_group_process_async(g, d_in, d_out, stream=None):
    return _check(load().conv_group_process_async(g, _dev_ptr(d_in), _dev_ptr(d_out), _stream_ptr(stream)))


def conv_group_process(g, inp: np.ndarray, out: np.ndarray, _shape=None):
    S, n_in, n_out, B = _shape if _shape else _gdims(g)
    return _check(load().conv_group_process(g, _host_ptr(inp, (S, n_in, B)), _host_ptr(out, (S, n_out, B), True)))


def conv_group_process_blocks(g, inp: np.ndarray, out: np.ndarray, _shape=None):
    """inp [sessions][n_in][n_blocks * block], out [sessions][n_out][n_blocks * block]."""
    S, n_in, n_out, B = _shape if _shape else _gdims(g)
    T = inp.shape[2] if inp.ndim == 3 else -1
    if T <= 0 or T % B:
        raise ValueError("input length must be a positive multiple of the block size")
    return _check(
        load().conv_group_process_blocks(g, _host_ptr(inp, (S, n_in, T)), _host_ptr(out, (S, n_out, T), True), T // B)
    )


def conv_group_reset(g):
    return _check(load().conv_group_reset(g))


def conv_group_synchronize(g):
    return _check(load().conv_group_synchronize(g))


def conv_group_plan_check(precision, block, n_in, n_out, taps, sessions, num_sms=152, tiling=None):
    t = conv_group_tiling(**(tiling or {}))
    return _check(
        load().conv_group_plan_check(
            int(PRECISIONS.get(precision, precision)), int(block), int(n_in), int(n_out), int(taps), int(sessions),
            int(num_sms), ctypes.byref(t),
        )
    )


def conv_group_profile_enable(g, enable: int):
    return _check(load().conv_group_profile_enable(g, int(enable)))


def conv_group_profile_read(g):
    ms = ctypes.c_double()
    n = ctypes.c_longlong()
    _check(load().conv_group_profile_read(g, ctypes.byref(ms), ctypes.byref(n)))
    return ms.value, n.value


def conv_group_destroy(g):
    if g:
        load().conv_group_destroy(g)


def _gdims(g):
    i = conv_group_get_info(g)
    return i["sessions"], i["n_in"], i["n_out"], i["block"]


def conv_destroy(h):
    if h:
        load().conv_destroy(h)


def _dims(h):
    i = conv_get_info(h)
    return i["n_in"], i["n_out"], i["block"]


# ------------------------------------------------------------ convenience


class Batch:
    """Owning wrapper of a conv_batch (sessions are Engine objects)."""

    def __init__(self, precision="fp32"):
        self.b = conv_batch_create(precision)
        self.sessions = []

    def add(self, eng):
        conv_batch_add(self.b, eng.h)
        self.sessions.append(eng)

    def remove(self, eng):
        conv_batch_remove(self.b, eng.h)
        self.sessions.remove(eng)

    def process_async(self, d_ins, d_outs, stream=None):
        conv_batch_process_async(self.b, d_ins, d_outs, stream)

    def process_some_async(self, idx, d_ins, d_outs, stream=None):
        conv_batch_process_some_async(self.b, idx, d_ins, d_outs, stream)

    def synchronize(self):
        conv_batch_synchronize(self.b)

    def set_persistent(self, mode=1):
        conv_batch_set_persistent(self.b, int(mode))

    def step_bytes(self):
        return conv_batch_step_bytes(self.b)

    def close(self):
        if self.b:
            conv_batch_destroy(self.b)
            self.b = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Group:
    """Owning wrapper of a conv_group: ``sessions`` lock-step streams sharing
    one filter set."""

    def __init__(self, precision, block, n_in, n_out, taps, sessions, tiling=None):
        if tiling == "tuned":
            from . import autotune

            tiling = autotune.lookup_group(precision, block, n_in, n_out, taps, sessions, autotune.device_sms())
        self.g = conv_group_create_tiled(precision, block, n_in, n_out, taps, sessions, tiling)
        self.shape = (int(sessions), int(n_in), int(n_out), int(block))

    def set_filters(self, h: np.ndarray):
        conv_group_set_filters(self.g, np.ascontiguousarray(h, dtype=np.float32))

    def process(self, x_blocks: np.ndarray, out: np.ndarray | None = None) -> np.ndarray:
        S, n_in, n_out, B = self.shape
        if out is None:
            out = np.empty((S, n_out, B), dtype=np.float32)
        conv_group_process(self.g, np.ascontiguousarray(x_blocks, dtype=np.float32), out, self.shape)
        return out

    def run(self, x: np.ndarray) -> np.ndarray:
        """Stream whole signals x [sessions][n_in][T] (zero-extended to whole blocks)."""
        S, n_in, n_out, B = self.shape
        T = x.shape[2]
        nb = -(-T // B)
        xp = np.zeros((S, n_in, nb * B), dtype=np.float32)
        xp[:, :, :T] = x
        y = np.empty((S, n_out, nb * B), dtype=np.float32)
        blk = np.empty((S, n_out, B), dtype=np.float32)
        for b in range(nb):
            self.process(np.ascontiguousarray(xp[:, :, b * B : (b + 1) * B]), blk)
            y[:, :, b * B : (b + 1) * B] = blk
        return y

    def render(self, x: np.ndarray) -> np.ndarray:
        """Whole signals x [sessions][n_in][T] in one multi-block call (zero-extended)."""
        S, n_in, n_out, B = self.shape
        T = x.shape[2]
        nb = -(-T // B)
        xp = np.zeros((S, n_in, nb * B), dtype=np.float32)
        xp[:, :, :T] = x
        y = np.empty((S, n_out, nb * B), dtype=np.float32)
        conv_group_process_blocks(self.g, xp, y, self.shape)
        return y

    def info(self):
        return conv_group_get_info(self.g)

    def reset(self):
        conv_group_reset(self.g)

    def close(self):
        if self.g:
            conv_group_destroy(self.g)
            self.g = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Engine:
    """Owning wrapper: ``with Engine(fs, block, n_in, n_out, taps) as e: ...``.

    ``tiling``: None (the planner's rule), a dict of ``conv_tiling`` fields, or
    "tuned": the autotuner's cached choice for this shape and GPU (the
    planner's rule when the cache has none, and in the spectrum-reuse form).
    ``reuse``: the n_f = 3 n_x spectrum-reuse form (``afc_set_spectrum_reuse``)."""

    def __init__(self, fs, block, n_in, n_out, taps, precision="fp32", tiling=None, far_block=0, reuse=False):
        self.h = conv_create(fs, block, n_in, n_out, taps)
        self.shape = (int(n_in), int(n_out), int(block))
        try:
            if precision not in ("fp32", CONV_FP32):
                conv_set_precision(self.h, precision)
            if reuse:
                afc_set_spectrum_reuse(self.h, True)
                if tiling == "tuned":
                    tiling = None
            if tiling == "tuned":
                from . import autotune

                prec = {v: k for k, v in PRECISIONS.items()}.get(precision, precision)
                tiling = autotune.lookup(prec, block, n_in, n_out, taps, autotune.device_sms())
            if tiling:
                conv_set_tiling(self.h, **tiling)
            if far_block:
                conv_set_far_block(self.h, far_block)
        except Exception:
            conv_destroy(self.h)
            raise

    def set_filters(self, h: np.ndarray):
        conv_set_filters(self.h, np.ascontiguousarray(h, dtype=np.float32))

    def set_paths(self, f: np.ndarray):
        afc_set_paths(self.h, np.ascontiguousarray(f, dtype=np.float32))

    def set_adaptation(self, mu, lam=0.9, delta=1e-6):
        afc_set_adaptation(self.h, mu, lam, delta)

    def path_spectra(self) -> np.ndarray:
        return afc_get_path_spectra(self.h)

    def process(self, x_block: np.ndarray, out: np.ndarray | None = None) -> np.ndarray:
        n_in, n_out, B = self.shape
        if out is None:
            out = np.empty((n_out, B), dtype=np.float32)
        conv_process_block(self.h, np.ascontiguousarray(x_block, dtype=np.float32), out, self.shape)
        return out

    def process_afc(self, mic_block, out=None, e_out=None):
        n_in, n_out, B = self.shape
        if out is None:
            out = np.empty((n_out, B), dtype=np.float32)
        afc_process_block(self.h, np.ascontiguousarray(mic_block, dtype=np.float32), out, e_out, self.shape)
        return out

    def run(self, x: np.ndarray) -> np.ndarray:
        """Stream a whole [n_in][T] signal block by block (zero-extended to whole blocks)."""
        n_in, n_out, B = self.shape
        T = x.shape[1]
        nb = -(-T // B)
        xp = np.zeros((n_in, nb * B), dtype=np.float32)
        xp[:, :T] = x
        y = np.empty((n_out, nb * B), dtype=np.float32)
        blk = np.empty((n_out, B), dtype=np.float32)
        for b in range(nb):
            self.process(np.ascontiguousarray(xp[:, b * B : (b + 1) * B]), blk)
            y[:, b * B : (b + 1) * B] = blk
        return y

    def render(self, x: np.ndarray) -> np.ndarray:
        """Stream a whole [n_in][T] signal in one multi-block call (zero-extended)."""
        n_in, n_out, B = self.shape
        T = x.shape[1]
        nb = -(-T // B)
        xp = np.zeros((n_in, nb * B), dtype=np.float32)
        xp[:, :T] = x
        y = np.empty((n_out, nb * B), dtype=np.float32)
        conv_process_blocks(self.h, xp, y, self.shape)
        return y

    def info(self):
        return conv_get_info(self.h)

    def stats(self):
        return conv_get_stats(self.h)

    def set_host_graph(self, mode):
        conv_set_host_graph(self.h, mode)

    def host_graph(self):
        return conv_get_host_graph(self.h)

    def reset(self):
        conv_reset(self.h)

    def close(self):
        if self.h:
            conv_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

"""The blocking host calls through their CUDA graphs against the stream path and the oracle.

The graph holds the same kernels, launch shapes and argument blocks as the
stream path (pack -> output, the next block's tail MAC beside the output), so
the two give the same bits; transitions between the graph and the stream
calls (conv_process_block_async, conv_process_blocks, a new plan, reset)
must keep the block chain intact.  afc_process_block's graph adds the
closed loop of Sec. 5 (push into the canceller's ring, prediction, the
canceller's tail); it is checked the same way, and like for like against the
oracle.
"""

import os
import time

import numpy as np
import pytest

from gpu_helpers import RoomPlant, check_replay, snr_db
from oracle import upols
from paper_2509_04390_gb300 import build, signals
from paper_2509_04390_gb300 import upols as U

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def engine_lib():
    if not os.path.exists(build.lib_path()):
        build.build()
    U.load()


def blocks_of(x, B):
    return [np.ascontiguousarray(x[:, b * B : (b + 1) * B]) for b in range(x.shape[1] // B)]


def run_blocks(w, mode, precision="fp32", tiling=None, pause_s=0.0):
    with U.Engine(w.fs, w.block, w.n_in, w.n_out, w.taps, precision, tiling) as e:
        e.set_host_graph(mode)
        e.set_filters(w.h)
        ys = []
        for xb in blocks_of(w.x, w.block):
            ys.append(e.process(xb))
            if pause_s:
                time.sleep(pause_s)
        U.conv_synchronize(e.h)
        return np.concatenate(ys, axis=1), e.host_graph()


@pytest.mark.parametrize("precision", ["fp32", "fp16", "bf16"])
def test_graph_equals_stream_path_bitwise(precision):
    # K = 9 partitions, 40 blocks: the ring wraps four times
    w = signals.random_case(31, 3, 5, 9 * 64 - 7, 64, 40, decay_s=0.05)
    y_g, (m_g, nb_g) = run_blocks(w, "always", precision)
    y_s, (m_s, nb_s) = run_blocks(w, "off", precision)
    assert (m_g, nb_g) == (2, 40)
    assert (m_s, nb_s) == (0, 0)
    np.testing.assert_array_equal(y_g, y_s)


def test_auto_mode_takes_the_graph_when_the_tail_is_done():
    # one call every 2 ms (real-time use): the previous tail has always finished
    w = signals.random_case(36, 2, 3, 6 * 64 + 1, 64, 20, decay_s=0.05)
    y_a, (m_a, nb_a) = run_blocks(w, "auto", pause_s=0.002)
    y_s, _ = run_blocks(w, "off")
    assert (m_a, nb_a) == (1, 20)
    np.testing.assert_array_equal(y_a, y_s)
    # back to back, whichever form each call takes, the bits are the same
    y_b, _ = run_blocks(w, "auto")
    np.testing.assert_array_equal(y_b, y_s)


def test_host_graph_mode_is_checked():
    with U.Engine(48000, 64, 1, 1, 64) as e:
        with pytest.raises(U.ConvError):
            U.conv_set_host_graph(e.h, 3)
        assert e.host_graph() == (1, 0)


def test_graph_matches_oracle_fp32():
    w = signals.random_case(32, 2, 4, 12 * 128 + 5, 128, 30, decay_s=0.1)
    y, (_, nb) = run_blocks(w, "always")
    assert nb == 30
    ref = upols(w.h.astype(np.float64), w.x.astype(np.float64), w.block)
    assert snr_db(y, ref) >= 120.0


@pytest.mark.parametrize("taps", [1, 50, 64])
def test_graph_single_partition_has_no_tail(taps):
    # K = 1: the graph holds only the pack and the output
    w = signals.random_case(33, 2, 3, taps, 64, 12)
    y_g, (_, nb) = run_blocks(w, "always")
    y_s, _ = run_blocks(w, "off")
    assert nb == 12
    np.testing.assert_array_equal(y_g, y_s)
    ref = upols(w.h.astype(np.float64), w.x.astype(np.float64), w.block)
    assert snr_db(y_g, ref) >= 120.0


@pytest.mark.parametrize("tiling", [dict(kernel="direct1"), dict(kernel="direct2"), dict(kernel="tma", warps=16)])
def test_graph_with_other_mac_kernels(tiling):
    w = signals.random_case(34, 2, 6, 10 * 128 - 3, 128, 24, decay_s=0.1)
    y_g, (_, nb) = run_blocks(w, "always", tiling=tiling)
    y_s, _ = run_blocks(w, "off", tiling=tiling)
    assert nb == 24
    np.testing.assert_array_equal(y_g, y_s)
    ref = upols(w.h.astype(np.float64), w.x.astype(np.float64), w.block)
    assert snr_db(y_g, ref) >= 120.0


def mixed_calls(w, mode, torch):
    """A block chain that moves between the graph and every stream entry
    point: host calls, caller-stream calls, a multi-block call, kernel timing,
    a new L2 budget, a replanned MAC (the graph is rebuilt) and a reset."""
    B, nb = w.block, w.x.shape[1] // w.block
    xb = blocks_of(w.x, B)
    d_x = torch.from_numpy(np.stack(xb)).cuda()
    d_y = torch.zeros((nb, w.n_out, B), dtype=torch.float32, device="cuda")
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()
    ys = [None] * nb
    with U.Engine(w.fs, B, w.n_in, w.n_out, w.taps) as e:
        e.set_host_graph(mode)
        e.set_filters(w.h)
        b = 0

        def host(n):
            nonlocal b
            for _ in range(n):
                ys[b] = e.process(xb[b])
                b += 1

        def dev(n):
            nonlocal b
            for _ in range(n):
                U.conv_process_block_async(e.h, d_x[b], d_y[b], stream)
                b += 1
            stream.synchronize()
            U.conv_join_async(e.h, stream)
            stream.synchronize()
            for i in range(b - n, b):
                ys[i] = d_y[i].cpu().numpy()

        host(6)
        dev(4)
        host(5)
        out = np.empty((w.n_out, 5 * B), dtype=np.float32)
        U.conv_process_blocks(e.h, np.ascontiguousarray(w.x[:, b * B : (b + 5) * B]), out, e.shape)
        for i in range(5):
            ys[b + i] = out[:, i * B : (i + 1) * B]
        b += 5
        host(3)
        U.conv_profile_enable(e.h, 1)
        host(3)
        U.conv_profile_enable(e.h, 0)
        host(3)
        U.conv_set_l2_keep(e.h, 0)
        host(4)
        assert b == 33
        # the canceller's paths replan the synthesis MAC beside it (the graph
        # is rebuilt) and restart the stream
        rng = np.random.default_rng(7)
        e.set_paths((0.01 * rng.standard_normal((w.n_in, w.n_out, 100))).astype(np.float32))
        host(3)
        e.reset()
        host(nb - b)
        U.conv_synchronize(e.h)
        used = e.host_graph()[1]
    return np.concatenate(ys, axis=1), used


def test_graph_transitions_keep_the_block_chain():
    torch = pytest.importorskip("torch")
    w = signals.random_case(35, 2, 4, 7 * 64 + 9, 64, 48, decay_s=0.05)
    y_g, used_g = mixed_calls(w, "always", torch)
    y_s, used_s = mixed_calls(w, "off", torch)
    assert used_s == 0 and used_g > 20
    np.testing.assert_array_equal(y_g, y_s)
    # the chain up to the reset is one continuous convolution
    n0 = 33
    ref = upols(w.h.astype(np.float64), w.x[:, : n0 * w.block].astype(np.float64), w.block)
    assert snr_db(y_g[:, : n0 * w.block], ref) >= 120.0


# ------------------------------------------------ the closed loop (Sec. 5)


def closed_loop(mode, h, f_true, f_hat, s, B, precision="fp32", switch=None):
    """The engine's static canceller in a simulated room, with the host-call
    graph mode `mode`; switch = {block: mode} changes it on the way.  Returns
    the loudspeaker and error signals, the microphone blocks and the number of
    blocks that went through a graph."""
    L, P, n_h = h.shape
    room = RoomPlant(f_true, B)
    nb = s.shape[1] // B
    out = np.zeros((L, nb * B), np.float32)
    err = np.zeros((P, nb * B), np.float32)
    mic = np.zeros((P, nb * B), np.float32)
    fb = np.zeros((P, B))
    with U.Engine(48000, B, P, L, n_h, precision) as e:
        e.set_host_graph(mode)
        e.set_filters(h)
        e.set_paths(f_hat)
        U.afc_set_guard(e.h, 1e3)  # computed from the error block the call returns; never trips here
        l_n = np.empty((L, B), np.float32)
        e_n = np.empty((P, B), np.float32)
        for b in range(nb):
            if switch and b in switch:
                e.set_host_graph(switch[b])
            m_n = (s[:, b * B : (b + 1) * B].astype(np.float64) + fb).astype(np.float32)
            e.process_afc(m_n, l_n, e_n)
            out[:, b * B : (b + 1) * B] = l_n
            err[:, b * B : (b + 1) * B] = e_n
            mic[:, b * B : (b + 1) * B] = m_n
            fb = room.step(l_n)
        U.conv_synchronize(e.h)
        used = e.host_graph()[1]
    return out, err, mic, used


def loop_case(seed, P, L, B, taps, taps_fb, n_blocks):
    rng = np.random.default_rng(seed)
    h = (rng.standard_normal((L, P, taps)) * np.exp(-np.arange(taps) / (taps / 3.5)) * 0.08).astype(np.float32)
    f = (rng.standard_normal((P, L, taps_fb)) * np.exp(-np.arange(taps_fb) / (taps_fb / 5.0)) * 0.05)
    s = (rng.standard_normal((P, n_blocks * B)) * 0.1).astype(np.float32)
    return h, f.astype(np.float32), s


@pytest.mark.parametrize("precision", ["fp32", "fp16", "bf16"])
@pytest.mark.parametrize("taps_fb", [300, 40])
def test_closed_loop_graph_equals_stream_path_bitwise(precision, taps_fb):
    # 11 synthesis partitions and 5 (or 1: no canceller tail) canceller
    # partitions over 48 blocks: both rings wrap
    h, f, s = loop_case(51, 2, 3, 64, 700, taps_fb, 48)
    fh = (0.5 * f).astype(np.float32)
    y_g, e_g, _, used_g = closed_loop("always", h, f, fh, s, 64, precision)
    y_s, e_s, _, used_s = closed_loop("off", h, f, fh, s, 64, precision)
    assert (used_g, used_s) == (48, 0)
    np.testing.assert_array_equal(y_g, y_s)
    np.testing.assert_array_equal(e_g, e_s)


def test_closed_loop_graph_against_oracle():
    # like for like: each stage of the loop fed the engine's own signals
    h, f, s = loop_case(52, 2, 3, 64, 700, 300, 60)
    fh = (0.5 * f).astype(np.float32)  # residual feedback recirculates
    y, e, mic, used = closed_loop("always", h, f, fh, s, 64)
    assert used == 60
    check_replay(h, fh, y, e, mic, 64, 120.0, "closed loop through the graph, F_hat = F/2")


def test_closed_loop_graph_transitions_keep_the_loop():
    # graph -> stream -> graph -> auto: the same bits as the stream path throughout
    h, f, s = loop_case(53, 3, 5, 64, 900, 200, 40)
    fh = (0.5 * f).astype(np.float32)
    y_m, e_m, _, used = closed_loop("always", h, f, fh, s, 64, switch={9: "off", 17: "always", 30: "auto"})
    y_s, e_s, _, _ = closed_loop("off", h, f, fh, s, 64)
    assert used >= 9 + 13
    np.testing.assert_array_equal(y_m, y_s)
    np.testing.assert_array_equal(e_m, e_s)

"""Failure paths, without a GPU fault.

* A bounded device-side wait that runs out: ``conv_inject_wait_timeout`` makes
  one CTA of the next synthesis tail MAC withhold a pipeline stage, so its
  consumers wait on a barrier that nothing completes and give up after a
  short limit.  The block that uses that tail must return CONV_E_TIMEOUT, the
  context must stay usable, and ``conv_reset`` must restart the stream so that
  it repeats a fresh engine's run bit-exactly.
* The closed-loop divergence guard (``afc_set_guard``): a simulated room whose
  feedback the canceller does not know makes the loop unstable; the call must
  return CONV_E_UNSTABLE and reset the loop state.
* The per-session counters (``conv_get_stats``).
* Kernel timing (``conv_profile_*``, with the L2 flush aid) leaves results
  unchanged.
"""

import os

import numpy as np
import pytest

from gpu_helpers import RoomPlant
from paper_2509_04390_gb300 import build, signals
from paper_2509_04390_gb300 import upols as U

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def engine_lib():
    if not os.path.exists(build.lib_path()):
        build.build()
    U.load()


def fresh_run(w, nb, precision="fp32"):
    with U.Engine(w.fs, w.block, w.n_in, w.n_out, w.taps, precision) as e:
        e.set_filters(w.h)
        return e.run(w.x[:, : nb * w.block])


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
def test_wait_timeout_is_reported_and_reset_recovers(precision):
    w = signals.random_case(3100, 3, 6, 5000, 64, 40)
    B, nb = w.block, 40
    with U.Engine(w.fs, B, w.n_in, w.n_out, w.taps, precision) as e:
        e.set_filters(w.h)
        ref = e.run(w.x[:, : nb * B])
        e.reset()
        for b in range(10):
            e.process(np.ascontiguousarray(w.x[:, b * B : (b + 1) * B]))
        U.conv_inject_wait_timeout(e.h, 2_000_000)  # 2 ms
        codes = []
        for b in range(10, 13):
            try:
                e.process(np.ascontiguousarray(w.x[:, b * B : (b + 1) * B]))
                codes.append(U.CONV_OK)
            except U.ConvError as err:
                codes.append(err.code)
        # the tail enqueued by block 10's call serves block 11: one of the
        # calls reports it, the others are clean
        assert codes.count(U.CONV_E_TIMEOUT) == 1, codes
        assert all(c in (U.CONV_OK, U.CONV_E_TIMEOUT) for c in codes)
        U.conv_synchronize(e.h)  # the record is cleared and the context works
        st = e.stats()
        assert st["device_errors"] == 1
        e.reset()
        again = e.run(w.x[:, : nb * B])
    np.testing.assert_array_equal(again, ref)


def test_wait_timeout_arguments_and_states():
    w = signals.random_case(3101, 1, 2, 40, 64, 4)  # one partition: no tail MAC
    with U.Engine(w.fs, w.block, 1, 2, w.taps) as e:
        with pytest.raises(U.ConvError) as ei:
            U.conv_inject_wait_timeout(e.h, 2_000_000)
        assert ei.value.code == U.CONV_E_STATE  # filters not set
        e.set_filters(w.h)
        with pytest.raises(U.ConvError) as ei:
            U.conv_inject_wait_timeout(e.h, 2_000_000)
        assert ei.value.code == U.CONV_E_STATE  # K = 1
    w = signals.random_case(3102, 2, 3, 2000, 64, 4)
    with U.Engine(w.fs, w.block, 2, 3, w.taps, tiling={"kernel": "direct1"}) as e:
        e.set_filters(w.h)
        with pytest.raises(U.ConvError) as ei:
            U.conv_inject_wait_timeout(e.h, 2_000_000)
        assert ei.value.code == U.CONV_E_STATE  # the direct-load MAC has no waits
    with U.Engine(w.fs, w.block, 2, 3, w.taps) as e:
        e.set_filters(w.h)
        for bad in (0, 999, 2_000_000_000):
            with pytest.raises(U.ConvError) as ei:
                U.conv_inject_wait_timeout(e.h, bad)
            assert ei.value.code == U.CONV_E_INVAL


def test_closed_loop_guard_trips_and_resets_the_loop():
    """Feedback paths at +6 dB above what the (zero) estimate cancels: the loop
    gain exceeds one and e grows until the guard trips.  After the trip the
    loop state is zero: the same engine then repeats a fresh engine's run of a
    stable (room-free) input bit-exactly."""
    rng = np.random.default_rng(71)
    P, L, B = 2, 4, 64
    h = (rng.standard_normal((L, P, 600)) * np.exp(-np.arange(600) / 150.0) * 0.5).astype(np.float32)
    f = (rng.standard_normal((P, L, 200)) * np.exp(-np.arange(200) / 40.0) * 0.5).astype(np.float32)
    zero = np.zeros_like(f)
    s = (rng.standard_normal((P, 400 * B)) * 0.1).astype(np.float32)
    guard = 10.0

    def stable_run(e, nb=30):
        out = []
        for b in range(nb):
            out.append(e.process_afc(np.ascontiguousarray(s[:, b * B : (b + 1) * B])).copy())
        return np.concatenate(out, axis=1)

    with U.Engine(48000, B, P, L, h.shape[2]) as fresh:
        fresh.set_filters(h)
        fresh.set_paths(zero)
        ref = stable_run(fresh)

    with U.Engine(48000, B, P, L, h.shape[2]) as e:
        e.set_filters(h)
        e.set_paths(zero)
        U.afc_set_guard(e.h, guard)
        room = RoomPlant(f, B)
        fb = np.zeros((P, B))
        l_n = np.empty((L, B), np.float32)
        e_n = np.empty((P, B), np.float32)
        tripped_at = None
        peak = 0.0
        for b in range(400):
            m_n = (s[:, b * B : (b + 1) * B].astype(np.float64) + fb).astype(np.float32)
            try:
                e.process_afc(m_n, l_n, e_n)
            except U.ConvError as err:
                assert err.code == U.CONV_E_UNSTABLE
                assert "guard" in str(err)
                tripped_at = b
                break
            peak = max(peak, float(np.sqrt(np.mean(e_n.astype(np.float64) ** 2))))
            fb = room.step(l_n)
        assert tripped_at is not None, f"the loop did not diverge (peak rms(e) {peak:.3g})"
        assert peak <= guard
        assert e.stats()["guard_trips"] == 1
        U.afc_set_guard(e.h, 0.0)
        got = stable_run(e)
    np.testing.assert_array_equal(got, ref)


def test_stats_count_blocks_calls_and_deadline_misses():
    w = signals.random_case(3103, 2, 3, 1500, 64, 24)
    B = w.block
    # fs = 1e9: a period of 64 ns, which every call misses
    with U.Engine(1e9, B, w.n_in, w.n_out, w.taps) as e:
        e.set_filters(w.h)
        for b in range(12):
            e.process(np.ascontiguousarray(w.x[:, b * B : (b + 1) * B]))
        U.conv_process_blocks(e.h, np.ascontiguousarray(w.x[:, 12 * B : 24 * B]),
                              np.empty((w.n_out, 12 * B), np.float32))
        st = e.stats()
        assert st["blocks"] == 24
        assert st["timed_calls"] == 12
        assert st["deadline_misses"] == 12
        assert sum(st["latency_hist"]) == 12
        assert 0.0 < st["max_latency_us"] and st["sum_latency_us"] >= st["max_latency_us"]
        e.reset()  # counters survive a stream reset
        assert e.stats()["blocks"] == 24
        U.conv_reset_stats(e.h)
        assert e.stats()["blocks"] == 0 and sum(e.stats()["latency_hist"]) == 0
    # a generous period: nothing missed
    with U.Engine(1.0, B, w.n_in, w.n_out, w.taps) as e:
        e.set_filters(w.h)
        for b in range(6):
            e.process(np.ascontiguousarray(w.x[:, b * B : (b + 1) * B]))
        assert e.stats()["deadline_misses"] == 0


def test_join_async_leaves_results_unchanged():
    """Blocks enqueued on a caller stream, each followed by conv_join_async on
    that stream (which then also waits for the background tail), give the
    host-call result exactly."""
    torch = pytest.importorskip("torch")
    w = signals.random_case(3104, 2, 5, 3000, 64, 20)
    B, nb = w.block, 20
    ref = fresh_run(w, nb)
    d_blocks = torch.from_numpy(w.x[:, : nb * B].copy()).cuda().reshape(w.n_in, nb, B).permute(1, 0, 2).contiguous()
    d_y = torch.zeros((nb, w.n_out, B), dtype=torch.float32, device="cuda")
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()
    with U.Engine(w.fs, B, w.n_in, w.n_out, w.taps) as e:
        e.set_filters(w.h)
        for b in range(nb):
            U.conv_process_block_async(e.h, d_blocks[b], d_y[b], stream)
            U.conv_join_async(e.h, stream)
        stream.synchronize()
        U.conv_synchronize(e.h)
    got = d_y.cpu().numpy().transpose(1, 0, 2).reshape(w.n_out, nb * B)
    np.testing.assert_array_equal(got, ref)


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
def test_kernel_timing_with_l2_flush_leaves_results_unchanged(precision):
    """conv_profile_enable with conv_profile_flush_l2: every block's tail MAC
    is timed (one launch per block after the first), each preceded by the
    scratch read; the outputs equal an untimed run bit for bit."""
    w = signals.random_case(3105, 2, 5, 3000, 64, 20)
    nb = 20
    ref = fresh_run(w, nb, precision)
    with U.Engine(w.fs, w.block, w.n_in, w.n_out, w.taps, precision) as e:
        e.set_filters(w.h)
        U.conv_profile_enable(e.h, nb + 4)
        U.conv_profile_flush_l2(e.h, 8 << 20)
        got = e.run(w.x[:, : nb * w.block])
        ms, n = U.conv_profile_read(e.h)
        U.conv_profile_flush_l2(e.h, 0)
        U.conv_profile_enable(e.h, 0)
        with pytest.raises(U.ConvError) as ei:
            U.conv_profile_flush_l2(e.h, -1)
        assert ei.value.code == U.CONV_E_INVAL
    np.testing.assert_array_equal(got, ref)
    assert n >= nb - 1 and ms > 0.0

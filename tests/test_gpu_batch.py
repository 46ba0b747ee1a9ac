"""Batched sessions: one launch per stage for many heterogeneous sessions.

Every session's output in the batch must be bit-identical to the same session
processed on its own (the batched kernels run the same code on the same plan,
and every reduction has a fixed order), and match the FP64 oracle.
"""

import os

import numpy as np
import pytest

from gpu_helpers import snr_db
from oracle import upols
from paper_2509_04390_gb300 import build, signals
from paper_2509_04390_gb300 import upols as U

pytestmark = pytest.mark.gpu

SHAPES = [  # n_in, n_out, taps, block
    (1, 2, 3000, 64),
    (3, 20, 9000, 128),
    (4, 16, 20000, 256),
    (2, 5, 700, 512),
    (1, 1, 1, 16),  # K = 1: no tail
    (5, 9, 40000, 1024),
]
BATCH_TILING = {"kernel": "tma", "warps": 8}
BOUND = {"fp32": 120.0, "fp16": 60.0}  # SNR against the FP64 oracle, as for single sessions


@pytest.fixture(scope="module", autouse=True)
def engine_lib():
    if not os.path.exists(build.lib_path()):
        build.build()
    U.load()


def make_sessions(precision, seed0=300):
    ws = [signals.random_case(seed0 + i, a, b, t, B, 24) for i, (a, b, t, B) in enumerate(SHAPES)]
    engs = []
    for w in ws:
        e = U.Engine(w.fs, w.block, w.n_in, w.n_out, w.taps, precision, BATCH_TILING)
        e.set_filters(w.h)
        engs.append(e)
    return ws, engs


def run_batched(torch, ws, engs, batch, blocks):
    outs = [np.zeros((w.n_out, blocks * w.block), np.float32) for w in ws]
    d_x = [torch.from_numpy(w.x).cuda() for w in ws]
    d_y = [torch.zeros((w.n_out, w.block), dtype=torch.float32, device="cuda") for w in ws]
    stream = torch.cuda.current_stream()
    for b in range(blocks):
        ins = [d_x[i][:, b * w.block : (b + 1) * w.block].contiguous() for i, w in enumerate(ws)]
        batch.process_async(ins, d_y, stream)
        torch.cuda.synchronize()
        for i, w in enumerate(ws):
            outs[i][:, b * w.block : (b + 1) * w.block] = d_y[i].cpu().numpy()
    batch.synchronize()
    return outs


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
def test_batch_equals_sessions_alone(precision):
    torch = pytest.importorskip("torch")
    ws, engs = make_sessions(precision)
    alone = [e.run(w.x) for e, w in zip(engs, ws)]
    for e in engs:
        e.reset()
    with U.Batch(precision) as batch:
        for e in engs:
            batch.add(e)
        assert U.conv_batch_size(batch.b) == len(engs)
        got = run_batched(torch, ws, engs, batch, 24)
    for i, w in enumerate(ws):
        np.testing.assert_array_equal(got[i], alone[i])
        ref = upols(w.h.astype(np.float64), w.x.astype(np.float64), w.block)
        s = snr_db(got[i], ref)
        print(f"batch {precision} session {i} {SHAPES[i]}: {s:.1f} dB against the oracle")
        assert s >= BOUND[precision]
    for e in engs:
        e.close()


def test_session_moves_into_and_out_of_a_batch():
    torch = pytest.importorskip("torch")
    ws, engs = make_sessions("fp32", seed0=500)
    ref = [e.run(w.x) for e, w in zip(engs, ws)]
    for e in engs:
        e.reset()
    e0, w0 = engs[2], ws[2]
    B = w0.block
    y = np.zeros_like(ref[2])
    # 8 blocks alone, 8 in a batch with the others, 8 alone again
    y[:, : 8 * B] = e0.run(w0.x[:, : 8 * B])
    with U.Batch("fp32") as batch:
        for e in engs:
            if e is not e0:
                batch.add(e)
        # the others start their stream in the batch now
        batch.add(e0)
        others = [i for i in range(len(engs)) if engs[i] is not e0]
        d_y = {i: torch.zeros((ws[i].n_out, ws[i].block), dtype=torch.float32, device="cuda") for i in range(len(engs))}
        order = others + [2]
        for b in range(8, 16):
            ins, outs = [], []
            for i in order:
                w = ws[i]
                blk = b if i == 2 else b - 8
                ins.append(torch.from_numpy(np.ascontiguousarray(w.x[:, blk * w.block : (blk + 1) * w.block])).cuda())
                outs.append(d_y[i])
            batch.process_async(ins, outs)
            batch.synchronize()
            y[:, b * B : (b + 1) * B] = d_y[2].cpu().numpy()
        batch.remove(e0)
    y[:, 16 * B : 24 * B] = e0.run(w0.x[:, 16 * B : 24 * B])
    np.testing.assert_array_equal(y, ref[2])
    for e in engs:
        e.close()


def test_batch_rejects_mismatched_sessions():
    w = signals.random_case(1, 1, 2, 500, 64, 4)
    with U.Batch("fp32") as batch:
        e16 = U.Engine(w.fs, 64, 1, 2, 500, "fp16", BATCH_TILING)
        e16.set_filters(w.h)
        with pytest.raises(U.ConvError):
            batch.add(e16)  # precision differs
        ed = U.Engine(w.fs, 64, 1, 2, 500, "fp32", {"kernel": "direct1"})
        ed.set_filters(w.h)
        with pytest.raises(U.ConvError):
            batch.add(ed)  # direct-load MAC
        en = U.Engine(w.fs, 64, 1, 2, 500)
        with pytest.raises(U.ConvError):
            batch.add(en)  # no filters
        for e in (e16, ed, en):
            e.close()


def test_sessions_due_on_different_ticks():
    """Continuous batching: a 64-sample tick; a session of block B is due every
    B / 64 ticks and is processed only then, alongside whatever else is due."""
    torch = pytest.importorskip("torch")
    shapes = [(2, 3, 1500, 64), (1, 4, 5000, 128), (3, 2, 9000, 256), (2, 6, 2000, 64)]
    ws = [signals.random_case(700 + i, a, b, t, B, 16) for i, (a, b, t, B) in enumerate(shapes)]
    engs = []
    for w in ws:
        e = U.Engine(w.fs, w.block, w.n_in, w.n_out, w.taps, "fp32", BATCH_TILING)
        e.set_filters(w.h)
        engs.append(e)
    alone = [e.run(w.x[:, : 4 * w.block]) for e, w in zip(engs, ws)]
    for e in engs:
        e.reset()
    got = [np.zeros_like(a) for a in alone]
    done = [0] * len(ws)
    d_y = [torch.zeros((w.n_out, w.block), dtype=torch.float32, device="cuda") for w in ws]
    with U.Batch("fp32") as batch:
        for e in engs:
            batch.add(e)
        for tick in range(16):
            due = [i for i, w in enumerate(ws) if (tick * 64) % w.block == 0 and done[i] < 4]
            if not due:
                continue
            ins = []
            for i in due:
                w, b = ws[i], done[i]
                ins.append(torch.from_numpy(np.ascontiguousarray(w.x[:, b * w.block : (b + 1) * w.block])).cuda())
            batch.process_some_async(due, ins, [d_y[i] for i in due])
            batch.synchronize()
            for i in due:
                w, b = ws[i], done[i]
                got[i][:, b * w.block : (b + 1) * w.block] = d_y[i].cpu().numpy()
                done[i] += 1
    assert done == [4] * len(ws)
    for g, a in zip(got, alone):
        np.testing.assert_array_equal(g, a)
    for e in engs:
        e.close()


def test_canceller_session_in_a_batch():
    torch = pytest.importorskip("torch")
    w = signals.random_case(900, 2, 6, 4000, 128, 12)
    rng = np.random.default_rng(901)
    f = (rng.standard_normal((2, 6, 700)) * 0.02).astype(np.float32)
    plain = signals.random_case(902, 3, 4, 2500, 256, 6)

    def make():
        e = U.Engine(w.fs, w.block, 2, 6, w.taps, "fp32", BATCH_TILING)
        e.set_filters(w.h)
        e.set_paths(f)
        p = U.Engine(plain.fs, plain.block, 3, 4, plain.taps, "fp32", BATCH_TILING)
        p.set_filters(plain.h)
        return e, p

    e, p = make()
    alone_e = np.concatenate(
        [e.process_afc(np.ascontiguousarray(w.x[:, b * 128 : (b + 1) * 128])).copy() for b in range(12)], axis=1
    )
    alone_p = p.run(plain.x)
    e.close()
    p.close()
    e, p = make()
    ye = np.zeros_like(alone_e)
    yp = np.zeros_like(alone_p)
    d_ye = torch.zeros((6, 128), dtype=torch.float32, device="cuda")
    d_yp = torch.zeros((4, 256), dtype=torch.float32, device="cuda")
    with U.Batch("fp32") as batch:
        batch.add(e)
        batch.add(p)
        for tick in range(12):  # 128-sample ticks; the 256-block session every other tick
            idx, ins, outs = [0], [torch.from_numpy(np.ascontiguousarray(w.x[:, tick * 128 : (tick + 1) * 128])).cuda()], [d_ye]
            if tick % 2 == 0:
                b = tick // 2
                idx.append(1)
                ins.append(torch.from_numpy(np.ascontiguousarray(plain.x[:, b * 256 : (b + 1) * 256])).cuda())
                outs.append(d_yp)
            batch.process_some_async(idx, ins, outs)
            batch.synchronize()
            ye[:, tick * 128 : (tick + 1) * 128] = d_ye.cpu().numpy()
            if tick % 2 == 0:
                yp[:, (tick // 2) * 256 : (tick // 2 + 1) * 256] = d_yp.cpu().numpy()
    np.testing.assert_array_equal(ye, alone_e)
    np.testing.assert_array_equal(yp, alone_p)
    e.close()
    p.close()


def afc_session(seed, P, L, taps, taps_fb, B, precision):
    rng = np.random.default_rng(seed)
    h = (rng.standard_normal((L, P, taps)) * np.exp(-np.arange(taps) / (taps / 4)) / np.sqrt(taps)).astype(np.float32)
    f = (rng.standard_normal((P, L, taps_fb)) * np.exp(-np.arange(taps_fb) / (taps_fb / 4)) * 0.02).astype(np.float32)
    x = (rng.standard_normal((P, 24 * B)) * 0.1).astype(np.float32)
    e = U.Engine(48000, B, P, L, taps, precision, BATCH_TILING)
    e.set_filters(h)
    e.set_paths(f)
    return signals.Workload(f"afc{seed}", 48000, B, h, x, f), e


def mixed_sessions(precision, seed0):
    ws, engs = make_sessions(precision, seed0)
    for k, (P, L, taps, taps_fb, B) in enumerate(((2, 5, 3000, 600, 64), (4, 16, 9000, 2000, 256))):
        w, e = afc_session(seed0 + 50 + k, P, L, taps, taps_fb, B, precision)
        ws.append(w)
        engs.append(e)
    return ws, engs


def run_steps(torch, ws, engs, persistent_at, blocks, some=None):
    """Blocks through one batch; persistent_at(b) says whether step b runs as
    one persistent launch; some(b): the session indices due at step b (all if None)."""
    outs = [np.zeros((w.n_out, blocks * w.block), np.float32) for w in ws]
    d_x = [torch.from_numpy(w.x).cuda() for w in ws]
    d_y = [torch.zeros((w.n_out, w.block), dtype=torch.float32, device="cuda") for w in ws]
    done = [0] * len(ws)
    with U.Batch(U.conv_get_info(engs[0].h)["precision"]) as batch:
        for e in engs:
            batch.add(e)
        for b in range(blocks):
            batch.set_persistent(persistent_at(b))
            idx = list(range(len(ws))) if some is None else some(b)
            ins = [d_x[i][:, done[i] * ws[i].block : (done[i] + 1) * ws[i].block].contiguous() for i in idx]
            batch.process_some_async(idx, ins, [d_y[i] for i in idx], torch.cuda.current_stream())
            batch.synchronize()
            torch.cuda.synchronize()
            for i in idx:
                outs[i][:, done[i] * ws[i].block : (done[i] + 1) * ws[i].block] = d_y[i].cpu().numpy()
                done[i] += 1
        for e in engs:
            batch.remove(e)
    return outs, done


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
def test_persistent_step_is_bit_exact(precision):
    """One persistent launch per step (work items claimed in dependency order)
    gives the separate launches' outputs bit for bit: plain and canceller
    sessions, all sessions every step or a changing subset, and switching the
    mode between steps."""
    torch = pytest.importorskip("torch")
    nb = 16
    ws, engs = mixed_sessions(precision, 700)
    ref, _ = run_steps(torch, ws, engs, lambda b: False, nb)
    for e in engs:
        e.reset()
    got, _ = run_steps(torch, ws, engs, lambda b: True, nb)
    for i in range(len(ws)):
        np.testing.assert_array_equal(got[i], ref[i])
    for e in engs:
        e.reset()
    mixed, _ = run_steps(torch, ws, engs, lambda b: (b % 3 != 1) * (1 + (b % 2)), nb)
    for i in range(len(ws)):
        np.testing.assert_array_equal(mixed[i], ref[i])
    # replayed from CUDA graphs (captured once per table parity, then replayed)
    for e in engs:
        e.reset()
    graphed, _ = run_steps(torch, ws, engs, lambda b: 2, nb)
    for i in range(len(ws)):
        np.testing.assert_array_equal(graphed[i], ref[i])
    # a changing subset of due sessions: each session's stream stays the same
    some = lambda b: [i for i in range(len(ws)) if (b + i) % 3 != 0]  # noqa: E731
    for e in engs:
        e.reset()
    sub_ref, done = run_steps(torch, ws, engs, lambda b: False, nb, some)
    for e in engs:
        e.reset()
    sub_got, _ = run_steps(torch, ws, engs, lambda b: True, nb, some)
    for e in engs:
        e.reset()
    sub_graph, _ = run_steps(torch, ws, engs, lambda b: 2, nb, some)  # due set changes: graphs re-captured
    for i in range(len(ws)):
        n = done[i] * ws[i].block
        np.testing.assert_array_equal(sub_got[i][:, :n], sub_ref[i][:, :n])
        np.testing.assert_array_equal(sub_graph[i][:, :n], sub_ref[i][:, :n])
    # and the plain sessions against the FP64 oracle
    for i, w in enumerate(ws):
        if w.f is None:
            s = snr_db(got[i], upols(w.h.astype(np.float64), w.x[:, : nb * w.block].astype(np.float64), w.block))
            assert s >= BOUND[precision], (i, s)
    for e in engs:
        e.close()

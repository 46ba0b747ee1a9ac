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
        if precision == "fp32":
            ref = upols(w.h.astype(np.float64), w.x.astype(np.float64), w.block)
            assert snr_db(got[i], ref) >= 120.0
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

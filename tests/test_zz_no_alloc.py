"""The allocation-free FDL MAC entry point (``conv_fdl_mac_noalloc``).

The entry point is for callers that cannot allocate device memory: a real-time
audio callback, where an allocation can block past the block deadline, or a
plugin whose host owns every device buffer.  It takes the filter spectra and
the delay-line ring from the caller and keeps its split partials in a fixed
file-scope device array.

Here the caller's spectra are built on the host (numpy FP64 FFTs, rounded to
float32 once), in the layout the entry point documents, and two consecutive
blocks are computed with it.  Each is compared with the FP64 oracle's UPOLS of
the same input and with the same block from the regular engine
(``conv_process_block``), at the FP32 parity bound, 120 dB SNR.  The calls
after the first must leave the device's free memory unchanged, and the error
report must be clean.  This file is collected last, and passes alone in a
fresh process as well as after the other tests.
"""

import os

import numpy as np
import pytest

from gpu_helpers import snr_db
from oracle import upols
from paper_2509_04390_gb300 import build, signals
from paper_2509_04390_gb300 import upols as U

pytestmark = pytest.mark.gpu

FP32_DB = 120.0


def packed_rfft(w, B):
    """2B-point R2C of the last axis, packed: bin 0 = (DC, Nyquist), bins 1..B-1."""
    X = np.fft.rfft(np.asarray(w, dtype=np.float64), n=2 * B, axis=-1)
    out = np.empty(X.shape[:-1] + (B, 2), dtype=np.float32)
    out[..., 0, 0] = X[..., 0].real
    out[..., 0, 1] = X[..., B].real
    out[..., 1:, 0] = X[..., 1:B].real
    out[..., 1:, 1] = X[..., 1:B].imag
    return out


@pytest.mark.parametrize("n_in,n_out,taps,B,nb", [(2, 5, 3000, 128, 30), (4, 16, 2100, 256, 12), (1, 3, 200, 16, 20)])
def test_noalloc_matches_oracle_and_engine_on_two_calls(n_in, n_out, taps, B, nb):
    torch = pytest.importorskip("torch")
    if not os.path.exists(build.lib_path()):
        build.build()
    w = signals.random_case(900 + taps, n_in, n_out, taps, B, nb)
    K = -(-taps // B)

    # the FP64 oracle and the regular engine, block by block
    y_oracle = upols(w.h.astype(np.float64), w.x.astype(np.float64), B)
    with U.Engine(w.fs, B, n_in, n_out, taps) as e:
        e.set_filters(w.h)
        y_ref = e.run(w.x)

    # caller-owned spectra in the documented layout: H[p][q][l][k], ring X[slot][q][k]
    hp = np.zeros((n_out, n_in, K * B))
    hp[:, :, :taps] = w.h
    sub = hp.reshape(n_out, n_in, K, B)  # [l][q][p][:]
    H = packed_rfft(sub, B).transpose(2, 1, 0, 3, 4).copy()  # [p][q][l][k][2]
    ring = np.zeros((K, n_in, B, 2), np.float32)
    x = w.x.astype(np.float64)

    d_H = torch.from_numpy(H).cuda()
    d_y = torch.empty((n_out, B), dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    last_two = (nb - 2, nb - 1)
    rings = {}
    for b in range(nb):
        prev = x[:, (b - 1) * B : b * B] if b > 0 else np.zeros((n_in, B))
        win = np.concatenate([prev, x[:, b * B : (b + 1) * B]], axis=1)
        slot0 = (-b) % K
        ring[slot0] = packed_rfft(win, B)
        if b in last_two:
            rings[b] = (torch.from_numpy(ring.copy()).cuda(), slot0)
    torch.cuda.synchronize()
    # every buffer exists before the calls: the first call sets the device up,
    # the calls after it must not change the device's free memory
    outs = {}
    free_before = None
    for b in last_two:
        d_X, slot0 = rings[b]
        U.conv_fdl_mac_noalloc(d_H, d_X, B, n_in, n_out, K, slot0, d_y, stream)
        U.conv_fdl_mac_noalloc_status(stream)  # waits for the call; raises on a device-side timeout
        outs[b] = d_y.cpu().numpy().copy()
        torch.cuda.synchronize()
        if free_before is None:
            free_before = torch.cuda.mem_get_info()[0]
    # the same two calls again: the array keeps the last call's contents, and
    # every call writes the partials it reads, so the results repeat exactly
    for b in last_two:
        d_X, slot0 = rings[b]
        U.conv_fdl_mac_noalloc(d_H, d_X, B, n_in, n_out, K, slot0, d_y, stream)
        U.conv_fdl_mac_noalloc_status(stream)
        np.testing.assert_array_equal(d_y.cpu().numpy(), outs[b])
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free_before
    for b in last_two:
        s_or = snr_db(outs[b], y_oracle[:, b * B : (b + 1) * B])
        s_en = snr_db(outs[b], y_ref[:, b * B : (b + 1) * B])
        print(f"noalloc {n_in}x{n_out} B={B} block {b}: {s_or:.1f} dB against the oracle, {s_en:.1f} dB against "
              f"the engine")
        assert s_or >= FP32_DB, f"block {b}: {s_or:.1f} dB against the oracle"
        assert s_en >= FP32_DB, f"block {b}: {s_en:.1f} dB against the engine"


def test_noalloc_rejects_sizes_and_pointers_beyond_its_limits():
    torch = pytest.importorskip("torch")
    if not os.path.exists(build.lib_path()):
        build.build()
    t = torch.zeros(64, dtype=torch.float32, device="cuda")
    for block, n_out in ((512, 2), (256, 17), (100, 2)):
        with pytest.raises(U.ConvError) as ei:
            U.conv_fdl_mac_noalloc(t, t, block, 1, n_out, 4, 0, t)
        assert ei.value.code == U.CONV_E_INVAL
        assert "conv_fdl_mac_noalloc" in str(ei.value)
    # spectra that do not start on a 16-byte boundary are refused before any launch
    off = t[1:]
    for d_H, d_X in ((off, t), (t, off)):
        with pytest.raises(U.ConvError) as ei:
            U.conv_fdl_mac_noalloc(d_H, d_X, 16, 1, 1, 1, 0, t)
        assert ei.value.code == U.CONV_E_INVAL
        assert "aligned" in str(ei.value)
    U.conv_fdl_mac_noalloc_status(None)  # nothing ran: a clean report

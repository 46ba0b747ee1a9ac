"""The allocation-free FDL MAC entry point agrees with the engine.

``conv_fdl_mac_noalloc`` is for callers that cannot allocate device memory,
e.g. a real-time audio callback, where an allocation can block past the block
deadline, or a plugin whose host owns every device buffer.  It takes the
filter spectra and the delay-line ring from the caller and keeps its split
partials in a fixed file-scope device array.

Here the caller's spectra are built on the host (numpy FP64 FFTs, rounded to
float32 once), in the layout the entry point documents, and two consecutive
blocks are computed with it.  Each is compared with the same block from the
regular engine (``conv_process_block``) at the FP32 parity bound, 120 dB SNR.
"""

import os

import numpy as np
import pytest

from gpu_helpers import snr_db
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
def test_noalloc_matches_engine_on_two_calls(n_in, n_out, taps, B, nb):
    torch = pytest.importorskip("torch")
    if not os.path.exists(build.lib_path()):
        build.build()
    w = signals.random_case(900 + taps, n_in, n_out, taps, B, nb)
    K = -(-taps // B)

    # the regular engine, block by block
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
    outs = {}
    last_two = (nb - 2, nb - 1)
    for b in range(nb):
        prev = x[:, (b - 1) * B : b * B] if b > 0 else np.zeros((n_in, B))
        win = np.concatenate([prev, x[:, b * B : (b + 1) * B]], axis=1)
        slot0 = (-b) % K
        ring[slot0] = packed_rfft(win, B)
        if b in last_two:
            d_X = torch.from_numpy(ring).cuda()
            torch.cuda.synchronize()
            U.conv_fdl_mac_noalloc(d_H, d_X, B, n_in, n_out, K, slot0, d_y, stream)
            torch.cuda.synchronize()
            outs[b] = d_y.cpu().numpy().copy()
    for b in last_two:
        ref = y_ref[:, b * B : (b + 1) * B]
        s = snr_db(outs[b], ref)
        assert s >= FP32_DB, f"block {b}: {s:.1f} dB"


def test_noalloc_rejects_sizes_beyond_its_limits():
    torch = pytest.importorskip("torch")
    if not os.path.exists(build.lib_path()):
        build.build()
    t = torch.zeros(16, dtype=torch.float32, device="cuda")
    for block, n_out in ((512, 2), (256, 17), (100, 2)):
        with pytest.raises(U.ConvError) as ei:
            U.conv_fdl_mac_noalloc(t, t, block, 1, n_out, 4, 0, t)
        assert ei.value.code == U.CONV_E_INVAL
        assert "conv_fdl_mac_noalloc" in str(ei.value)

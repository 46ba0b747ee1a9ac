"""Host logic of the serving loop: the HBM load a session adds per tick."""

from paper_2509_04390_gb300 import serve, signals


def test_tick_bytes_counts_every_spectrum_once_per_block():
    spec = signals.SessionSpec(n_in=4, n_out=16, taps=48000, block=256, seed=1, rt60=1.0)
    K = -(-48000 // 256)  # 188 partitions
    per_block_fp32 = (16 + 1) * 4 * K * 256 * 8  # filters + delay-line rows of one output tile
    assert serve.tick_bytes(spec, "fp32", tick=128) == per_block_fp32 * 128 / 256
    assert serve.tick_bytes(spec, "fp16", tick=128) == per_block_fp32 / 2 * 128 / 256
    assert serve.tick_bytes(spec, "fp32", tick=256) == per_block_fp32


def test_tick_bytes_adds_the_canceller():
    plain = signals.SessionSpec(n_in=2, n_out=8, taps=1000, block=128, seed=1, rt60=1.0)
    afc = signals.SessionSpec(n_in=2, n_out=8, taps=1000, block=128, seed=1, rt60=1.0, taps_fb=500)
    K_fb = -(-500 // 128)
    extra = (2 + 1) * 8 * K_fb * 128 * 4  # the canceller streams F_hat [mic][speaker] and its delay line
    assert serve.tick_bytes(afc, "fp16") - serve.tick_bytes(plain, "fp16") == extra

"""The device side of the counter-based input generator equals the host side
bit for bit (GB300 only): float32 and 8-bit, pulses, row offsets, odd channel
counts and counters beyond 2^32."""
import numpy as np
import pytest

import synth
import synth.gpu
from synth import philox

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    synth.gpu.build()


@pytest.mark.parametrize("u8", [False, True])
@pytest.mark.parametrize("n_chan,n_rows,t0", [(64, 4096, 0), (37, 3001, 12345),
                                              (1536, 700, (1 << 32) // 1536 - 300)])
def test_device_equals_host(n_chan, n_rows, t0, u8):
    w = synth.WORKLOADS["fdd_64ch_4096t_128dm"].scaled(
        n_chan=n_chan, n_t=t0 + n_rows, pulses_per_beam=3, fixed_pulse=None,
        noise_mean=128.0 if u8 else 0.0, noise_sigma=16.0 if u8 else 1.0,
        dtype="u8" if u8 else "f32")
    kw, _ = synth.philox_beam_args(w, 99, 5)
    host = philox.filterbank(n_rows=n_rows, t0=t0, **kw)
    dev = torch.empty(n_rows * n_chan, dtype=torch.uint8 if u8 else torch.float32, device="cuda")
    synth.gpu.filterbank(dev, n_rows=n_rows, t0=t0, **kw)
    torch.cuda.synchronize()
    got = dev.cpu().numpy().reshape(n_rows, n_chan)
    assert got.tobytes() == host.tobytes()

"""The counter-based input generator (synth.philox, host side): the
published Philox4x32-10 known-answer vectors, the deviate's moments, slice
consistency, 8-bit rounding and pulse placement.  The device side is checked
bit for bit against this one in test_gpu_synth.py."""
import os

import numpy as np

import synth
from synth import philox

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat():
    for line in open(GOLDEN):
        if line.strip() and not line.startswith("#"):
            v = [int(t, 16) for t in line.split()]
            yield v[:4], v[4:6], v[6:]


def test_known_answer_vectors():
    n = 0
    for ctr, key, want in _kat():
        got = philox.philox4x32_10(*[np.array([c], np.uint64) for c in ctr], *key)
        assert [int(g[0]) for g in got] == want
        n += 1
    assert n == 3


def test_vectorised_equals_elementwise():
    rng = np.random.default_rng(0)
    ctr = rng.integers(0, 2 ** 32, size=(4, 64), dtype=np.uint64)
    k0, k1 = 0x12345678, 0x9ABCDEF0
    whole = philox.philox4x32_10(*ctr, k0, k1)
    for i in range(0, 64, 9):
        one = philox.philox4x32_10(*[c[i:i + 1] for c in ctr], k0, k1)
        assert [int(o[0]) for o in one] == [int(w[i]) for w in whole]


def test_deviate_moments_and_range():
    z = philox.standard_normal(2021, 3, np.arange(1 << 21, dtype=np.uint64)).astype(np.float64)
    assert abs(z.mean()) < 3e-3 and abs(z.var() - 1.0) < 4e-3
    # Irwin-Hall(8): bounded at +-(262140 / sigma) = +-4.899; kurtosis 3 - 1.2/8
    assert np.abs(z).max() < 4.9
    kurt = np.mean(z ** 4) / np.mean(z ** 2) ** 2
    assert abs(kurt - (3.0 - 1.2 / 8)) < 0.02
    # distinct beams and seeds give uncorrelated streams
    z2 = philox.standard_normal(2021, 4, np.arange(1 << 21, dtype=np.uint64))
    z3 = philox.standard_normal(2022, 3, np.arange(1 << 21, dtype=np.uint64))
    assert abs(np.corrcoef(z, z2)[0, 1]) < 3e-3 and abs(np.corrcoef(z, z3)[0, 1]) < 3e-3


def test_slices_regenerate_exactly():
    w = synth.WORKLOADS["fdd_64ch_4096t_128dm"].scaled(pulses_per_beam=3, fixed_pulse=None)
    full, _ = synth.philox_filterbank(w, 11, beam=2)
    part, _ = synth.philox_filterbank(w, 11, beam=2, t0=1234, rows=777)
    assert np.array_equal(part, full[1234:2011])
    small = philox.filterbank(n_chan=w.n_chan, n_rows=4096, t0=0, seed=11, beam=2,
                              pulses=synth.philox_beam_args(w, 11, 2)[0]["pulses"],
                              block_rows=100, threads=3)
    assert np.array_equal(small, full)


def test_u8_rounding_and_clipping():
    x = philox.filterbank(n_chan=16, n_rows=20000, t0=0, seed=1, beam=0, mean=128.0,
                          sigma=40.0, u8=True)
    f = philox.filterbank(n_chan=16, n_rows=20000, t0=0, seed=1, beam=0, mean=128.0,
                          sigma=40.0)
    assert x.dtype == np.uint8
    assert np.array_equal(x, np.clip(np.rint(f), 0, 255).astype(np.uint8))
    assert x.min() == 0 and x.max() == 255  # 3.2 sigma reaches both ends


def test_pulses_follow_the_sweep():
    w = synth.WORKLOADS["fdd_1024ch_2p20t_2048dm"].scaled(n_t=1 << 15, pulses_per_beam=2)
    kw, pulses = synth.philox_beam_args(w, 5, 0)
    noise = philox.filterbank(n_rows=w.n_t, t0=0, **dict(kw, pulses=(), u8=False, mean=0.0,
                                                         sigma=1.0))
    sig = philox.filterbank(n_rows=w.n_t, t0=0, **dict(kw, u8=False, mean=0.0, sigma=1.0))
    diff = sig - noise
    nu = w.channel_centres()
    expect = np.zeros_like(diff)
    for p in pulses:
        st = synth.sweep_starts(nu, w.t_samp_s, p.t0, p.dm)
        assert st.max() + p.width <= w.n_t and st.min() == p.t0  # top channel: no delay
        for c in range(w.n_chan):
            expect[st[c]: st[c] + p.width, c] += p.amp
    assert np.allclose(diff, expect, atol=1e-5)

"""Counter-based Gaussian filterbanks: Philox4x32-10 (Salmon, Moraes, Dror and
Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC 2011), host side.

Every sample is a pure function of (seed, beam, time, channel), so any slice
of an input too large to hold (hundreds of GB) can be regenerated on its own,
on the host (this module, numpy) or on the device (``synth.gpu``), with
bit-identical results.  That is what lets a check on a few bins or trials of a
huge workload rebuild exactly the input the GPU saw.

Sample (t, c) of beam b: the Philox4x32-10 block of counter
(i mod 2^32, i div 2^32, b, 0) with i = t * n_chan + c, under the key
(seed mod 2^32, seed div 2^32 mod 2^32).  Its four 32-bit words are split into
eight 16-bit integers whose sum s (0 .. 524280) gives an Irwin-Hall(8)
deviate z = (s - 262140) * IH8_INV_SIGMA, of mean 0 and variance 1 (range
+-4.9 sigma; close to Gaussian in the body, which is all the noise model
needs).  Then x = z * sigma + mean, pulses added in list order, and 8-bit
data rounded half-to-even and clipped to 0..255.  Each of these is one
correctly rounded float32 operation, so host and device agree bit for bit.

Like the rest of ``synth`` this makes inputs only: no dedispersion arithmetic.
"""
from __future__ import annotations

import concurrent.futures as cf
import os

import numpy as np

PHILOX_M0 = 0xD2511F53
PHILOX_M1 = 0xCD9E8D57
PHILOX_W0 = 0x9E3779B9   # key schedule (Weyl sequence) increments
PHILOX_W1 = 0xBB67AE85
ROUNDS = 10

# 1 / standard deviation of the sum of eight independent uniform integers on
# 0..65535 (each of variance (65536^2 - 1) / 12), as float32.
IH8_MEAN = 8 * 65535 // 2          # 262140
IH8_INV_SIGMA = np.float32(1.0 / np.sqrt(8.0 * (65536.0 ** 2 - 1.0) / 12.0))

_MASK = np.uint64(0xFFFFFFFF)


def philox4x32_10(c0, c1, c2, c3, k0: int, k1: int):
    """The Philox4x32 bijection with 10 rounds, elementwise over counter arrays.

    One round maps (x0, x1, x2, x3) under the round key (k0, k1) to
    (hi(M1 x2) ^ x1 ^ k0, lo(M1 x2), hi(M0 x0) ^ x3 ^ k1, lo(M0 x0)); the key
    advances by (W0, W1) between rounds.  Returns four uint32 arrays.
    """
    x = [np.asarray(v).astype(np.uint64) for v in (c0, c1, c2, c3)]
    ka = np.uint64(k0 & 0xFFFFFFFF)
    kb = np.uint64(k1 & 0xFFFFFFFF)
    m0, m1, s32 = np.uint64(PHILOX_M0), np.uint64(PHILOX_M1), np.uint64(32)
    for r in range(ROUNDS):
        if r:
            ka = (ka + np.uint64(PHILOX_W0)) & _MASK
            kb = (kb + np.uint64(PHILOX_W1)) & _MASK
        p0 = m0 * x[0]  # < 2^64: exact
        p1 = m1 * x[2]
        x = [((p1 >> s32) ^ x[1] ^ ka) & _MASK, p1 & _MASK,
             ((p0 >> s32) ^ x[3] ^ kb) & _MASK, p0 & _MASK]
    return [v.astype(np.uint32) for v in x]


def irwin_hall8(words) -> np.ndarray:
    """Four uint32 words -> float32 deviate of mean 0, variance 1."""
    s = np.zeros(np.shape(words[0]), dtype=np.int64)
    for w in words:
        w = w.astype(np.int64)
        s += (w & 0xFFFF) + (w >> 16)
    return (s - IH8_MEAN).astype(np.float32) * IH8_INV_SIGMA


def standard_normal(seed: int, beam: int, index) -> np.ndarray:
    """Deviates for flat sample indices ``index`` (uint64 array) of one beam."""
    i = np.asarray(index, dtype=np.uint64)
    words = philox4x32_10(i & _MASK, i >> np.uint64(32), np.full(i.shape, beam, np.uint64),
                          np.zeros(i.shape, np.uint64), seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    return irwin_hall8(words)


def pulse_windows(starts: np.ndarray, width: int, t0: int, t1: int):
    """(channel, row range) pairs where a pulse with per-channel start samples
    ``starts`` and ``width`` overlaps rows [t0, t1)."""
    for c in np.nonzero((starts < t1) & (starts + width > t0))[0]:
        yield int(c), max(int(starts[c]), t0), min(int(starts[c]) + width, t1)


def filterbank(n_chan: int, n_rows: int, t0: int, seed: int, beam: int, *, mean: float = 0.0,
               sigma: float = 1.0, u8: bool = False, pulses=(), block_rows: int = 1 << 14,
               threads: int | None = None):
    """Rows [t0, t0 + n_rows) of one beam's [n_t, n_chan] time-major filterbank.

    ``pulses`` is a sequence of (starts, width, amp): starts[c] is the first
    sample of the pulse in channel c (int64 array of n_chan).  The same call on
    the device (``synth.gpu.filterbank``) returns the same bytes.
    """
    out = np.empty((n_rows, n_chan), dtype=np.uint8 if u8 else np.float32)
    cols = np.arange(n_chan, dtype=np.uint64)
    block_rows = max(1, min(block_rows, (1 << 21) // n_chan))

    def fill(r0: int) -> None:
        r1 = min(n_rows, r0 + block_rows)
        rows = np.arange(t0 + r0, t0 + r1, dtype=np.uint64)
        idx = rows[:, None] * np.uint64(n_chan) + cols[None, :]
        x = standard_normal(seed, beam, idx)
        if sigma != 1.0:
            x *= np.float32(sigma)
        if mean != 0.0:
            x += np.float32(mean)
        for starts, width, amp in pulses:
            for c, a, e in pulse_windows(np.asarray(starts), int(width), t0 + r0, t0 + r1):
                x[a - t0 - r0: e - t0 - r0, c] += np.float32(amp)
        if u8:
            np.rint(x, out=x)
            np.clip(x, 0, 255, out=x)
            out[r0:r1] = x.astype(np.uint8)
        else:
            out[r0:r1] = x

    starts = range(0, n_rows, block_rows)
    workers = threads or min(16, os.cpu_count() or 1)
    if workers > 1 and len(starts) > 1:
        with cf.ThreadPoolExecutor(max_workers=workers) as ex:
            list(ex.map(fill, starts))
    else:
        for r0 in starts:
            fill(r0)
    return out

"""Seeded synthetic filterbank inputs for the dedispersion tests and benchmark.

This module only *makes inputs*.  It holds none of the dedispersion
arithmetic (no phasors, no transforms, no shift-and-sum) and imports neither
the oracle nor the CUDA package, so both can be fed from it.

A filterbank is a [n_t, n_chan] time-major array (the 8-bit or float32
dynamic spectrum of Sect. 3 of the paper) of Gaussian noise, with boxcar
pulses injected along a dispersion sweep.  The sweep uses this module's own
sky model: a pulse emitted at sample t0 arrives in channel c at
    t0 + round(DM * K_DM_SKY * (nu_c^-2 - nu_top^-2) / t_samp),
with nu_c the channel centre and nu_top the highest channel centre, and
K_DM_SKY = 4.148808e3 MHz^2 pc^-1 cm^3 s (the value the 64-channel workload
states; the dedisperser's own constant is a plan parameter).

The workloads stand in for the simulated SUPERB-like survey data of the paper
(Sect. 4: 1024 channels, 64 us sampling), which is not available; their
shapes follow the paper's parameter space.
"""
from __future__ import annotations

import concurrent.futures as cf
import math
import os
from dataclasses import dataclass, field

import numpy as np

K_DM_SKY = 4.148808e3


@dataclass
class Pulse:
    t0: int          # emission sample at the top channel
    dm: float
    amp: float
    width: int


@dataclass
class Workload:
    name: str
    n_chan: int
    band_lo_mhz: float   # lower band edge
    band_hi_mhz: float   # upper band edge
    t_samp_s: float
    n_t: int
    dtype: str           # "u8" or "f32"
    dm0: float
    ddm: float
    n_dm: int
    chunk_len: int       # 0 = whole series zero padded to a power of two
    n_beams: int = 1
    output: str = "time"  # "time" | "spectra" | "power"
    pulses_per_beam: int = 1
    fixed_pulse: Pulse | None = None
    noise_mean: float = 0.0
    noise_sigma: float = 1.0
    extra: dict = field(default_factory=dict)

    @property
    def dnu_mhz(self) -> float:
        return (self.band_hi_mhz - self.band_lo_mhz) / self.n_chan

    @property
    def nu_lo_mhz(self) -> float:
        """Centre of channel 0."""
        return self.band_lo_mhz + 0.5 * self.dnu_mhz

    def channel_centres(self) -> np.ndarray:
        return self.nu_lo_mhz + self.dnu_mhz * np.arange(self.n_chan, dtype=np.float64)

    def dms(self) -> np.ndarray:
        return self.dm0 + self.ddm * np.arange(self.n_dm, dtype=np.float64)

    def scaled(self, **kw) -> "Workload":
        d = dict(self.__dict__)
        d.update(kw)
        return Workload(**d)


# The workloads, named by what they are.  Sizes as stated for each.
WORKLOADS = {
    # 64 channels of 4.6875 MHz over 1250-1550 MHz, 0.25 ms, 4096 float32
    # samples of N(0,1), one boxcar (amp 2, width 4) at t=1000, DM 57.3;
    # 128 trials 0..127; whole series, time-domain output.
    "fdd_64ch_4096t_128dm": Workload(
        name="fdd_64ch_4096t_128dm", n_chan=64, band_lo_mhz=1250.0, band_hi_mhz=1550.0,
        t_samp_s=0.25e-3, n_t=4096, dtype="f32", dm0=0.0, ddm=1.0, n_dm=128, chunk_len=0,
        fixed_pulse=Pulse(t0=1000, dm=57.3, amp=2.0, width=4)),
    # survey-shaped: 1024 channels over 1210-1520 MHz, 64 us, 2^20 uint8
    # samples N(128,16) clipped, 5 pulses; 2048 trials 0..1023.5; 2^18 chunks.
    "fdd_1024ch_2p20t_2048dm": Workload(
        name="fdd_1024ch_2p20t_2048dm", n_chan=1024, band_lo_mhz=1210.0, band_hi_mhz=1520.0,
        t_samp_s=64e-6, n_t=1 << 20, dtype="u8", dm0=0.0, ddm=0.5, n_dm=2048,
        chunk_len=1 << 18, pulses_per_beam=5, noise_mean=128.0, noise_sigma=16.0),
    # 32 beams sharing the bins: 1024 channels over 1250-1550 MHz, 0.25 ms,
    # 2^19 float32 samples per beam; 4096 trials 0..2047.5; whole series.
    "fdd_32beam_1024ch_2p19t_4096dm": Workload(
        name="fdd_32beam_1024ch_2p19t_4096dm", n_chan=1024, band_lo_mhz=1250.0,
        band_hi_mhz=1550.0, t_samp_s=0.25e-3, n_t=1 << 19, dtype="f32", dm0=0.0, ddm=0.5,
        n_dm=4096, chunk_len=0, n_beams=32, pulses_per_beam=1),
    # low frequency, long delays: 4096 channels over 110-190 MHz, 491.52 us,
    # 2^21 float32 samples, 8192 trials 0..409.55; power spectra out; 16 beams.
    "fdd_16beam_4096ch_2p21t_8192dm_power": Workload(
        name="fdd_16beam_4096ch_2p21t_8192dm_power", n_chan=4096, band_lo_mhz=110.0,
        band_hi_mhz=190.0, t_samp_s=491.52e-6, n_t=1 << 21, dtype="f32", dm0=0.0, ddm=0.05,
        n_dm=8192, chunk_len=1 << 19, n_beams=16, output="power", pulses_per_beam=1),
}


def sky_delay_samples(w: Workload, dm: float) -> np.ndarray:
    """Sky-model arrival offsets (samples, rounded) of each channel for one DM."""
    nu = w.channel_centres()
    top = nu.max()
    return np.rint(dm * K_DM_SKY * (nu ** -2 - top ** -2) / w.t_samp_s).astype(np.int64)


def draw_pulses(w: Workload, rng: np.random.Generator) -> list[Pulse]:
    if w.fixed_pulse is not None:
        return [w.fixed_pulse]
    dms = w.dms()
    lo, hi = float(dms.min()), float(dms.max())
    out = []
    for _ in range(w.pulses_per_beam):
        dm = float(rng.uniform(lo, hi))
        sweep = int(sky_delay_samples(w, dm).max())
        t_hi = max(1, w.n_t - sweep - 4)
        out.append(Pulse(t0=int(rng.integers(0, t_hi)), dm=dm, amp=2.0 * w.noise_sigma, width=4))
    return out


def _noise_block(rng: np.random.Generator, w: Workload, rows: int) -> np.ndarray:
    z = rng.standard_normal((rows, w.n_chan), dtype=np.float32)
    if w.noise_sigma != 1.0:
        z *= np.float32(w.noise_sigma)
    if w.noise_mean != 0.0:
        z += np.float32(w.noise_mean)
    return z


def filterbank(w: Workload, seed: int, beam: int = 0, rows: int | None = None,
               block_rows: int = 1 << 14, threads: int | None = None):
    """One beam's [n_t, n_chan] time-major filterbank and its pulses.

    Pulses come from PCG64 seeded by (seed, beam); the noise of row block b
    (block_rows rows) from PCG64 seeded by (seed, beam, b), so blocks are
    drawn in parallel threads and ``rows`` < n_t returns exactly the leading
    rows of the full array.  u8 workloads are rounded and clipped to 0..255
    after the pulses are added.
    """
    pulses = draw_pulses(w, np.random.default_rng([seed, beam]))
    n_rows = w.n_t if rows is None else min(int(rows), w.n_t)
    out = np.empty((n_rows, w.n_chan), dtype=np.uint8 if w.dtype == "u8" else np.float32)
    sweeps = [(p, sky_delay_samples(w, p.dm)) for p in pulses]

    def fill(b: int) -> None:
        r0 = b * block_rows
        r1 = min(n_rows, r0 + block_rows)
        blk = _noise_block(np.random.default_rng([seed, beam, b]), w, r1 - r0)
        for p, off in sweeps:
            start = p.t0 + off
            for c in np.nonzero((start < r1) & (start + p.width > r0))[0]:
                a, e = max(int(start[c]), r0), min(int(start[c]) + p.width, r1)
                blk[a - r0: e - r0, c] += np.float32(p.amp)
        if w.dtype == "u8":
            np.rint(blk, out=blk)
            np.clip(blk, 0, 255, out=blk)
            out[r0:r1] = blk.astype(np.uint8)
        else:
            out[r0:r1] = blk

    n_blocks = (n_rows + block_rows - 1) // block_rows
    workers = threads or min(16, os.cpu_count() or 1)
    if workers > 1 and n_blocks > 1:
        with cf.ThreadPoolExecutor(max_workers=workers) as ex:
            list(ex.map(fill, range(n_blocks)))
    else:
        for b in range(n_blocks):
            fill(b)
    return out, pulses


@dataclass
class BatchWorkload:
    """Many beams of uneven length and uneven trial grids (the batching form)."""
    name: str
    n_beams: int
    n_chan: int
    band_lo_mhz: float
    band_hi_mhz: float
    t_samp_s: float
    n_t_lo: int          # beam lengths drawn log-uniformly in [n_t_lo, n_t_hi]
    n_t_hi: int
    trials_lo: int       # trial counts drawn uniformly from multiples of trials_step
    trials_hi: int
    trials_step: int
    ddm: float           # trials dm = 0, ddm, 2 ddm, ...
    output: str = "power"

    @property
    def dnu_mhz(self) -> float:
        return (self.band_hi_mhz - self.band_lo_mhz) / self.n_chan

    @property
    def nu_lo_mhz(self) -> float:
        return self.band_lo_mhz + 0.5 * self.dnu_mhz

    def beams(self, seed: int, n_t_div: int = 1):
        """[(n_t, dm0, ddm, n_dm)] per beam; lengths divided by n_t_div."""
        n_t = log_uniform_lengths(self.n_beams, self.n_t_lo, self.n_t_hi, seed) // n_t_div
        rng = np.random.default_rng([seed, 1])
        steps = np.arange(self.trials_lo, self.trials_hi + 1, self.trials_step)
        n_dm = rng.choice(steps, size=self.n_beams)
        return [(int(max(n, 2)), 0.0, self.ddm, int(m)) for n, m in zip(n_t, n_dm)]


BATCH_WORKLOADS = {
    # 96 beams, lengths log-uniform in 2^16..2^20 samples, 1536 channels over
    # 1100-1700 MHz, 81.92 us, 512..4096 trials (multiples of 64) of step 0.5.
    "fdd_96beam_1536ch_uneven": BatchWorkload(
        name="fdd_96beam_1536ch_uneven", n_beams=96, n_chan=1536, band_lo_mhz=1100.0,
        band_hi_mhz=1700.0, t_samp_s=81.92e-6, n_t_lo=1 << 16, n_t_hi=1 << 20, trials_lo=512,
        trials_hi=4096, trials_step=64, ddm=0.5),
}


# ------------------------------------------------- counter-based (Philox) inputs
def sweep_starts(nu_mhz: np.ndarray, t_samp_s: float, t0: int, dm: float) -> np.ndarray:
    """First sample of a pulse emitted at t0 (top channel) in every channel,
    along the sky-model sweep (module docstring)."""
    nu = np.asarray(nu_mhz, dtype=np.float64)
    return t0 + np.rint(dm * K_DM_SKY * (nu ** -2 - nu.max() ** -2) / t_samp_s).astype(np.int64)


def philox_pulses(nu_mhz: np.ndarray, t_samp_s: float, n_t: int, dm_lo: float, dm_hi: float,
                  seed: int, beam: int, n_pulses: int, amp: float = 2.0, width: int = 4):
    """Pulses of one beam for the counter-based generator: DMs uniform in
    [dm_lo, dm_hi], emission times uniform in [0, n_t - sweep - 4), drawn from
    PCG64 seeded by (seed, beam, 7).  Returns ([Pulse], [(starts, width, amp)])."""
    rng = np.random.default_rng([seed, beam, 7])
    pulses, specs = [], []
    for _ in range(n_pulses):
        dm = float(rng.uniform(dm_lo, dm_hi))
        starts0 = sweep_starts(nu_mhz, t_samp_s, 0, dm)
        t_hi = max(1, n_t - int(starts0.max()) - 4)
        t0 = int(rng.integers(0, t_hi))
        pulses.append(Pulse(t0=t0, dm=dm, amp=amp, width=width))
        specs.append((starts0 + t0, width, amp))
    return pulses, specs


def philox_beam_args(w: Workload, seed: int, beam: int) -> dict:
    """Keyword arguments of ``synth.philox.filterbank`` / ``synth.gpu.filterbank``
    for one beam of a workload (noise, 8-bit or float, the beam's pulses)."""
    dms = w.dms()
    pulses, specs = philox_pulses(w.channel_centres(), w.t_samp_s, w.n_t, float(dms.min()),
                                  float(dms.max()), seed, beam, w.pulses_per_beam,
                                  amp=2.0 * w.noise_sigma)
    return dict(n_chan=w.n_chan, seed=seed, beam=beam, mean=w.noise_mean, sigma=w.noise_sigma,
                u8=w.dtype == "u8", pulses=specs), pulses


def batch_beam_args(bw: "BatchWorkload", desc, seed: int, beam: int,
                    pulses_per_beam: int = 1) -> tuple[dict, list]:
    """Counter-based generator arguments for beam ``beam`` of a batch, whose
    (n_t, dm0, ddm, n_dm) is ``desc``: float32 N(0,1) noise and pulses with DMs
    in the beam's own trial range."""
    n_t, dm0, ddm, n_dm = desc
    nu = bw.nu_lo_mhz + bw.dnu_mhz * np.arange(bw.n_chan, dtype=np.float64)
    pulses, specs = philox_pulses(nu, bw.t_samp_s, int(n_t), float(dm0),
                                  float(dm0 + ddm * (n_dm - 1)), seed, beam, pulses_per_beam)
    return dict(n_chan=bw.n_chan, seed=seed, beam=beam, pulses=specs), pulses


def philox_filterbank(w: Workload, seed: int, beam: int = 0, t0: int = 0,
                      rows: int | None = None):
    """Host copy of rows [t0, t0 + rows) of one beam (counter-based generator);
    ``synth.gpu.filterbank`` makes the same bytes on the device."""
    from . import philox
    kw, pulses = philox_beam_args(w, seed, beam)
    n = w.n_t - t0 if rows is None else rows
    return philox.filterbank(n_rows=n, t0=t0, **kw), pulses


def log_uniform_lengths(n: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """n integers drawn log-uniformly in [lo, hi] (uneven beam lengths)."""
    rng = np.random.default_rng(seed)
    u = rng.uniform(math.log(lo), math.log(hi), size=n)
    return np.floor(np.exp(u)).astype(np.int64)

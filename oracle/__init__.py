"""FP64 CPU oracle for Fourier-domain dedispersion (arXiv 2110.03482).

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference legs may import this package.  It shares
no code with the CUDA path (``paper_2110_03482_gb300``) and never imports it.

The heavy loops live in ``fdd_oracle.c`` (plain C, FP64, libm, OpenMP); this
module compiles it with gcc, wraps it with ctypes and adds the chunking logic.

Readings of the paper that the oracle takes (each one listed in the design
notes as well):

* Phasor sign.  Eq. 2 writes the shifted series as I(t - Delta t) and Eq. 4
  writes W = exp(-2 pi i f Delta t); with the forward transform of Eq. 3 both
  would *delay* the low channels further.  The discard rule of Sect. 2.2 (the
  contaminated samples sit at the *end* of each series when dedispersing
  against the highest channel) only holds for an advance, so the oracle uses
  y[n] = x[n + d] and W = exp(+2 pi i k d / L).
* Reference frequency nu_0 (Eq. 1) defaults to the highest channel centre
  ("dedispersing against the highest observing frequency channel", Sect. 2.2).
* k_DM defaults to (2.41e-4)^-1 MHz^2 pc^-1 cm^3 s (Sect. 2.1).
* Channel frequencies are channel centres nu_c = nu_lo + c * dnu.
* Scaling of the inverse transform is 1/L, so a DM of zero returns the plain
  channel sum (the paper leaves ``apply_scaling`` unspecified, Sect. 3).
* The DC and Nyquist bins contribute only their real parts to the inverse
  transform (standard real-inverse convention; the paper is silent).
* Chunking.  chunk_len == 0: the whole series is zero padded to the next power
  of two (Sect. 3) and transformed once; the output keeps the first n_t
  samples, of which the last D_max are contaminated (Sect. 2.2).
  chunk_len == L > 0 (overlap-save): D_max = ceil(max delay in samples),
  hop = L - D_max, the valid output is n_out = n_t - D_max samples, and chunk
  c reads x[c*hop, c*hop + L) (zero beyond n_t) and keeps its first hop
  output samples (the discard rule of Sect. 2.2 applied per chunk).
* Spin-frequency-dependent DM grids (Sect. 2.3, Eqs. 8 and 9: the paper
  gives the scaled grid and says the result is to be re-sampled to the wanted
  trials, with no rule, and leaves the tolerable DM contraction open).  Bins
  are taken in groups of G consecutive bins from a first grouped bin
  K_min = max(1, ceil((G - 1) / eps)) on (bin 0, whose phasors are 1 at every
  DM, has no scaled grid), so that within a group the DM contraction
  1 - k / k_ref stays below eps; each group uses the phasors of its highest
  bin k_ref (Eq. 9 with f_s0 at k_ref), which for bin k evaluate Eq. 7 at the
  trial DMs DM'_j k_ref / k (Eq. 8), DM'_j = DM'_0 + j dDM over the scaled
  grid j = 0 .. n_s - 1 (DM'_0 = DM_0 + j_lo dDM reaches below DM_0 far
  enough, j_lo = 0 for DM_0 = 0 else floor(-eps DM_0 / dDM) - 1).  Bin k is
  re-sampled to trial t of the plan's grid by linear interpolation along the
  scaled trial axis at x = (DM_t k / k_ref - DM'_0) / dDM.  Bins below K_min
  follow Eq. 7 exactly.
* Down-sampling by a shorter inverse transform (Sect. 2.2, last paragraph:
  the paper names the technique, not its details).  A factor f (a power of
  two dividing L/2) keeps the bins k <= L/(2f) of the dedispersed spectrum
  and inverts them with length L/f, scaled by 1/L (not 1/(L/f)): that is the
  series low-passed to those bins and sampled every f native samples, at the
  native amplitude (a constant input keeps its level).  The kept Nyquist bin
  of the short transform contributes its real part only.  With chunking, the
  hop is rounded down to a multiple of f, so the chunks tile the down-sampled
  grid; the output keeps ceil(n_out / f) samples.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

K_DM_PAPER = 1.0 / 2.41e-4  # Sect. 2.1, constant of Eq. 1

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fdd_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle.so")
_lib = None
_lock = threading.Lock()

_dp = ctypes.POINTER(ctypes.c_double)
_i64p = ctypes.POINTER(ctypes.c_int64)


def build(force: bool = False, src: str = _SRC, out: str = _LIB_PATH) -> str:
    """Compile the C oracle with gcc (IEEE FP64, no contraction, OpenMP)."""
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(src):
        return out
    os.makedirs(os.path.dirname(out), exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", src, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def load_library(path: str) -> ctypes.CDLL:
    lib = ctypes.CDLL(path)
    lib.oracle_num_threads.restype = ctypes.c_int
    lib.oracle_delays.argtypes = [ctypes.c_int, _dp, ctypes.c_double, ctypes.c_double,
                                  ctypes.c_double, ctypes.c_int, _dp, _dp]
    lib.oracle_dft_r2c.argtypes = [ctypes.c_int64, _dp, ctypes.c_int64, ctypes.c_int64, _dp]
    lib.oracle_fft.argtypes = [ctypes.c_int64, _dp, ctypes.c_int]
    lib.oracle_fft.restype = ctypes.c_int
    lib.oracle_fft_r2c_many.argtypes = [ctypes.c_int64, ctypes.c_int64, _dp, _dp]
    lib.oracle_fft_r2c_many.restype = ctypes.c_int
    lib.oracle_fdd_bins.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_int64, _i64p, _dp,
                                    ctypes.c_int, _dp, _dp]
    lib.oracle_fdd_bins_spin.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_int64, _i64p,
                                         _dp, ctypes.c_int, _dp, ctypes.c_int, _dp,
                                         ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_int64, ctypes.c_int64, _dp]
    lib.oracle_fdd_bins_spin.restype = ctypes.c_int
    lib.oracle_irdft.argtypes = [ctypes.c_int64, _dp, _dp]
    lib.oracle_irfft_many.argtypes = [ctypes.c_int64, ctypes.c_int64, _dp, _dp]
    lib.oracle_irfft_many.restype = ctypes.c_int
    lib.oracle_tdd.argtypes = [ctypes.c_int, ctypes.c_int64, _dp, ctypes.c_int, _i64p,
                               ctypes.c_int, ctypes.c_int64, _dp]
    return lib


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            _lib = load_library(build())
        return _lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def _iptr(a: np.ndarray):
    return a.ctypes.data_as(_i64p)


def num_threads() -> int:
    return int(lib().oracle_num_threads())


# --------------------------------------------------------------------------
# Sect. 2.1, Eq. 1
# --------------------------------------------------------------------------
def channel_centres(n_chan: int, nu_lo_mhz: float, dnu_mhz: float) -> np.ndarray:
    return nu_lo_mhz + dnu_mhz * np.arange(n_chan, dtype=np.float64)


def delays(nu_mhz, dms, t_samp_s: float, k_dm: float = K_DM_PAPER,
           nu_ref_mhz: float | None = None) -> np.ndarray:
    """Eq. 1 in samples: d[j, c] = DM_j k_DM (nu_c^-2 - nu_ref^-2) / t_samp."""
    nu = _f64(nu_mhz)
    dm = _f64(dms)
    if nu_ref_mhz is None:
        nu_ref_mhz = float(nu.max())
    out = np.empty((dm.size, nu.size), dtype=np.float64)
    lib().oracle_delays(nu.size, _ptr(nu), float(nu_ref_mhz), float(k_dm), float(t_samp_s),
                        dm.size, _ptr(dm), _ptr(out))
    return out


# --------------------------------------------------------------------------
# Sect. 2.2, Eq. 3
# --------------------------------------------------------------------------
def dft_r2c(x, bins=None) -> np.ndarray:
    """Direct DFT of one real series at bins k0..k0+nk-1 (all L/2+1 if None)."""
    x = _f64(x)
    L = x.size
    if bins is None:
        k0, nk = 0, L // 2 + 1
    else:
        k0, nk = int(bins[0]), int(bins[1])
    out = np.empty(2 * nk, dtype=np.float64)
    lib().oracle_dft_r2c(L, _ptr(x), k0, nk, _ptr(out))
    return out[0::2] + 1j * out[1::2]


def fft_r2c(x) -> np.ndarray:
    """Radix-2 FFT of each row of x (rows of power-of-two length L) -> [rows, L/2+1]."""
    x = _f64(x)
    if x.ndim == 1:
        return fft_r2c(x[None, :])[0]
    rows, L = x.shape
    K = L // 2 + 1
    out = np.empty((rows, 2 * K), dtype=np.float64)
    rc = lib().oracle_fft_r2c_many(L, rows, _ptr(x), _ptr(out))
    if rc != 0:
        raise ValueError(f"oracle FFT failed (rc={rc}); L={L} must be a power of two")
    return out[:, 0::2] + 1j * out[:, 1::2]


def fft_c2c(z, sign: int) -> np.ndarray:
    """Complex radix-2 FFT with exponent sign (used by the self-tests)."""
    z = np.ascontiguousarray(z, dtype=np.complex128)
    buf = np.empty(2 * z.size, dtype=np.float64)
    buf[0::2] = z.real
    buf[1::2] = z.imag
    if lib().oracle_fft(z.size, _ptr(buf), int(sign)) != 0:
        raise ValueError("length must be a power of two")
    return buf[0::2] + 1j * buf[1::2]


# --------------------------------------------------------------------------
# Sect. 2.2, Eqs. 4 and 7
# --------------------------------------------------------------------------
def fdd_bins(X, bins, L: int, d) -> np.ndarray:
    """Y[j, q] = sum_c exp(+2 pi i k_q d[j, c] / L) X[c, q]  (Eqs. 4, 7)."""
    X = np.ascontiguousarray(X, dtype=np.complex128)
    n_chan, nq = X.shape
    b = np.ascontiguousarray(bins, dtype=np.int64)
    assert b.size == nq
    d = _f64(d)
    n_dm = d.shape[0]
    assert d.shape == (n_dm, n_chan)
    xi = np.empty(2 * X.size, dtype=np.float64)
    xi[0::2] = X.real.ravel()
    xi[1::2] = X.imag.ravel()
    out = np.empty(2 * n_dm * nq, dtype=np.float64)
    lib().oracle_fdd_bins(n_chan, int(L), nq, _iptr(b), _ptr(xi), n_dm, _ptr(d), _ptr(out))
    return (out[0::2] + 1j * out[1::2]).reshape(n_dm, nq)


# --------------------------------------------------------------------------
# Sect. 2.3, Eqs. 8 and 9 (reading in the module header)
# --------------------------------------------------------------------------
@dataclass
class SpinGroups:
    G: int          # bins per group
    eps: float      # largest relative DM contraction within a group
    k_min: int      # first grouped bin (bins below follow Eq. 7)
    j_lo: int       # the scaled grid starts at trial j_lo of the plan's grid
    n_s: int        # trials of the scaled grid


def spin_groups(K: int, dm0: float, ddm: float, n_dm: int, G: int, eps: float) -> SpinGroups:
    """Grouping of bins 0 .. K-1 for the spin-frequency-dependent DM grid."""
    if G < 1 or not eps > 0:
        raise ValueError("G >= 1 and eps > 0")
    # (bin 0 never groups: its phasors are 1 for every DM, Eq. 8 has no grid)
    k_min = min(K, max(1, int(math.ceil((G - 1) / eps))))
    j_lo = 0 if dm0 == 0 else int(math.floor(-eps * dm0 / ddm)) - 1
    return SpinGroups(G, eps, k_min, j_lo, n_dm - j_lo)


def spin_reference_bin(k: int, K: int, sg: SpinGroups) -> int:
    """k_ref of bin k: the highest bin of its group (k itself below k_min)."""
    if k < sg.k_min:
        return k
    g = (k - sg.k_min) // sg.G
    return min(sg.k_min + (g + 1) * sg.G, K) - 1


def fdd_bins_spin(X, bins, L: int, nu_mhz, dm0: float, ddm: float, n_dm: int,
                  t_samp_s: float, G: int, eps: float, k_dm: float = K_DM_PAPER,
                  nu_ref_mhz: float | None = None) -> np.ndarray:
    """Eq. 7 on the spin-frequency-dependent DM grids of Eqs. 8, 9, re-sampled
    to the trials dm0 + t ddm (t < n_dm) by linear interpolation; Y[t, q] for
    the spectra X[c, q] of the bins `bins` (module header)."""
    X = np.ascontiguousarray(X, dtype=np.complex128)
    n_chan, nq = X.shape
    b = np.ascontiguousarray(bins, dtype=np.int64)
    assert b.size == nq
    K = L // 2 + 1
    if n_dm < 2 or not ddm > 0:
        raise ValueError("the scaled grid needs at least two trials of positive step")
    sg = spin_groups(K, dm0, ddm, n_dm, G, eps)
    dm0s = dm0 + sg.j_lo * ddm
    d_s = delays(nu_mhz, dm0s + ddm * np.arange(sg.n_s), t_samp_s, k_dm, nu_ref_mhz)
    d_t = delays(nu_mhz, dm0 + ddm * np.arange(n_dm), t_samp_s, k_dm, nu_ref_mhz)
    xi = np.empty(2 * X.size, dtype=np.float64)
    xi[0::2] = X.real.ravel()
    xi[1::2] = X.imag.ravel()
    out = np.empty(2 * n_dm * nq, dtype=np.float64)
    rc = lib().oracle_fdd_bins_spin(n_chan, int(L), nq, _iptr(b), _ptr(xi), n_dm, _ptr(d_t),
                                    sg.n_s, _ptr(d_s), float(dm0), float(ddm), float(dm0s),
                                    int(sg.G), int(sg.k_min), _ptr(out))
    if rc != 0:
        raise ValueError("interpolation point outside the scaled grid")
    return (out[0::2] + 1j * out[1::2]).reshape(n_dm, nq)


# --------------------------------------------------------------------------
# Sect. 2.2, Eq. 6
# --------------------------------------------------------------------------
def irdft(Y, L: int) -> np.ndarray:
    """Direct inverse of a half spectrum (length L/2+1) to L real samples, 1/L scaled."""
    Y = np.ascontiguousarray(Y, dtype=np.complex128)
    assert Y.size == L // 2 + 1
    yi = np.empty(2 * Y.size, dtype=np.float64)
    yi[0::2] = Y.real
    yi[1::2] = Y.imag
    out = np.empty(L, dtype=np.float64)
    lib().oracle_irdft(int(L), _ptr(yi), _ptr(out))
    return out


def irfft(Y, L: int) -> np.ndarray:
    """Same inverse by the oracle FFT; Y is [rows, L/2+1] -> [rows, L]."""
    Y = np.ascontiguousarray(Y, dtype=np.complex128)
    if Y.ndim == 1:
        return irfft(Y[None, :], L)[0]
    rows, K = Y.shape
    assert K == L // 2 + 1
    yi = np.empty((rows, 2 * K), dtype=np.float64)
    yi[:, 0::2] = Y.real
    yi[:, 1::2] = Y.imag
    out = np.empty((rows, L), dtype=np.float64)
    if lib().oracle_irfft_many(int(L), rows, _ptr(yi), _ptr(out)) != 0:
        raise ValueError("L must be a power of two")
    return out


# --------------------------------------------------------------------------
# Sect. 2.1, Eq. 2
# --------------------------------------------------------------------------
def tdd(x, shifts, circular: bool, n_out: int | None = None) -> np.ndarray:
    """y[j, n] = sum_c x[c, n + s[j, c]] (integer shifts; circular or zero fill)."""
    x = _f64(x)
    n_chan, n_t = x.shape
    s = np.ascontiguousarray(shifts, dtype=np.int64)
    n_dm = s.shape[0]
    assert s.shape == (n_dm, n_chan)
    if n_out is None:
        n_out = n_t
    out = np.empty((n_dm, n_out), dtype=np.float64)
    lib().oracle_tdd(n_chan, n_t, _ptr(x), n_dm, _iptr(s), 1 if circular else 0, int(n_out),
                     _ptr(out))
    return out


# --------------------------------------------------------------------------
# Whole-pipeline oracle: chunking (the readings in the module header)
# --------------------------------------------------------------------------
@dataclass
class Geometry:
    L: int          # transform length
    K: int          # bins, L/2 + 1
    d_max: int      # ceil of the largest delay, samples
    hop: int        # output samples kept per chunk
    n_chunks: int
    n_out: int      # output samples per trial DM


def next_pow2(n: int) -> int:
    p = 1
    while p < n:
        p <<= 1
    return p


def geometry(n_t: int, chunk_len: int, d) -> Geometry:
    d = np.asarray(d, dtype=np.float64)
    d_max = int(math.ceil(float(d.max()))) if d.size else 0
    if d_max < 0:
        d_max = 0
    if chunk_len == 0:
        L = next_pow2(n_t)
        return Geometry(L, L // 2 + 1, d_max, n_t, 1, n_t)
    L = int(chunk_len)
    hop = L - d_max
    n_out = n_t - d_max
    if hop <= 0 or n_out <= 0:
        raise ValueError("chunk too short for the largest delay, or series too short")
    return Geometry(L, L // 2 + 1, d_max, hop, (n_out + hop - 1) // hop, n_out)


def chunk_series(x, geo: Geometry, c: int) -> np.ndarray:
    """Chunk c of a [n_chan, n_t] series: x[:, c*hop : c*hop + L], zero beyond n_t."""
    n_chan, n_t = x.shape
    out = np.zeros((n_chan, geo.L), dtype=np.float64)
    s = c * geo.hop
    e = min(s + geo.L, n_t)
    if e > s:
        out[:, : e - s] = x[:, s:e]
    return out


def spectra(x, geo: Geometry, c: int) -> np.ndarray:
    """Eq. 3 of chunk c for every channel: [n_chan, K] by the oracle FFT."""
    xc = chunk_series(x, geo, c)
    if geo.L & (geo.L - 1) == 0:
        return fft_r2c(xc)
    return np.stack([dft_r2c(row) for row in xc])


def geometry_downsampled(n_t: int, chunk_len: int, d, f: int) -> Geometry:
    """geometry() with the hop rounded down to a multiple of the factor f and
    n_out counted in down-sampled samples (reading in the module header)."""
    g = geometry(n_t, chunk_len, d)
    if f == 1:
        return g
    if f < 1 or f & (f - 1) or g.L % (2 * f):
        raise ValueError("f must be a power of two dividing L/2")
    if chunk_len == 0:  # one chunk: keep ceil(n_t / f) samples
        n_out = -(-g.n_out // f)
        return Geometry(g.L, g.K, g.d_max, n_out * f, 1, n_out)
    hop = g.hop // f * f
    if hop <= 0:
        raise ValueError("chunk too short for the largest delay at this factor")
    n_out_native = g.n_out
    return Geometry(g.L, g.K, g.d_max, hop, -(-n_out_native // hop), -(-n_out_native // f))


def fdd_time_downsampled(x, d, chunk_len: int, f: int) -> np.ndarray:
    """FDD with the inverse transform shortened by f (Sect. 2.2, last
    paragraph): per chunk, Eq. 7 on the bins k <= L/(2f) only, then their
    inverse of length L/f scaled by 1/L; y [n_dm, ceil(n_out / f)]."""
    x = _f64(x)
    n_t = x.shape[1]
    geo = geometry_downsampled(n_t, chunk_len, d, f)
    Ls = geo.L // f
    bins = np.arange(Ls // 2 + 1, dtype=np.int64)
    y = np.empty((d.shape[0], geo.n_out), dtype=np.float64)
    for c in range(geo.n_chunks):
        X = spectra(x, geometry(n_t, chunk_len, d) if chunk_len == 0 else
                    Geometry(geo.L, geo.K, geo.d_max, geo.hop, geo.n_chunks, n_t - geo.d_max), c)
        Y = fdd_bins(X[:, : bins.size], bins, geo.L, d)
        yc = irfft(Y, Ls) / f  # irfft scales by f / L: back to 1 / L
        s = c * geo.hop // f
        n = min(geo.hop // f, geo.n_out - s)
        y[:, s: s + n] = yc[:, :n]
    return y


def fdd_time(x, d, chunk_len: int) -> np.ndarray:
    """Full FDD of one beam: x [n_chan, n_t] -> y [n_dm, n_out] (Eqs. 3, 4, 7, 6)."""
    x = _f64(x)
    geo = geometry(x.shape[1], chunk_len, d)
    y = np.empty((d.shape[0], geo.n_out), dtype=np.float64)
    bins = np.arange(geo.K, dtype=np.int64)
    for c in range(geo.n_chunks):
        X = spectra(x, geo, c)
        Y = fdd_bins(X, bins, geo.L, d)
        yc = irfft(Y, geo.L) if geo.L & (geo.L - 1) == 0 else np.stack(
            [irdft(r, geo.L) for r in Y])
        s = c * geo.hop
        n = min(geo.hop, geo.n_out - s)
        y[:, s: s + n] = yc[:, :n]
    return y

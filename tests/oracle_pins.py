"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each ``pin_*`` function raises AssertionError when the oracle is wrong.  They
are run as tests by ``test_oracle_pins.py`` and, against copies of the oracle
with planted mistakes, by ``test_oracle_mutations.py``.  None of them re-types
the oracle's own formula: each compares with an independent quantity (a
closed form in other units, a brute-force shift-and-sum, a library FFT, a
textbook identity, or a simulated pulse).
"""
from __future__ import annotations

import os

import numpy as np

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _rng(seed):
    return np.random.default_rng(seed)


# ---------------------------------------------------------------- Eq. 1
def pin_delay_law_golden():
    """Eq. 1 against the paper's constant and textbook closed-form values."""
    rows = []
    k_paper = None
    with open(os.path.join(GOLDEN, "delay_law.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("k_dm_paper"):
                k_paper = float(line.split()[1])
                continue
            rows.append([float(v) for v in line.split()])
    assert k_paper is not None and abs(oracle.K_DM_PAPER / k_paper - 1) < 1e-12
    for f_lo, f_hi, dm, ts, kdm, expect, tol in rows:
        d = oracle.delays([f_lo, f_hi], [dm], ts, k_dm=kdm, nu_ref_mhz=f_hi)
        assert abs(d[0, 0] / expect - 1) < tol, (d[0, 0], expect)
        assert d[0, 1] == 0.0  # the reference channel itself has no delay


def pin_delay_law_scaling():
    """Delay is linear in DM, zero at DM 0, and positive below nu_ref."""
    nu = np.array([1200.0, 1300.0, 1400.0])
    d = oracle.delays(nu, [0.0, 1.0, 3.0], 1e-3, nu_ref_mhz=1400.0)
    assert np.all(d[0] == 0.0)
    assert np.allclose(d[2], 3.0 * d[1], rtol=1e-14, atol=0)
    assert d[1, 0] > d[1, 1] > d[1, 2] == 0.0


# ---------------------------------------------------------------- Eq. 3
def pin_dft_closed_forms():
    """Direct DFT: a delta and a cosine give their textbook spectra."""
    L = 64
    x = np.zeros(L)
    x[5] = 1.0
    X = oracle.dft_r2c(x)
    k = np.arange(L // 2 + 1)
    ref = np.exp(-2j * np.pi * ((k * 5) % L) / L)
    assert np.max(np.abs(X - ref)) < 1e-13
    n = np.arange(L)
    X = oracle.dft_r2c(np.cos(2 * np.pi * 3 * n / L))
    expect = np.zeros(L // 2 + 1, complex)
    expect[3] = L / 2
    assert np.max(np.abs(X - expect)) < 1e-12


def pin_fft_matches_dft_and_numpy():
    """Oracle FFT == its direct DFT == numpy's rfft (an independent library)."""
    x = _rng(1).standard_normal((3, 256))
    F = oracle.fft_r2c(x)
    D = np.stack([oracle.dft_r2c(r) for r in x])
    N = np.fft.rfft(x, axis=1)
    scale = np.max(np.abs(N))
    assert np.max(np.abs(F - N)) < 1e-12 * scale
    assert np.max(np.abs(D - N)) < 1e-11 * scale


# ---------------------------------------------------------------- Eq. 6
def pin_inverse_matches_numpy_and_roundtrip():
    """irfft / irdft equal numpy's irfft (imag of DC and Nyquist ignored)."""
    L = 128
    Y = _rng(2).standard_normal(L // 2 + 1) + 1j * _rng(3).standard_normal(L // 2 + 1)
    ref = np.fft.irfft(Y, L)
    assert np.max(np.abs(oracle.irfft(Y, L) - ref)) < 1e-13
    assert np.max(np.abs(oracle.irdft(Y, L) - ref)) < 1e-12
    x = _rng(4).standard_normal(L)
    assert np.max(np.abs(oracle.irfft(oracle.fft_r2c(x), L) - x)) < 1e-12


# ---------------------------------------------------------------- Eq. 2
def pin_tdd_hand_example():
    """Brute-force TDD against a hand-worked two-channel example."""
    x = np.array([[1.0, 2.0, 3.0, 4.0], [10.0, 20.0, 30.0, 40.0]])
    s = np.array([[0, 0], [1, 0], [0, 2]])
    y = oracle.tdd(x, s, circular=True)
    expect = np.array([[11, 22, 33, 44], [12, 23, 34, 41], [31, 42, 13, 24]], float)
    assert np.array_equal(y, expect)
    y = oracle.tdd(x, s, circular=False)
    expect = np.array([[11, 22, 33, 44], [12, 23, 34, 40], [31, 42, 3, 4]], float)
    assert np.array_equal(y, expect)


# ---------------------------------------------------------------- Eqs. 4, 7
def pin_dm_zero_is_channel_sum():
    """At DM 0 every phasor is 1: Y is the plain sum over channels (Eq. 7)."""
    X = _rng(5).standard_normal((7, 9)) + 1j * _rng(6).standard_normal((7, 9))
    bins = np.arange(9)
    Y = oracle.fdd_bins(X, bins, 16, np.zeros((3, 7)))
    for j in range(3):
        assert np.max(np.abs(Y[j] - X.sum(axis=0))) < 1e-13


def pin_integer_shift_equals_tdd():
    """Fourier shift theorem: FDD with integer delays == circular brute-force TDD.

    Pins the phasor sign, the factor k, the 1/L in the phase and the index
    order of the delay table in one go (Eqs. 2, 3, 4, 6, 7).
    """
    rng = _rng(7)
    n_chan, L, n_dm = 5, 64, 4
    x = rng.standard_normal((n_chan, L))
    shifts = rng.integers(0, L, size=(n_dm, n_chan))
    X = oracle.fft_r2c(x)
    Y = oracle.fdd_bins(X, np.arange(L // 2 + 1), L, shifts.astype(float))
    y = oracle.irfft(Y, L)
    ref = oracle.tdd(x, shifts, circular=True)
    assert np.max(np.abs(y - ref)) < 1e-12 * np.max(np.abs(ref))


def pin_fractional_shift_of_sinusoid():
    """A band-limited sinusoid shifted by a fractional delay is the advanced sinusoid.

    x_c[n] = cos(2 pi k0 n / L + phi_c); after FDD each channel reads
    cos(2 pi k0 (n + d_c) / L + phi_c), summed over channels.
    """
    rng = _rng(8)
    n_chan, L, k0 = 4, 32, 5
    n = np.arange(L)
    phi = rng.uniform(0, 2 * np.pi, n_chan)
    d = rng.uniform(0, 40, size=(2, n_chan))
    x = np.cos(2 * np.pi * k0 * n[None, :] / L + phi[:, None])
    Y = oracle.fdd_bins(oracle.fft_r2c(x), np.arange(L // 2 + 1), L, d)
    y = oracle.irfft(Y, L)
    for j in range(2):
        ref = np.cos(2 * np.pi * k0 * (n[None, :] + d[j][:, None]) / L + phi[:, None]).sum(0)
        assert np.max(np.abs(y[j] - ref)) < 1e-11


def pin_large_phase_reduction():
    """Phases of ~1e4 cycles still rotate exactly: a delta shifted by a large
    integer delay returns to itself modulo L (Eq. 4 at large k d / L)."""
    L = 4096
    x = np.zeros((1, L))
    x[0, 17] = 1.0
    d = np.array([[L * 7919.0 + 17.0]])  # advance by 17 modulo L
    Y = oracle.fdd_bins(oracle.fft_r2c(x), np.arange(L // 2 + 1), L, d)
    y = oracle.irfft(Y, L)[0]
    expect = np.zeros(L)
    expect[0] = 1.0
    assert np.max(np.abs(y - expect)) < 1e-9


def pin_unit_modulus():
    """Phasors are pure rotations: with one channel |Y| == |X| (Sect. 2.2)."""
    rng = _rng(9)
    X = rng.standard_normal((1, 33)) + 1j * rng.standard_normal((1, 33))
    d = rng.uniform(0, 100, size=(6, 1))
    Y = oracle.fdd_bins(X, np.arange(33), 64, d)
    assert np.max(np.abs(np.abs(Y) - np.abs(X))) < 1e-12


def pin_linearity():
    rng = _rng(10)
    X1 = rng.standard_normal((3, 8)) + 1j * rng.standard_normal((3, 8))
    X2 = rng.standard_normal((3, 8)) + 1j * rng.standard_normal((3, 8))
    d = rng.uniform(0, 50, size=(4, 3))
    b = np.arange(8)
    lhs = oracle.fdd_bins(2.0 * X1 - 3.0 * X2, b, 16, d)
    rhs = 2.0 * oracle.fdd_bins(X1, b, 16, d) - 3.0 * oracle.fdd_bins(X2, b, 16, d)
    assert np.max(np.abs(lhs - rhs)) < 1e-12


def pin_sum_ifft_swap():
    """Eq. 5 == Eq. 6: per-channel inverse transforms summed == one inverse of the sum."""
    rng = _rng(11)
    n_chan, L = 3, 32
    x = rng.standard_normal((n_chan, L))
    d = rng.uniform(0, 20, size=(2, n_chan))
    X = oracle.fft_r2c(x)
    bins = np.arange(L // 2 + 1)
    one = oracle.irfft(oracle.fdd_bins(X, bins, L, d), L)
    per = np.zeros((2, L))
    for c in range(n_chan):
        per += oracle.irfft(oracle.fdd_bins(X[c:c + 1], bins, L, d[:, c:c + 1]), L)
    assert np.max(np.abs(one - per)) < 1e-12


def pin_bin_subset_consistent():
    """Evaluating a subset of bins gives the same values as the full set."""
    rng = _rng(12)
    X = rng.standard_normal((4, 17)) + 1j * rng.standard_normal((4, 17))
    d = rng.uniform(0, 30, size=(3, 4))
    full = oracle.fdd_bins(X, np.arange(17), 32, d)
    sub = np.array([0, 3, 16])
    part = oracle.fdd_bins(X[:, sub], sub, 32, d)
    assert np.max(np.abs(full[:, sub] - part)) < 1e-14


# ---------------------------------------------------------------- whole pipeline
def pin_injected_pulse_peaks_at_its_dm():
    """The 64-channel workload's simulated pulse (DM 57.3, t=1000) comes out at
    trial 57 and sample ~1000 (Fig. 1 narrative: delays removed, pulses aligned).
    """
    w = synth.WORKLOADS["fdd_64ch_4096t_128dm"]
    fb, pulses = synth.filterbank(w, seed=20211008)
    x = fb.T.astype(np.float64)
    d = oracle.delays(w.channel_centres(), w.dms(), w.t_samp_s)
    y = oracle.fdd_time(x, d, w.chunk_len)
    j, n = np.unravel_index(np.argmax(y), y.shape)
    assert j == 57, (j, n)
    assert 998 <= n <= 1004, (j, n)


def pin_contamination_only_at_end():
    """Circular FDD with integer delays equals zero-fill TDD except in the last
    D_max samples (the discard rule of Sect. 2.2)."""
    rng = _rng(13)
    n_chan, L = 6, 128
    x = rng.standard_normal((n_chan, L))
    shifts = np.stack([np.arange(n_chan)[::-1] * 3, np.arange(n_chan)[::-1] * 5])
    dmax = int(shifts.max())
    X = oracle.fft_r2c(x)
    y = oracle.irfft(oracle.fdd_bins(X, np.arange(L // 2 + 1), L, shifts.astype(float)), L)
    lin = oracle.tdd(x, shifts, circular=False)
    good = L - dmax
    assert np.max(np.abs(y[:, :good] - lin[:, :good])) < 1e-12
    assert np.max(np.abs(y[:, good:] - lin[:, good:])) > 1e-3


def pin_overlap_save_equals_linear_tdd():
    """Chunked FDD (overlap-save) with integer delays equals the zero-fill
    brute-force TDD over the whole valid output."""
    rng = _rng(14)
    n_chan, n_t = 4, 300
    x = rng.standard_normal((n_chan, n_t))
    shifts = np.array([[9, 6, 3, 0], [0, 0, 0, 0], [21, 14, 7, 0]])
    y = oracle.fdd_time(x, shifts.astype(float), chunk_len=64)
    geo = oracle.geometry(n_t, 64, shifts)
    assert geo.d_max == 21 and geo.hop == 43 and geo.n_out == 279 and geo.n_chunks == 7
    ref = oracle.tdd(x, shifts, circular=False, n_out=geo.n_out)
    assert np.max(np.abs(y - ref)) < 1e-12


# ---------------------------------------------------------------- Sect. 2.3, Eqs. 8, 9
def _spin_case(seed=5, n_chan=24, L=4096, dm0=3.0, ddm=0.25, n_dm=48):
    rng = _rng(seed)
    nu = oracle.channel_centres(n_chan, 1150.0, 12.5)
    bins = np.array([0, 1, 37, 499, 500, 501, 1023, 1500, 2047, 2048])
    X = rng.standard_normal((n_chan, bins.size)) + 1j * rng.standard_normal((n_chan, bins.size))
    d = oracle.delays(nu, dm0 + ddm * np.arange(n_dm), 1e-3)
    return nu, bins, X, d, L, dm0, ddm, n_dm


def pin_spin_groups_of_one_are_eq7():
    """Groups of one bin: every bin is its own reference (Eq. 8 scales by
    k/k = 1), so the scaled grid is the plan's grid, shifted below DM_0 > 0,
    and the result is Eq. 7 exactly (brute-force reference)."""
    nu, bins, X, d, L, dm0, ddm, n_dm = _spin_case()
    ref = oracle.fdd_bins(X, bins, L, d)
    got = oracle.fdd_bins_spin(X, bins, L, nu, dm0, ddm, n_dm, 1e-3, G=1, eps=0.01)
    assert np.max(np.abs(got - ref)) <= 1e-11 * np.max(np.abs(ref))


def pin_spin_group_top_bins_are_eq7():
    """The highest bin of a group is its own reference: Eq. 7 exactly there;
    bins below the first group are Eq. 7 too; other bins differ."""
    nu, bins, X, d, L, dm0, ddm, n_dm = _spin_case()
    K = L // 2 + 1
    G, eps = 16, 0.05
    sg = oracle.spin_groups(K, dm0, ddm, n_dm, G, eps)
    assert sg.k_min == 300 and sg.j_lo < 0
    ref = oracle.fdd_bins(X, bins, L, d)
    got = oracle.fdd_bins_spin(X, bins, L, nu, dm0, ddm, n_dm, 1e-3, G=G, eps=eps)
    for q, k in enumerate(bins):
        top = k < sg.k_min or (k - sg.k_min) % G == G - 1 or k == K - 1
        err = np.max(np.abs(got[:, q] - ref[:, q])) / np.max(np.abs(ref[:, q]))
        if top:
            assert err <= 1e-11, (k, err)
        else:
            assert err > 1e-9, (k, err)


def pin_spin_single_tone_within_interpolation_bound():
    """A unit tone in one channel: Eq. 7 of bin k at DM is exp(i a_k DM) and
    the scaled grid samples exp(i a_ref DM') at DM' = DM'_0 + j dDM, the same
    exponential of DM k_ref / k.  Linear interpolation between unit-spaced
    samples of exp(i b x) errs by at most b^2 / 8 (the textbook bound
    h^2 max|f''| / 8), b = a_ref dDM the phase step of the scaled grid; half
    way between samples the error comes within a few percent of it."""
    n_chan, L, dm0, ddm, n_dm = 8, 8192, 0.0, 0.05, 400
    nu = oracle.channel_centres(n_chan, 1150.0, 25.0)
    K = L // 2 + 1
    G, eps = 32, 0.02
    c1 = 0  # the lowest channel: the largest delay
    bins = np.array([2500, 2517, 3100, 3131, 4000])
    X = np.zeros((n_chan, bins.size), dtype=np.complex128)
    X[c1, :] = 1.0
    d = oracle.delays(nu, dm0 + ddm * np.arange(n_dm), 1e-3)
    exact = oracle.fdd_bins(X, bins, L, d)
    got = oracle.fdd_bins_spin(X, bins, L, nu, dm0, ddm, n_dm, 1e-3, G=G, eps=eps)
    rate = oracle.delays(nu, [1.0], 1e-3)[0, c1]  # samples of delay per unit DM
    sg = oracle.spin_groups(K, dm0, ddm, n_dm, G, eps)
    worst = 0.0
    for q, k in enumerate(bins):
        k_ref = oracle.spin_reference_bin(int(k), K, sg)
        b = 2 * np.pi * k_ref * rate * ddm / L
        bound = b * b / 8
        err = np.abs(got[:, q] - exact[:, q])
        assert np.max(err) <= bound * (1 + 1e-6) + 1e-12, (k, np.max(err), bound)
        if k != k_ref:
            worst = max(worst, np.max(err) / bound)
    assert worst > 0.9, worst


def pin_downsampled_inverse_f1_is_fdd_time():
    """A shortening factor of 1 is the plain inverse (whole series and chunked)."""
    rng = _rng(41)
    nu = 1200.0 + 10.0 * np.arange(8)
    d = oracle.delays(nu, 1.5 * np.arange(6), 1e-3)
    x = rng.standard_normal((8, 1000))
    for chunk in (0, 256):
        assert np.array_equal(oracle.fdd_time_downsampled(x, d, chunk, 1),
                              oracle.fdd_time(x, d, chunk))


def pin_downsampled_inverse_decimates_band_limited_series():
    """Sect. 2.2, last paragraph: with every input bin below L/(2f), shortening
    the inverse transform by f returns every f-th sample of the full output
    (nothing above the kept bins to lose), at the native amplitude."""
    L, f = 1024, 4
    n = np.arange(L)
    nu = 1200.0 + 10.0 * np.arange(8)
    d = oracle.delays(nu, 2.0 * np.arange(5), 1e-3)
    x = np.stack([np.cos(2 * np.pi * (3 + c) * n / L + c) + 0.5 * np.sin(2 * np.pi * (40 + c) * n / L)
                  for c in range(8)])
    full = oracle.fdd_time(x, d, 0)
    short = oracle.fdd_time_downsampled(x, d, 0, f)
    assert short.shape == (5, L // f)
    assert np.max(np.abs(short - full[:, ::f])) < 1e-12
    # a constant filling the whole transform keeps its level (DC scaled by 1/L)
    const = oracle.fdd_time_downsampled(np.full((8, L), 3.0), d, 0, f)
    assert np.allclose(const, 24.0, atol=1e-12)


def pin_downsampled_chunks_tile_the_grid():
    """Chunked, the hop is a multiple of f, the output has ceil(n_out / f)
    samples, and a constant input (a pure DC bin in every full chunk, whatever
    the circular shifts) comes out at the native level n_chan * value in every
    chunk that lies inside the series."""
    f = 2
    nu = 1200.0 + 10.0 * np.arange(4)
    d = oracle.delays(nu, np.arange(3.0), 1e-3)
    geo = oracle.geometry_downsampled(4000, 512, d, f)
    assert geo.hop % f == 0 and geo.n_out == -(-(4000 - geo.d_max) // f)
    y = oracle.fdd_time_downsampled(np.full((4, 4000), 3.0), d, 512, f)
    assert y.shape == (3, geo.n_out)
    full_chunks = (4000 - geo.L) // geo.hop + 1  # chunks read entirely inside the series
    m = full_chunks * geo.hop // f
    assert m > 0 and np.allclose(y[:, :m], 12.0, atol=1e-11)


ALL_PINS = [
    pin_spin_groups_of_one_are_eq7,
    pin_spin_group_top_bins_are_eq7,
    pin_spin_single_tone_within_interpolation_bound,
    pin_downsampled_inverse_f1_is_fdd_time,
    pin_downsampled_inverse_decimates_band_limited_series,
    pin_downsampled_chunks_tile_the_grid,
    pin_delay_law_golden,
    pin_delay_law_scaling,
    pin_dft_closed_forms,
    pin_fft_matches_dft_and_numpy,
    pin_inverse_matches_numpy_and_roundtrip,
    pin_tdd_hand_example,
    pin_dm_zero_is_channel_sum,
    pin_integer_shift_equals_tdd,
    pin_fractional_shift_of_sinusoid,
    pin_large_phase_reduction,
    pin_unit_modulus,
    pin_linearity,
    pin_sum_ifft_swap,
    pin_bin_subset_consistent,
    pin_injected_pulse_peaks_at_its_dm,
    pin_contamination_only_at_end,
    pin_overlap_save_equals_linear_tdd,
]

"""Plant plausible mistakes in a copy of the oracle (on the CPU) and check that
at least one pin catches each of them.  The committed oracle source is never
modified: every mutant is a text substitution compiled into a temporary
library that is swapped in for the duration of one check.
"""
import contextlib
import os

import pytest

import oracle
import oracle_pins

# (name, text in fdd_oracle.c, replacement).  Each text must occur exactly once.
MUTATIONS = [
    ("phasor_sign", "double wr = cos(TWO_PI * p), wi = sin(TWO_PI * p);",
     "double wr = cos(TWO_PI * p), wi = -sin(TWO_PI * p);"),
    ("phase_drops_k", "double p = k * d[(int64_t)j * n_chan + c] / (double)L;",
     "double p = d[(int64_t)j * n_chan + c] / (double)L;"),
    ("phase_uses_K_not_L", "double p = k * d[(int64_t)j * n_chan + c] / (double)L;",
     "double p = k * d[(int64_t)j * n_chan + c] / (double)(L / 2 + 1);"),
    ("delay_one_channel", "double p = k * d[(int64_t)j * n_chan + c] / (double)L;",
     "double p = k * d[(int64_t)j * n_chan] / (double)L;"),
    ("mac_drops_cross_term", "re += wr * xr - wi * xi;", "re += wr * xr;"),
    ("mac_imag_sign", "im += wr * xi + wi * xr;", "im += wr * xi - wi * xr;"),
    ("phase_reduced_in_fp32", "p -= floor(p);", "p = (float)p - floorf((float)p);"),
    ("delay_wrong_power",
     "(1.0 / (nu_mhz[c] * nu_mhz[c]) - 1.0 / (nu_ref_mhz * nu_ref_mhz))",
     "(1.0 / nu_mhz[c] - 1.0 / nu_ref_mhz)"),
    ("delay_times_tsamp", "d_out[(int64_t)j * n_chan + c] = dt / t_samp_s;",
     "d_out[(int64_t)j * n_chan + c] = dt * t_samp_s;"),
    ("fft_forward_sign", "oracle_fft(L, z, -1);", "oracle_fft(L, z, +1);"),
    ("fft_twiddle_sign", "double wr = cos(ang), wi = sin(ang);",
     "double wr = cos(ang), wi = -sin(ang);"),
    ("dft_sign", "im -= x[n] * sin(ang);", "im += x[n] * sin(ang);"),
    ("irfft_no_scale", "y[s * L + n] = z[2 * n] / (double)L;", "y[s * L + n] = z[2 * n];"),
    ("irfft_no_conjugate", "z[2 * k + 1] = -h[2 * (L - k) + 1];",
     "z[2 * k + 1] = h[2 * (L - k) + 1];"),
    ("irdft_no_factor_two", "acc += 2.0 * t;", "acc += t;"),
    ("tdd_delays_instead", "int64_t t = n + shift[(int64_t)j * n_chan + c];",
     "int64_t t = n - shift[(int64_t)j * n_chan + c];"),
    ("tdd_wrong_modulus", "t %= n_t;", "t %= (n_t - 1);"),
    ("spin_phasor_of_bin_not_reference",
     "spin_sum((double)k_ref, d_s + (int64_t)j * n_chan",
     "spin_sum((double)k, d_s + (int64_t)j * n_chan"),
    ("spin_ratio_inverted", "((double)k / (double)k_ref)", "((double)k_ref / (double)k)"),
    ("spin_nearest_not_interpolated", "double delta = x - (double)m;",
     "double delta = 0.0;"),
    ("spin_grid_origin_ignored", "- dm0s) / ddm;", "- dm0) / ddm;"),
    ("spin_phase_drops_cross_term", "sr += cr * a - ci * b;", "sr += cr * a;"),
]


@contextlib.contextmanager
def _mutant(tmp_path, text, repl):
    with open(oracle._SRC) as f:
        src = f.read()
    assert src.count(text) == 1, f"mutation anchor not unique: {text!r}"
    path = os.path.join(str(tmp_path), "mutant.c")
    with open(path, "w") as f:
        f.write(src.replace(text, repl))
    so = oracle.build(force=True, src=path, out=os.path.join(str(tmp_path), "libmutant.so"))
    mlib = oracle.load_library(so)
    old = oracle.lib()
    oracle._lib = mlib
    try:
        yield
    finally:
        oracle._lib = old


@pytest.mark.parametrize("name,text,repl", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_catch_mutation(tmp_path, name, text, repl):
    caught = []
    with _mutant(tmp_path, text, repl):
        for pin in oracle_pins.ALL_PINS:
            try:
                pin()
            except AssertionError:
                caught.append(pin.__name__)
            except ValueError:
                caught.append(pin.__name__)
    assert caught, f"no pin caught the planted mistake {name!r}"


def test_unmutated_copy_passes(tmp_path):
    """Control: the copy-and-rebuild machinery itself does not trip the pins."""
    with _mutant(tmp_path, "p -= floor(p);", "p -= floor(p);"):
        for pin in oracle_pins.ALL_PINS:
            pin()

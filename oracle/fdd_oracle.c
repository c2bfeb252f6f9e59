/*
 * fdd_oracle.c -- slow, plain FP64 CPU oracle for Fourier-domain dedispersion.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and
 * its Python binding) may include, link or call this file.  It shares no code,
 * header, table or constant with the CUDA path.  Only the tests, the smoke
 * check and the benchmark's CPU-baseline leg use it.
 *
 * Every function is the plain definition from the paper (Bassa et al.,
 * "Fourier-domain dedispersion", arXiv 2110.03482), written out without
 * blocking, fusion or recurrences:
 *
 *   oracle_delays     Sect. 2.1, Eq. 1   dispersion delay, in samples
 *   oracle_dft_r2c    Sect. 2.2, Eq. 3   forward Fourier transform, direct sum
 *   oracle_fft        Sect. 2.2, Eq. 3   the same transform by radix-2 FFT
 *   oracle_fdd_bins   Sect. 2.2, Eqs. 4 and 7   phasors and sum over channels
 *   oracle_fdd_bins_spin  Sect. 2.3, Eqs. 8, 9   the same on spin-frequency-
 *                     dependent DM grids, re-sampled to the plan's trials
 *   oracle_irdft      Sect. 2.2, Eq. 6   inverse transform back to time
 *   oracle_tdd        Sect. 2.1, Eq. 2   brute-force time-domain shift-and-sum
 *
 * Sign convention (a reading of the paper, see the Python driver's header):
 * the forward transform is X[k] = sum_n x[n] exp(-2 pi i k n / L) (Eq. 3) and
 * the phasor that removes a dispersion delay of d samples is
 * exp(+2 pi i k d / L), i.e. it ADVANCES channel nu by d samples so that the
 * dispersed pulse lines up with its arrival time at the reference frequency.
 *
 * Complex arrays are interleaved (re, im) doubles.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

static const double TWO_PI = 6.283185307179586476925286766559;

int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/*
 * Eq. 1: Delta t(nu, DM) = DM * k_DM * (nu^-2 - nu_0^-2), expressed in samples
 * by dividing by the sampling time.  nu in MHz, k_DM in MHz^2 pc^-1 cm^3 s.
 * d_out[j * n_chan + c] is the delay of channel c at trial DM dm[j].
 */
void oracle_delays(int n_chan, const double* nu_mhz, double nu_ref_mhz,
                   double k_dm, double t_samp_s, int n_dm, const double* dm,
                   double* d_out) {
  for (int j = 0; j < n_dm; ++j) {
    for (int c = 0; c < n_chan; ++c) {
      double dt = dm[j] * k_dm *
                  (1.0 / (nu_mhz[c] * nu_mhz[c]) - 1.0 / (nu_ref_mhz * nu_ref_mhz));
      d_out[(int64_t)j * n_chan + c] = dt / t_samp_s;
    }
  }
}

/*
 * Eq. 3 as a direct sum, for bins k0 .. k0+nk-1 of a length-L real series:
 *   X[k] = sum_{n=0}^{L-1} x[n] exp(-2 pi i k n / L).
 * The twiddle index (k n mod L) is formed exactly in integers, and the
 * twiddle itself comes from libm cos/sin of 2 pi m / L.
 */
void oracle_dft_r2c(int64_t L, const double* x, int64_t k0, int64_t nk,
                    double* X) {
  for (int64_t q = 0; q < nk; ++q) {
    int64_t k = k0 + q;
    double re = 0.0, im = 0.0;
    for (int64_t n = 0; n < L; ++n) {
      int64_t m = (int64_t)(((__int128)k * n) % L);
      double ang = TWO_PI * (double)m / (double)L;
      re += x[n] * cos(ang);
      im -= x[n] * sin(ang);
    }
    X[2 * q] = re;
    X[2 * q + 1] = im;
  }
}

/*
 * In-place iterative radix-2 complex FFT of length L (a power of two) with
 * sign s: out[k] = sum_n in[n] exp(s * 2 pi i k n / L).  Twiddles come from
 * libm for every index (no twiddle recurrence).  Returns 0, or -1 when L is
 * not a power of two.
 */
int oracle_fft(int64_t L, double* z, int sign) {
  if (L < 1 || (L & (L - 1)) != 0) return -1;
  /* bit-reversal permutation */
  for (int64_t i = 1, j = 0; i < L; ++i) {
    int64_t bit = L >> 1;
    for (; j & bit; bit >>= 1) j ^= bit;
    j ^= bit;
    if (i < j) {
      double tr = z[2 * i], ti = z[2 * i + 1];
      z[2 * i] = z[2 * j];
      z[2 * i + 1] = z[2 * j + 1];
      z[2 * j] = tr;
      z[2 * j + 1] = ti;
    }
  }
  for (int64_t len = 2; len <= L; len <<= 1) {
    int64_t half = len >> 1;
    for (int64_t m = 0; m < half; ++m) {
      double ang = (double)sign * TWO_PI * (double)m / (double)len;
      double wr = cos(ang), wi = sin(ang);
      for (int64_t s = 0; s < L; s += len) {
        int64_t a = s + m, b = s + m + half;
        double br = z[2 * b] * wr - z[2 * b + 1] * wi;
        double bi = z[2 * b] * wi + z[2 * b + 1] * wr;
        z[2 * b] = z[2 * a] - br;
        z[2 * b + 1] = z[2 * a + 1] - bi;
        z[2 * a] += br;
        z[2 * a + 1] += bi;
      }
    }
  }
  return 0;
}

/*
 * Eq. 3 for n_series independent real series of length L (row-major,
 * x[s * L + n]), by oracle_fft.  X[s * (L/2+1) + k] for k = 0 .. L/2.
 */
int oracle_fft_r2c_many(int64_t L, int64_t n_series, const double* x,
                        double* X) {
  if (L < 2 || (L & (L - 1)) != 0) return -1;
  int64_t K = L / 2 + 1;
  int err = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : err)
  for (int64_t s = 0; s < n_series; ++s) {
    double* z = (double*)malloc(sizeof(double) * 2 * (size_t)L);
    if (!z) { err |= 1; continue; }
    for (int64_t n = 0; n < L; ++n) {
      z[2 * n] = x[s * L + n];
      z[2 * n + 1] = 0.0;
    }
    oracle_fft(L, z, -1);
    memcpy(X + 2 * s * K, z, sizeof(double) * 2 * (size_t)K);
    free(z);
  }
  return err ? -2 : 0;
}

/*
 * Eqs. 4 and 7: for each listed bin k_q (of an L-point transform) and trial j
 *   Y[j][q] = sum_c W(k_q, c, j) X[c][q],
 *   W = exp(+2 pi i k_q d[j][c] / L)  (phasor of Eq. 4, sign as in the header).
 * The phase in cycles, p = k d / L, is reduced to its fractional part in FP64
 * before libm cos/sin, and every phasor is evaluated directly.
 * X is [n_chan][nq] complex, Y is [n_dm][nq] complex, d is [n_dm][n_chan].
 */
void oracle_fdd_bins(int n_chan, int64_t L, int64_t nq, const int64_t* bins,
                     const double* X, int n_dm, const double* d, double* Y) {
#pragma omp parallel for collapse(2) schedule(static)
  for (int j = 0; j < n_dm; ++j) {
    for (int64_t q = 0; q < nq; ++q) {
      double k = (double)bins[q];
      double re = 0.0, im = 0.0;
      for (int c = 0; c < n_chan; ++c) {
        double p = k * d[(int64_t)j * n_chan + c] / (double)L;
        p -= floor(p);
        double wr = cos(TWO_PI * p), wi = sin(TWO_PI * p);
        double xr = X[2 * ((int64_t)c * nq + q)];
        double xi = X[2 * ((int64_t)c * nq + q) + 1];
        re += wr * xr - wi * xi;
        im += wr * xi + wi * xr;
      }
      Y[2 * ((int64_t)j * nq + q)] = re;
      Y[2 * ((int64_t)j * nq + q) + 1] = im;
    }
  }
}

/*
 * Sect. 2.3, Eqs. 8 and 9: Eq. 7 on spin-frequency-dependent DM grids, the
 * reading of the Python driver's header.  Bins below k_min follow Eq. 7 at
 * the plan's delays d_t (n_dm x n_chan).  Bin k >= k_min belongs to the group
 * (k - k_min) / G, whose highest bin k_ref supplies the phasors: over the
 * scaled grid (delays d_s, n_s x n_chan, of the DMs dm0s + j ddm)
 *   ys[j] = sum_c exp(+2 pi i k_ref d_s[j][c] / L) X[c][q],
 * which is Eq. 7 of bin k at the DMs (dm0s + j ddm) k_ref / k (Eq. 8); then
 * trial t of the plan's grid (DM_t = dm0 + t ddm) is the linear
 * interpolation of ys at x = (DM_t k / k_ref - dm0s) / ddm.
 * ys is scratch of 2 n_s doubles per thread (allocated here).
 */
/* One sum of Eq. 7 for phasor frequency kk (in bins) and one row of delays. */
static void spin_sum(double kk, const double* d_row, int n_chan, int64_t L, const double* X,
                     int64_t q, int64_t nq, double* out) {
  double sr = 0.0, si = 0.0;
  for (int c = 0; c < n_chan; ++c) {
    double ph = kk * d_row[c] / (double)L;
    ph -= floor(ph);
    const double cr = cos(TWO_PI * ph), ci = sin(TWO_PI * ph);
    const double a = X[2 * ((int64_t)c * nq + q)], b = X[2 * ((int64_t)c * nq + q) + 1];
    sr += cr * a - ci * b;
    si += cr * b + ci * a;
  }
  out[0] = sr;
  out[1] = si;
}

int oracle_fdd_bins_spin(int n_chan, int64_t L, int64_t nq, const int64_t* bins,
                         const double* X, int n_dm, const double* d_t, int n_s,
                         const double* d_s, double dm0, double ddm, double dm0s, int64_t G,
                         int64_t k_min, double* Y) {
  const int64_t K = L / 2 + 1;
  int bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
  for (int64_t q = 0; q < nq; ++q) {
    const int64_t k = bins[q];
    if (k < k_min) {
      for (int j = 0; j < n_dm; ++j)
        spin_sum((double)k, d_t + (int64_t)j * n_chan, n_chan, L, X, q, nq,
                 Y + 2 * ((int64_t)j * nq + q));
      continue;
    }
    int64_t k_ref = k_min + ((k - k_min) / G + 1) * G - 1;
    if (k_ref > K - 1) k_ref = K - 1;
    double* ys = (double*)malloc(sizeof(double) * 2 * (size_t)n_s);
    if (!ys) {
      bad = 1;
      continue;
    }
    for (int j = 0; j < n_s; ++j)
      spin_sum((double)k_ref, d_s + (int64_t)j * n_chan, n_chan, L, X, q, nq, ys + 2 * j);
    for (int t = 0; t < n_dm; ++t) {
      const double x = ((dm0 + t * ddm) * ((double)k / (double)k_ref) - dm0s) / ddm;
      int64_t m = (int64_t)floor(x);
      double delta = x - (double)m;
      if (m < 0 || m > n_s - 1) {
        bad = 1;
        m = m < 0 ? 0 : n_s - 1;
      }
      const int64_t m1 = m + 1 < n_s ? m + 1 : n_s - 1;
      Y[2 * ((int64_t)t * nq + q)] = (1.0 - delta) * ys[2 * m] + delta * ys[2 * m1];
      Y[2 * ((int64_t)t * nq + q) + 1] = (1.0 - delta) * ys[2 * m + 1] + delta * ys[2 * m1 + 1];
    }
    free(ys);
  }
  return bad ? -1 : 0;
}

/*
 * Eq. 6, the inverse transform of a half spectrum Y[0 .. L/2] of a real
 * series, written out as the direct sum over the full Hermitian spectrum:
 *   y[n] = (1/L) sum_{k=0}^{L-1} Yfull[k] exp(+2 pi i k n / L),
 *   Yfull[k] = Y[k] for k <= L/2, conj(Y[L-k]) above.
 * For even L the DC and Nyquist terms contribute only their real parts (the
 * usual real-inverse convention).  Output y[0 .. L-1].
 */
void oracle_irdft(int64_t L, const double* Y, double* y) {
  int64_t K = L / 2 + 1;
#pragma omp parallel for schedule(static)
  for (int64_t n = 0; n < L; ++n) {
    double acc = Y[0];
    for (int64_t k = 1; k < K; ++k) {
      int64_t m = (int64_t)(((__int128)k * n) % L);
      double ang = TWO_PI * (double)m / (double)L;
      double t = Y[2 * k] * cos(ang) - Y[2 * k + 1] * sin(ang);
      if ((L % 2 == 0) && k == L / 2)
        acc += Y[2 * k] * cos(ang);
      else
        acc += 2.0 * t;
    }
    y[n] = acc / (double)L;
  }
}

/*
 * The same inverse by oracle_fft on the full Hermitian spectrum (L a power of
 * two), for many series: Y is [n_series][L/2+1] complex, y is [n_series][L].
 */
int oracle_irfft_many(int64_t L, int64_t n_series, const double* Y,
                      double* y) {
  if (L < 2 || (L & (L - 1)) != 0) return -1;
  int64_t K = L / 2 + 1;
  int err = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : err)
  for (int64_t s = 0; s < n_series; ++s) {
    double* z = (double*)malloc(sizeof(double) * 2 * (size_t)L);
    if (!z) { err |= 1; continue; }
    const double* h = Y + 2 * s * K;
    for (int64_t k = 0; k < K; ++k) {
      z[2 * k] = h[2 * k];
      z[2 * k + 1] = h[2 * k + 1];
    }
    z[1] = 0.0;               /* DC: real part only */
    z[2 * (L / 2) + 1] = 0.0; /* Nyquist: real part only */
    for (int64_t k = K; k < L; ++k) {
      z[2 * k] = h[2 * (L - k)];
      z[2 * k + 1] = -h[2 * (L - k) + 1];
    }
    oracle_fft(L, z, +1);
    for (int64_t n = 0; n < L; ++n) y[s * L + n] = z[2 * n] / (double)L;
    free(z);
  }
  return err ? -2 : 0;
}

/*
 * Eq. 2, brute force: shift each channel's series by an integer number of
 * samples and sum over channels,
 *   y[j][n] = sum_c x[c][n + s[j][c]]        (advance by s samples),
 * with the index taken modulo n_t when circular != 0 and reading zero outside
 * [0, n_t) otherwise.  x is [n_chan][n_t], y is [n_dm][n_out].
 */
void oracle_tdd(int n_chan, int64_t n_t, const double* x, int n_dm,
                const int64_t* shift, int circular, int64_t n_out, double* y) {
#pragma omp parallel for schedule(static)
  for (int j = 0; j < n_dm; ++j) {
    for (int64_t n = 0; n < n_out; ++n) {
      double acc = 0.0;
      for (int c = 0; c < n_chan; ++c) {
        int64_t t = n + shift[(int64_t)j * n_chan + c];
        if (circular) {
          t %= n_t;
          if (t < 0) t += n_t;
          acc += x[(int64_t)c * n_t + t];
        } else if (t >= 0 && t < n_t) {
          acc += x[(int64_t)c * n_t + t];
        }
      }
      y[(int64_t)j * n_out + n] = acc;
    }
  }
}

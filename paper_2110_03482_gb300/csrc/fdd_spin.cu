// fdd_spin.cu -- spin-frequency-dependent DM grids on the tensor cores
// (Sect. 2.3, Eqs. 8 and 9), for one beam.
//
// Bins from k_min on are taken in groups of G consecutive bins.  All bins of
// a group use the phasors of its highest bin k_ref (Eq. 9 with f_s0 at
// k_ref): for bin k of the group they evaluate Eq. 7 at the trial DMs
// DM'_j k_ref / k (Eq. 8), DM'_j = DM'_0 + j dDM.  Sharing the phasors turns
// each group into one complex GEMM, (scaled trials x channels) times
// (channels x G bins), even for a single beam: the tensor-core kernel runs
// it with the group's bins in place of beams (phase bin k_begin + g G,
// spectra read bin-major).  Each bin is then re-sampled to the plan's trials
// by linear interpolation along the scaled trial axis at
//   x = (DM_t k / k_ref - DM'_0) / dDM.
// Bins below k_min (where a group would contract the DM grid by more than
// the plan's tolerance) follow Eq. 7 exactly on the FP32 kernels.
#include <algorithm>
#include <cmath>

#include "fdd_internal.h"

namespace fdd {
namespace {

constexpr int kTile = 32;
constexpr size_t kAlign = 256;
constexpr size_t kCap = size_t(3) << 30;  // scratch of one block of groups

size_t align_up(size_t p) { return (p + kAlign - 1) & ~(kAlign - 1); }

// gmax[g] = the largest of absmax[g G .. g G + G - 1] (bins below n_bins).
__global__ void group_max_kernel(const unsigned int* __restrict__ absmax, int n_bins, int G,
                                 unsigned int* __restrict__ gmax, int n_groups) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n_groups) return;
  unsigned int m = 0;
  for (int s = 0; s < G && g * G + s < n_bins; ++s) m = max(m, absmax[g * G + s]);
  gmax[g] = m;
}

struct ResampleArgs {
  const float2* ys;     // [group][bin of group][n_sj] scaled-grid spectra of the block
  int n_sj;             // scaled trials held, j_a .. j_a + n_sj - 1
  int j_a;
  int G;
  int k_block;          // absolute bin of the block's first bin (a group start)
  int n_bins;           // bins of the block
  int k_min, K;         // first grouped bin, bins of the transform
  double dm0, ddm, dm0s;
  int t0, n_dm;         // the plan's trials t0 .. t0 + n_dm - 1
  void* Y;              // bin k_block + i, trial t0 + r at Y + r * y_dm_stride + i
  int64_t y_dm_stride;
  int out_kind;         // 1 complex, 2 |Y|^2
  float scale;
  int real_bin;         // absolute bin whose imaginary part is zeroed, or -1
};

// 32 bins x 32 trials per tile: interpolate along trials (reads run along
// each bin's scaled trials), then store along bins through shared memory.
__global__ void __launch_bounds__(256) spin_resample_kernel(const ResampleArgs a) {
  __shared__ float2 tile[kTile][kTile + 1];
  __shared__ float r_hi[kTile], r_lo[kTile], c_hi[kTile], c_lo[kTile];
  const int ib0 = blockIdx.x * kTile;  // bin offset within the block
  const int tr0 = blockIdx.y * kTile;  // trial offset within t0 ..
  if (threadIdx.y == 0) {
    // x = t r + c with r = k / k_ref and c = (DM_0 r - DM'_0) / dDM - j_a,
    // each split into two floats (FP64 here, once per bin)
    const int i = ib0 + threadIdx.x;
    double r = 1.0, c = 0.0;
    if (i < a.n_bins) {
      const int k = a.k_block + i;
      int k_ref = a.k_min + ((k - a.k_min) / a.G + 1) * a.G - 1;
      if (k_ref > a.K - 1) k_ref = a.K - 1;
      r = static_cast<double>(k) / static_cast<double>(k_ref);
      c = (a.dm0 * r - a.dm0s) / a.ddm - a.j_a;
    }
    r_hi[threadIdx.x] = static_cast<float>(r);
    r_lo[threadIdx.x] = static_cast<float>(r - static_cast<double>(static_cast<float>(r)));
    c_hi[threadIdx.x] = static_cast<float>(c);
    c_lo[threadIdx.x] = static_cast<float>(c - static_cast<double>(static_cast<float>(c)));
  }
  __syncthreads();
#pragma unroll
  for (int ii = threadIdx.y; ii < kTile; ii += 8) {
    const int i = ib0 + ii;
    const int tr = tr0 + threadIdx.x;
    float2 y = make_float2(0.f, 0.f);
    if (i < a.n_bins && tr < a.n_dm) {
      const float t = static_cast<float>(a.t0 + tr);
      // m = floor(x), delta = x - m, with the products split so that delta
      // keeps its bits whatever the size of x
      int m = static_cast<int>(floorf(fmaf(t, r_hi[ii], c_hi[ii])));
      float delta = fmaf(t, r_hi[ii], c_hi[ii] - static_cast<float>(m)) +
                    fmaf(t, r_lo[ii], c_lo[ii]);
      if (delta < 0.f) {
        m -= 1;
        delta += 1.f;
      } else if (delta >= 1.f) {
        m += 1;
        delta -= 1.f;
      }
      m = m < 0 ? 0 : (m > a.n_sj - 1 ? a.n_sj - 1 : m);
      const int m1 = m + 1 < a.n_sj ? m + 1 : a.n_sj - 1;
      const float2* row = a.ys + static_cast<int64_t>(i) * a.n_sj;
      const float2 y0 = row[m], y1 = row[m1];
      y = make_float2((1.f - delta) * y0.x + delta * y1.x, (1.f - delta) * y0.y + delta * y1.y);
    }
    tile[ii][threadIdx.x] = y;
  }
  __syncthreads();
#pragma unroll
  for (int rr = threadIdx.y; rr < kTile; rr += 8) {
    const int tr = tr0 + rr;
    const int i = ib0 + threadIdx.x;
    if (i < a.n_bins && tr < a.n_dm) {
      const float2 v = tile[threadIdx.x][rr];
      const float re = v.x * a.scale;
      const float im = (a.k_block + i == a.real_bin) ? 0.f : v.y * a.scale;
      const int64_t o = static_cast<int64_t>(tr) * a.y_dm_stride + i;
      if (a.out_kind == 2)
        static_cast<float*>(a.Y)[o] = re * re + im * im;
      else
        static_cast<float2*>(a.Y)[o] = make_float2(re, im);
    }
  }
}

}  // namespace

void spin_geometry(int64_t K, int n_dm, double dm0, double ddm, int G, double eps,
                   SpinGeometry* out) {
  SpinGeometry sg{};
  sg.G = G;
  sg.eps = eps;
  const double km = std::ceil((G - 1) / eps);
  sg.k_min = static_cast<int>(std::min<double>(static_cast<double>(K), std::max(1.0, km)));
  sg.j_lo = dm0 == 0.0 ? 0 : static_cast<int>(std::floor(-eps * dm0 / ddm)) - 1;
  sg.n_s = n_dm - sg.j_lo;
  sg.dm0 = dm0;
  sg.ddm = ddm;
  sg.dm0s = dm0 + sg.j_lo * ddm;
  *out = sg;
}

size_t spin_scratch_bytes(const SpinGeometry& sg, int n_chan, int64_t K) {
  const size_t per_group = static_cast<size_t>(sg.G) *
                               (sizeof(float2) * (static_cast<size_t>(n_chan) + sg.n_s) +
                                sizeof(unsigned int)) +
                           sizeof(unsigned int);
  const int64_t n_g = (K - sg.k_min + sg.G - 1) / sg.G;
  int64_t kb = static_cast<int64_t>(kCap / per_group);
  if (kb < 1) kb = 1;
  if (kb > n_g) kb = n_g;
  return per_group * static_cast<size_t>(kb) + 6 * kAlign;
}

cudaError_t launch_mac_spin(const MacArgs& a, const SpinGeometry& sg, const PhaseConst* pc_spin,
                            int fp32_variant, int precision, int n_sms, void* scratch,
                            size_t scratch_bytes, cudaStream_t s) {
  if (a.n_dm <= 0 || a.n_bins <= 0) return cudaSuccess;
  if (a.n_series != 1 || a.k_begin != 0) return cudaErrorInvalidValue;
  const int K = a.n_bins;
  cudaError_t e;
  // bins below k_min: Eq. 7 exactly, FP32 kernels
  if (sg.k_min > 0) {
    MacArgs x = a;
    x.n_bins = sg.k_min < K ? sg.k_min : K;
    if ((e = launch_mac_fp32(x, fp32_variant, s)) != cudaSuccess) return e;
  }
  if (sg.k_min >= K) return cudaSuccess;
  // the scaled trials the requested ones interpolate between
  const double r_min = static_cast<double>(sg.k_min) / static_cast<double>(sg.k_min + sg.G - 1);
  const double t_a = sg.dm0 + a.j_begin * sg.ddm, t_b = sg.dm0 + (a.j_begin + a.n_dm - 1) * sg.ddm;
  const double x_min = ((t_a >= 0 ? t_a * r_min : t_a) - sg.dm0s) / sg.ddm;
  const double x_max = (t_b - sg.dm0s) / sg.ddm;
  int j_a = static_cast<int>(std::floor(x_min)) - 1;
  int j_b = static_cast<int>(std::floor(x_max)) + 1;
  j_a = j_a < 0 ? 0 : j_a;
  j_b = j_b > sg.n_s - 1 ? sg.n_s - 1 : j_b;
  const int n_sj = j_b - j_a + 1;
  const int G = sg.G;
  const int n_chan = a.n_chan;
  const int64_t n_grouped = K - sg.k_min;
  const int64_t n_g = (n_grouped + G - 1) / G;
  const size_t per_group = static_cast<size_t>(G) *
                               (sizeof(float2) * (static_cast<size_t>(n_chan) + n_sj) +
                                sizeof(unsigned int)) +
                           sizeof(unsigned int);
  if (scratch_bytes < 6 * kAlign + per_group) return cudaErrorInvalidValue;
  int64_t kb = static_cast<int64_t>((scratch_bytes - 6 * kAlign) / per_group);
  if (kb > n_g) kb = n_g;
  char* base = static_cast<char*>(scratch);
  float2* x_t = reinterpret_cast<float2*>(base);
  char* p = base + align_up(sizeof(float2) * static_cast<size_t>(kb) * G * n_chan);
  float2* ys = reinterpret_cast<float2*>(p);
  p += align_up(sizeof(float2) * static_cast<size_t>(kb) * G * n_sj);
  unsigned int* absmax = reinterpret_cast<unsigned int*>(p);
  p += align_up(sizeof(unsigned int) * static_cast<size_t>(kb) * G);
  unsigned int* gmax = reinterpret_cast<unsigned int*>(p);
  const bool f16 = precision == FDD_PREC_FP16 || precision == FDD_PREC_FP8;  // scaled data
  for (int64_t g0 = 0; g0 < n_g; g0 += kb) {
    const int nbg = static_cast<int>((n_g - g0) < kb ? (n_g - g0) : kb);
    const int64_t k_lo = sg.k_min + g0 * G;
    const int64_t k_hi = std::min<int64_t>(k_lo + static_cast<int64_t>(nbg) * G, K);
    const int nb = static_cast<int>(k_hi - k_lo);
    if (f16) {
      e = cudaMemsetAsync(absmax, 0, sizeof(unsigned int) * static_cast<size_t>(nb), s);
      if (e != cudaSuccess) return e;
    }
    BinTransposeArgs t{a.X, a.x_chan_stride, n_chan, k_lo, nb, x_t, f16 ? absmax : nullptr};
    if ((e = launch_bin_transpose(t, s)) != cudaSuccess) return e;
    if (f16) {
      group_max_kernel<<<(nbg + 127) / 128, 128, 0, s>>>(absmax, nb, G, gmax, nbg);
      note_launches(1);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    // full groups in one launch, a short last group (the top of the band) in another
    const int n_full = nb / G;
    const int rest = nb - n_full * G;
    for (int part = 0; part < 2; ++part) {
      const int ng = part == 0 ? n_full : (rest > 0 ? 1 : 0);
      if (ng == 0) continue;
      MacArgs m = a;
      m.X = x_t + static_cast<int64_t>(part == 0 ? 0 : n_full) * G * n_chan;
      m.x_bin_stride = static_cast<int64_t>(G) * n_chan;
      m.x_series_stride = n_chan;
      m.x_chan_stride = 1;
      m.pc = pc_spin;
      m.n_series = part == 0 ? G : rest;
      m.n_bins = ng;
      m.k_begin = static_cast<int>(part == 0 ? k_lo + G - 1 : K - 1);
      m.k_step = G;
      m.j_begin = j_a;
      m.n_dm = n_sj;
      m.Y = ys + static_cast<int64_t>(part == 0 ? 0 : n_full) * G * n_sj;
      m.y_bin_stride = static_cast<int64_t>(G) * n_sj;
      m.y_series_stride = n_sj;
      m.y_dm_stride = 1;
      m.out_kind = 1;
      m.scale = 1.0f;
      m.real_bin_a = -1;
      m.real_bin_b = -1;
      m.bin_absmax = reinterpret_cast<const float*>(gmax + (part == 0 ? 0 : n_full));
      if ((e = launch_mac_tc_direct(m, precision, n_sms, s)) != cudaSuccess) return e;
    }
    ResampleArgs r{};
    r.ys = ys;
    r.n_sj = n_sj;
    r.j_a = j_a;
    r.G = G;
    r.k_block = static_cast<int>(k_lo);
    r.n_bins = nb;
    r.k_min = sg.k_min;
    r.K = K;
    r.dm0 = sg.dm0;
    r.ddm = sg.ddm;
    r.dm0s = sg.dm0s;
    r.t0 = a.j_begin;
    r.n_dm = a.n_dm;
    r.Y = static_cast<char*>(a.Y) + (a.out_kind == 2 ? sizeof(float) : sizeof(float2)) * k_lo;
    r.y_dm_stride = a.y_dm_stride;
    r.out_kind = a.out_kind;
    r.scale = a.scale;
    r.real_bin = a.real_bin_b >= 0 ? a.real_bin_b : -1;
    dim3 grid((nb + kTile - 1) / kTile, (a.n_dm + kTile - 1) / kTile);
    spin_resample_kernel<<<grid, dim3(kTile, 8), 0, s>>>(r);
    note_launches(1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace fdd

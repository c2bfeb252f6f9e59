// fdd_api.cu -- the C ABI of include/fdd.h: parameter checks and plan
// geometry, the FP64 plan constants (Eq. 1 delay rates and exact fixed-point
// phase rates), device workspace, cuFFT plans for the channel transforms
// (Eq. 3) and the inverse transforms (Eq. 6), and the execute orchestration
// of Algorithm 1 (Sect. 3) on device-resident data.
#include <cufft.h>

#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <atomic>
#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <limits>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "fdd.h"
#include "fdd_internal.h"

struct fdd_plan_s {
  fdd_params p{};
  std::vector<double> dms;
  fdd_info info{};
  int device = -1;
  fdd::CoreGeometry core{};   // Eq. 1 constants and the chunking
  std::vector<double> rate;  // c_nu, samples per unit DM (Eq. 1 / t_samp)
  std::vector<fdd::PhaseConst> pc_host;
  fdd::PhaseConst* d_pc = nullptr;
  float* d_xw = nullptr;      // [n_chan][L] channel series of one chunk
  float2* d_X = nullptr;      // [n_chan][bin_pitch] their spectra
                              // (tensor-core form: [beam][n_chan][bin_pitch], every beam)
  bool tc = false;            // tensor-core form (any precision but FDD_PREC_FP32)
  float2* d_tcx = nullptr;    // tensor-core form: bin-major spectra of a block of bins
  size_t tcx_bytes = 0;
  int n_sms = 0;
  float2* d_Y = nullptr;      // [dm_batch][bin_pitch] dedispersed spectra (time output;
                              // tensor-core form: [beam][dm_batch][bin_pitch])
  float* d_yt = nullptr;      // [dm_batch][L] inverse transforms (time output)
  // spin-frequency-dependent grids (fdd_params.spin_group): the scaled grid's
  // phase table, the scratch of the groups, and the FP32 tile of the bins
  // below the first group
  bool spin_on = false;
  fdd::SpinGeometry spin{};
  fdd::PhaseConst* d_pc_spin = nullptr;
  void* d_spin_scratch = nullptr;
  size_t spin_scratch_bytes = 0;
  int spin_fp32_variant = 0;
  float2* d_xb = nullptr;     // tensor-core form: one beam's spectra [n_chan][bin_pitch]
  float2* d_Yb = nullptr;     // tensor-core form, time output: one beam's DM batch
                              // [dm_batch][bin_pitch] with bins innermost
  void* d_fftwork = nullptr;
  int* d_status = nullptr;
  cufftHandle r2c = 0, c2r = 0, c2r_tail = 0;
  bool has_r2c = false, has_c2r = false, has_c2r_tail = false;
  int c2r_tail_batch = 0;
  // streamed calls (fdd_execute_stream, fdd_execute_host): rings of two input
  // windows [n_chan x L] and two output blocks (made on the first such call),
  // the trials per spectra / power block, and for host buffers the copy
  // streams and the events that order them with the compute stream
  void* d_win[2] = {nullptr, nullptr};
  void* d_blk[2] = {nullptr, nullptr};
  size_t blk_bytes = 0;
  int block_dm = 0;
  unsigned win_next = 0, blk_next = 0;
  bool win_used[2] = {false, false}, blk_used[2] = {false, false};
  void* blk_release[2] = {nullptr, nullptr};  // a sink's event per block slot
  // Borrowed workspace (plans made by a tensor-core batch, which run one
  // after another on one stream): per-call buffers come from [arena, arena +
  // arena_bytes), bumped from its start; constants stay in the plan's own
  // allocations.
  char* arena = nullptr;
  size_t arena_bytes = 0, arena_used = 0;
  cudaStream_t h2d = nullptr, d2h = nullptr;
  cudaEvent_t win_free[2] = {}, win_full[2] = {}, blk_free[2] = {}, blk_done[2] = {};
  cudaEvent_t pipe_start = nullptr, pipe_end = nullptr;
  // fdd_tdd_execute: rounded shift tables (relative to each block of trials'
  // smallest, and those smallest) and one beam's channel-major series
  int* d_shift = nullptr;
  int* d_shift_base = nullptr;
  float* d_tdd_x = nullptr;
  int tdd_win = 0;
  size_t bytes_held = 0;
  // profiling: event pairs around stage launches (fdd_profile_enable)
  bool prof_on = false;
  std::vector<cudaEvent_t> prof_ev;  // 2 per slot
  std::vector<int> prof_stage;
  int prof_n = 0;
  int64_t prof_dropped = 0;
  long long prof_launch0 = 0;  // the library's launch count when profiling started
};

namespace {

// Last error message of this thread (a fixed buffer: reporting an error
// never allocates).
thread_local char g_err[512];

fdd_status fail(fdd_status s, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
  return s;
}

#define FDD_CUDA(call)                                                                  \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess) return fail(FDD_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

#define FDD_CUFFT(call)                                                   \
  do {                                                                    \
    cufftResult r_ = (call);                                              \
    if (r_ != CUFFT_SUCCESS) return fail(FDD_ERR_CUFFT, "%s: cufftResult %d", #call, (int)r_); \
  } while (0)

constexpr double kKdmPaper = 1.0 / 2.41e-4;  // Sect. 2.1
constexpr size_t kDefaultWorkspace = size_t(16) << 30;
constexpr size_t kMaxSmem = 227 * 1024;
constexpr int kProfSlots = 4096;

// Records an event pair around one stage launch when profiling is on.
const char* const kStageNames[FDD_STAGE_COUNT] = {"fdd unpack", "fdd r2c",     "fdd mac",
                                                   "fdd c2r",    "fdd scatter", "fdd tdd",
                                                   "fdd transpose"};

// CUDA events around a stage launch when profiling is on, and an NVTX range
// (named after the stage) always; both cost next to nothing without a tool.
class StageTimer {
 public:
  StageTimer(fdd_plan_s* P, int stage, cudaStream_t s) : P_(P), s_(s) {
    nvtxRangePushA(kStageNames[stage]);
    if (!P->prof_on) return;
    if (P->prof_n >= kProfSlots) {
      ++P->prof_dropped;
      return;
    }
    idx_ = P->prof_n++;
    P->prof_stage[idx_] = stage;
    cudaEventRecord(P->prof_ev[2 * idx_], s_);
  }
  ~StageTimer() {
    if (idx_ >= 0) cudaEventRecord(P_->prof_ev[2 * idx_ + 1], s_);
    nvtxRangePop();
  }
  StageTimer(const StageTimer&) = delete;
  StageTimer& operator=(const StageTimer&) = delete;

 private:
  fdd_plan_s* P_;
  cudaStream_t s_;
  int idx_ = -1;
};

int64_t next_pow2(int64_t n) {
  int64_t p = 2;
  while (p < n) p <<= 1;
  return p;
}

int64_t round_up(int64_t n, int64_t m) { return (n + m - 1) / m * m; }

// (x_hi + x_lo) mod 1 as a 64-bit fixed-point fraction of a cycle.
uint64_t frac_to_fixed64(double x_hi, double x_lo) {
  const double f = x_hi - std::floor(x_hi);     // exact
  const double a = std::ldexp(f, 64);           // exact scaling, in [0, 2^64)
  const double a_int = std::floor(a);
  uint64_t ua;
  if (a_int >= 18446744073709551616.0)
    ua = 0;  // cannot happen for f < 1, kept for safety
  else
    ua = static_cast<uint64_t>(a_int);
  const double rest = (a - a_int) + std::ldexp(x_lo, 64);  // small
  const long long adj = std::llround(rest);
  return ua + static_cast<uint64_t>(adj);  // wraps modulo 2^64
}

// (m * c / L) as an unevaluated double-double sum.
void scaled_product(double m, double c, double L, double* hi, double* lo) {
  const double p = m * c;
  const double pe = std::fma(m, c, -p);  // exact error of the product
  const double q = p / L;
  const double r = std::fma(-q, L, p);   // exact remainder of the division
  *hi = q;
  *lo = (r + pe) / L;
}

}  // namespace

namespace fdd {

double delay_rate(const fdd_params& p, const CoreGeometry& g, int c) {
  const double nu = p.nu_lo_mhz + p.dnu_mhz * c;
  return g.k_dm * (1.0 / (nu * nu) - 1.0 / (g.nu_ref * g.nu_ref)) / p.t_samp_s;
}

PhaseConst phase_const(double rate, double L, double dm0, double ddm) {
  double hi, lo;
  scaled_product(dm0, rate, L, &hi, &lo);
  const uint64_t u = frac_to_fixed64(hi, lo);
  scaled_product(ddm, rate, L, &hi, &lo);
  const uint64_t v = frac_to_fixed64(hi, lo);
  return PhaseConst{static_cast<uint32_t>(u), static_cast<uint32_t>(u >> 32),
                    static_cast<uint32_t>(v), static_cast<uint32_t>(v >> 32)};
}

fdd_status core_geometry(const fdd_params* p, CoreGeometry* out) {
  if (!p) return fail(FDD_ERR_INVALID_ARG, "params is NULL");
  if (p->n_chan < 1) return fail(FDD_ERR_INVALID_ARG, "n_chan must be >= 1 (got %d)", p->n_chan);
  if (!(p->t_samp_s > 0.0) || !std::isfinite(p->t_samp_s))
    return fail(FDD_ERR_INVALID_ARG, "t_samp_s must be > 0");
  if (p->n_t < 2) return fail(FDD_ERR_INVALID_ARG, "n_t must be >= 2");
  if (!p->dm_list) return fail(FDD_ERR_INVALID_ARG, "dm_list is NULL");
  if (p->n_dm < 1) return fail(FDD_ERR_INVALID_ARG, "n_dm must be >= 1");
  if (p->chunk_len < 0 || (p->chunk_len % 2) != 0)
    return fail(FDD_ERR_INVALID_ARG, "chunk_len must be 0 or a positive even length");
  if (!(p->dnu_mhz != 0.0) || !std::isfinite(p->dnu_mhz))
    return fail(FDD_ERR_INVALID_ARG, "dnu_mhz must be nonzero");
  if (!(p->k_dm >= 0.0) || !std::isfinite(p->k_dm))
    return fail(FDD_ERR_INVALID_ARG, "k_dm must be >= 0 (0 selects the default)");

  CoreGeometry g{};
  const int nc = p->n_chan;
  double nu_max = -1.0;
  for (int c = 0; c < nc; ++c) {
    const double nu = p->nu_lo_mhz + p->dnu_mhz * c;
    if (!(nu > 0.0) || !std::isfinite(nu))
      return fail(FDD_ERR_INVALID_ARG, "channel %d centre %.6g MHz is not positive", c, nu);
    nu_max = nu > nu_max ? nu : nu_max;
  }
  g.nu_ref = p->nu_ref_mhz == 0.0 ? nu_max : p->nu_ref_mhz;
  if (!(g.nu_ref >= nu_max) || !std::isfinite(g.nu_ref))
    return fail(FDD_ERR_INVALID_ARG, "nu_ref_mhz (%.9g) must be >= the highest channel centre (%.9g)",
                g.nu_ref, nu_max);
  g.k_dm = p->k_dm == 0.0 ? kKdmPaper : p->k_dm;
  g.rate_max = 0.0;
  for (int c = 0; c < nc; ++c) {
    const double r = delay_rate(*p, g, c);
    g.rate_max = r > g.rate_max ? r : g.rate_max;
  }

  double dm_max = 0.0;
  for (int j = 0; j < p->n_dm; ++j) {
    const double dm = p->dm_list[j];
    if (!(dm >= 0.0) || !std::isfinite(dm))
      return fail(FDD_ERR_INVALID_ARG, "dm_list[%d] = %g must be finite and >= 0", j, dm);
    dm_max = dm > dm_max ? dm : dm_max;
  }
  // Uniform grid check: every entry within 4 ulp of dm0 + j ddm.
  g.dm0 = p->dm_list[0];
  g.ddm = p->n_dm > 1 ? (p->dm_list[p->n_dm - 1] - g.dm0) / (p->n_dm - 1) : 0.0;
  const double tol = 4.0 * std::ldexp(std::numeric_limits<double>::epsilon(),
                                      std::ilogb(dm_max > 1.0 ? dm_max : 1.0));
  // (A non-uniform list makes a valid plan: the time-domain path takes any
  // list; the Fourier-domain calls refuse it, see need_uniform_grid.)
  g.uniform = 1;
  for (int j = 0; j < p->n_dm && g.uniform; ++j)
    if (std::fabs(p->dm_list[j] - (g.dm0 + j * g.ddm)) > tol) g.uniform = 0;

  const double max_delay = dm_max * g.rate_max;  // both factors are >= 0
  if (max_delay > 4.0e18) return fail(FDD_ERR_INVALID_ARG, "delays overflow");
  g.d_max = static_cast<int64_t>(std::ceil(max_delay));

  int64_t L, hop, n_chunks, out_len, valid_len;
  if (p->chunk_len == 0) {
    L = next_pow2(p->n_t);
    hop = p->n_t;
    n_chunks = 1;
    out_len = p->n_t;
    valid_len = p->n_t > g.d_max ? p->n_t - g.d_max : 0;
  } else {
    L = p->chunk_len;
    hop = L - g.d_max;
    if (hop <= 0)
      return fail(FDD_ERR_INVALID_ARG,
                  "chunk_len %lld does not exceed the largest delay (%lld samples)",
                  (long long)L, (long long)g.d_max);
    out_len = p->n_t - g.d_max;
    if (out_len <= 0)
      return fail(FDD_ERR_INVALID_ARG, "n_t %lld does not exceed the largest delay %lld",
                  (long long)p->n_t, (long long)g.d_max);
    n_chunks = (out_len + hop - 1) / hop;
    valid_len = out_len;
  }
  // Down-sampling by a shorter inverse transform (Sect. 2.2, last paragraph):
  // the hop becomes a multiple of f and the output counts samples of f.
  const int f = p->downsample > 1 ? p->downsample : 1;
  if (p->downsample < 0 || (f & (f - 1)) != 0)
    return fail(FDD_ERR_INVALID_ARG, "downsample must be 0, 1 or a power of two");
  if (f > 1) {
    if (p->output != FDD_OUT_TIME)
      return fail(FDD_ERR_INVALID_ARG, "downsample applies to FDD_OUT_TIME output");
    if (L % (2 * static_cast<int64_t>(f)) != 0)
      return fail(FDD_ERR_INVALID_ARG, "transform length %lld is not divisible by 2 x %d",
                  (long long)L, f);
    if (p->chunk_len == 0) {
      out_len = (out_len + f - 1) / f;
      valid_len = (valid_len + f - 1) / f;
      hop = out_len * f;
    } else {
      hop = hop / f * f;
      if (hop <= 0)
        return fail(FDD_ERR_INVALID_ARG, "chunk_len %lld leaves no hop at downsample %d",
                    (long long)L, f);
      n_chunks = (out_len + hop - 1) / hop;
      out_len = (out_len + f - 1) / f;
      valid_len = out_len;
    }
  }
  const int64_t n_bins = L / 2 + 1;
  if (L > (int64_t(1) << 30)) return fail(FDD_ERR_UNSUPPORTED, "transform length above 2^30");
  // The kernels form k * j in 32-bit integers.
  if (static_cast<double>(n_bins - 1) * static_cast<double>(p->n_dm - 1) >= 4294967296.0)
    return fail(FDD_ERR_UNSUPPORTED, "(n_bins-1)*(n_dm-1) must be below 2^32");
  g.L = L;
  g.n_bins = n_bins;
  g.hop = hop;
  g.n_chunks = n_chunks;
  g.out_len = out_len;
  g.valid_len = valid_len;
  g.downsample = f;
  *out = g;
  return FDD_OK;
}

}  // namespace fdd

namespace {

// Device bytes a spin-frequency plan adds: the scaled grid's phase table and
// the scratch of its blocks of groups.
size_t spin_plan_bytes(const fdd_params* p, const fdd::CoreGeometry& cg, int64_t n_bins) {
  fdd::SpinGeometry sg;
  fdd::spin_geometry(n_bins, p->n_dm, cg.dm0, cg.ddm, p->spin_group,
                     p->spin_tol > 0.0 ? p->spin_tol : 0.01, &sg);
  return sizeof(fdd::PhaseConst) * p->n_chan + fdd::spin_scratch_bytes(sg, p->n_chan, n_bins);
}

fdd_status compute_plan(const fdd_params* p, fdd_info* g, fdd::CoreGeometry* core_out) {
  if (!p) return fail(FDD_ERR_INVALID_ARG, "params is NULL");
  if (!g) return fail(FDD_ERR_INVALID_ARG, "info is NULL");
  if (p->n_beams < 1) return fail(FDD_ERR_INVALID_ARG, "n_beams must be >= 1");
  if (p->in_dtype != FDD_IN_U8 && p->in_dtype != FDD_IN_F32)
    return fail(FDD_ERR_INVALID_ARG, "in_dtype %d unknown", p->in_dtype);
  if (p->in_layout != FDD_LAYOUT_TIME_MAJOR && p->in_layout != FDD_LAYOUT_CHAN_MAJOR)
    return fail(FDD_ERR_INVALID_ARG, "in_layout %d unknown", p->in_layout);
  if (p->output != FDD_OUT_TIME && p->output != FDD_OUT_SPECTRA && p->output != FDD_OUT_POWER)
    return fail(FDD_ERR_INVALID_ARG, "output %d unknown", p->output);
  if (p->precision != FDD_PREC_FP32 && p->precision != FDD_PREC_BF16_HILO &&
      p->precision != FDD_PREC_BF16 && p->precision != FDD_PREC_FP16 &&
      p->precision != FDD_PREC_FP8)
    return fail(FDD_ERR_INVALID_ARG, "precision %d unknown", p->precision);
  if (p->mac_variant < 0 || p->mac_variant > FDD_MAC_VARIANTS)
    return fail(FDD_ERR_INVALID_ARG, "mac_variant %d outside [0, %d]", p->mac_variant,
                FDD_MAC_VARIANTS);
  if (p->spin_group != 0) {
    if (p->spin_group != 16 && p->spin_group != 32)
      return fail(FDD_ERR_INVALID_ARG, "spin_group must be 0, 16 or 32");
    if (p->precision == FDD_PREC_FP32 || p->n_beams != 1)
      return fail(FDD_ERR_UNSUPPORTED,
                  "spin-frequency grids run on the tensor-core form for one beam");
    if (!(p->spin_tol >= 0.0) || !(p->spin_tol < 1.0))
      return fail(FDD_ERR_INVALID_ARG, "spin_tol must be in [0, 1) (0 selects 0.01)");
  }
  fdd::CoreGeometry cg;
  fdd_status st = fdd::core_geometry(p, &cg);
  if (st != FDD_OK) return st;
  const int nc = p->n_chan;
  const int64_t L = cg.L, n_bins = cg.n_bins, n_chunks = cg.n_chunks, out_len = cg.out_len;
  const int f = cg.downsample;

  std::memset(g, 0, sizeof *g);
  g->fft_len = L;
  g->n_bins = n_bins;
  g->bin_pitch = round_up(n_bins, 64);
  g->n_chunks = n_chunks;
  g->hop = cg.hop;
  g->d_max = cg.d_max;
  g->out_len = out_len;
  g->valid_len = cg.valid_len;
  g->downsample = f;
  g->in_elems = static_cast<int64_t>(p->n_beams) * p->n_t * nc;
  if (p->output == FDD_OUT_TIME) {
    g->out_elems = static_cast<int64_t>(p->n_beams) * p->n_dm * out_len;
    g->out_bytes = g->out_elems * 4;
  } else {
    g->out_elems = static_cast<int64_t>(p->n_beams) * n_chunks * p->n_dm * n_bins;
    g->out_bytes = g->out_elems * (p->output == FDD_OUT_SPECTRA ? 8 : 4);
  }
  g->dm0 = cg.dm0;
  g->ddm = cg.ddm;
  g->dm_uniform = cg.uniform;
  if (p->spin_group != 0) {
    if (p->n_dm < 2 || !(cg.ddm > 0.0))
      return fail(FDD_ERR_UNSUPPORTED, "spin-frequency grids need two or more increasing trials");
    fdd::SpinGeometry sg;
    fdd::spin_geometry(n_bins, p->n_dm, cg.dm0, cg.ddm, p->spin_group,
                       p->spin_tol > 0.0 ? p->spin_tol : 0.01, &sg);
    if (static_cast<double>(n_bins - 1) * static_cast<double>(sg.n_s - 1) >= 4294967296.0)
      return fail(FDD_ERR_UNSUPPORTED, "(n_bins-1)*(scaled trials-1) must be below 2^32");
    g->spin_group = sg.G;
    g->spin_k_min = sg.k_min;
    g->spin_j_lo = sg.j_lo;
    g->spin_n_s = sg.n_s;
  }
  const bool tc = p->precision != FDD_PREC_FP32;
  g->mac_variant = tc ? FDD_MAC_TC : (p->mac_variant ? p->mac_variant - 1
                                                     : fdd::mac_variant_for(p->n_dm, nc));
  // tensor cores: the CTA-pair form where its passes are full enough.  A
  // pass of either form costs a fixed part (the phasor rows P, evaluated per
  // pass and CTA) plus a part per a (Z and the MMAs); measured on 32 beams x
  // 1024 channels, in whole-GPU time per bin, the pair's pass (2048 trials)
  // costs 375 ns + 12.2 ns per a of 256 trials, the one-CTA pass (1024
  // trials) 197 ns + 8.9 ns per a of 128: the
  // pair wins on calls whose last pair pass is more than half full (or
  // full).  A plan keeps one form, so its streamed and whole calls agree.
  const int64_t pass2 = tc ? fdd::mac_tc_trials_per_pass(p->n_beams, true) : 0;
  auto pair_wins = [&](int64_t n) {
    const int64_t r = n % pass2;
    return n > pass2 / 2 && (r == 0 || r > pass2 / 2);
  };
  bool pair = tc && p->spin_group == 0 && pair_wins(p->n_dm);
  if (!tc && fdd::mac_smem_bytes(g->mac_variant, nc) > kMaxSmem)
    return fail(FDD_ERR_UNSUPPORTED, "n_chan %d needs more shared memory than a CTA has", nc);

  const size_t spectra_sets = tc ? static_cast<size_t>(p->n_beams) : 1;
  const size_t fixed = sizeof(fdd::PhaseConst) * nc + sizeof(float) * size_t(nc) * L +
                       sizeof(float2) * size_t(nc) * g->bin_pitch * (spectra_sets + (tc ? 1 : 0)) +
                       256 +
                       (tc ? fdd::mac_tc_scratch_bytes(p->n_beams, nc, p->n_dm, n_bins) : 0) +
                       (p->spin_group ? spin_plan_bytes(p, cg, n_bins) : 0);
  const size_t limit = p->workspace_limit ? p->workspace_limit : kDefaultWorkspace;
  int64_t batch = p->n_dm;
  size_t per_dm = 0;
  if (p->output == FDD_OUT_TIME) {
    per_dm = sizeof(float2) * g->bin_pitch * (spectra_sets + (tc ? 1 : 0)) + sizeof(float) * (L / f);
    if (fixed + per_dm > limit)
      return fail(FDD_ERR_INVALID_ARG, "workspace_limit %zu is below the minimum %zu", limit,
                  fixed + per_dm);
    const int64_t fit = static_cast<int64_t>((limit - fixed) / per_dm);
    if (fit < batch) {
      // whole kernel passes or trial blocks, else whatever fits; the pair
      // form only in batches of whole passes (partial ones lose to the
      // one-CTA form's whole passes)
      if (pair && fit < pass2) pair = false;
      const int64_t blk = tc ? fdd::mac_tc_trials_per_pass(p->n_beams, pair)
                             : fdd::mac_variant_trials_per_block(g->mac_variant);
      batch = fit >= blk ? fit / blk * blk : fit;
    }
    if (batch > 65535) batch = 65535 / 64 * 64;
  } else if (pair) {
    // streamed blocks are whole passes: the pair's only where two blocks of
    // one pass stay within half the limit
    const size_t per_trial = (p->output == FDD_OUT_SPECTRA ? 8 : 4) * spectra_sets *
                             static_cast<size_t>(n_bins);
    if (per_trial * static_cast<size_t>(pass2) > limit / 4) pair = false;
  }
  if (tc) g->mac_variant = pair ? FDD_MAC_TC_PAIR : FDD_MAC_TC;
  g->dm_batch = static_cast<int32_t>(batch);
  g->workspace_bytes = static_cast<int64_t>(fixed + per_dm * batch);
  // Streamed calls: output blocks of one beam's DM batch (time), or of
  // block_dm trials of every spectra set (spectra, power; whole passes of the
  // kernel tile, up to 4 GiB or a quarter of workspace_limit, at least one
  // pass); two input windows of one beam's chunk.
  const size_t in_esz = p->in_dtype == FDD_IN_U8 ? 1 : 4;
  size_t blk_bytes;
  if (p->output == FDD_OUT_TIME) {
    g->block_dm = g->dm_batch;
    blk_bytes = sizeof(float) * static_cast<size_t>(batch) * (cg.hop / f);
  } else {
    const size_t per_trial = (p->output == FDD_OUT_SPECTRA ? 8 : 4) * spectra_sets *
                             static_cast<size_t>(n_bins);
    const int64_t pass = tc ? fdd::mac_tc_trials_per_pass(p->n_beams, pair)
                            : fdd::mac_variant_trials_per_block(g->mac_variant);
    const size_t cap = std::min<size_t>(size_t(4) << 30, limit / 4);
    int64_t bd = static_cast<int64_t>(cap / per_trial) / pass * pass;
    if (bd < pass) bd = pass;
    if (bd > p->n_dm) bd = p->n_dm;
    g->block_dm = static_cast<int32_t>(bd);
    blk_bytes = per_trial * static_cast<size_t>(bd);
  }
  g->stream_bytes = static_cast<int64_t>(2 * blk_bytes + 2 * in_esz * size_t(nc) * L);
  if (core_out) *core_out = cg;
  return FDD_OK;
}

void release(fdd_plan_s* P) {
  if (!P) return;
  if (P->has_r2c) cufftDestroy(P->r2c);
  if (P->has_c2r) cufftDestroy(P->c2r);
  if (P->has_c2r_tail) cufftDestroy(P->c2r_tail);
  void* ptrs[] = {P->d_pc, P->d_xw, P->d_X, P->d_Y, P->d_yt, P->d_xb, P->d_Yb, P->d_fftwork,
                  P->d_pc_spin, P->d_spin_scratch, P->d_status,
                  P->d_win[0], P->d_win[1], P->d_blk[0], P->d_blk[1], P->d_tcx, P->d_shift,
                  P->d_shift_base, P->d_tdd_x};
  for (void* q : ptrs)
    if (q && !(P->arena && static_cast<char*>(q) >= P->arena &&
               static_cast<char*>(q) < P->arena + P->arena_bytes))
      cudaFree(q);
  for (cudaEvent_t e : P->prof_ev)
    if (e) cudaEventDestroy(e);
  cudaEvent_t pipe[] = {P->win_free[0], P->win_free[1], P->win_full[0], P->win_full[1],
                        P->blk_free[0], P->blk_free[1], P->blk_done[0], P->blk_done[1],
                        P->pipe_start, P->pipe_end};
  for (cudaEvent_t e : pipe)
    if (e) cudaEventDestroy(e);
  if (P->h2d) cudaStreamDestroy(P->h2d);
  if (P->d2h) cudaStreamDestroy(P->d2h);
  delete P;
}

// The Fourier-domain kernels form the phase as k u + k j v (a uniform grid).
fdd_status need_uniform_grid(const fdd_plan_s* P) {
  if (P->info.dm_uniform) return FDD_OK;
  return fail(FDD_ERR_UNSUPPORTED,
              "the Fourier-domain kernels need a uniform DM grid (fdd_tdd_execute takes any list)");
}

fdd_status dev_alloc(fdd_plan_s* P, void** ptr, size_t bytes) {
  if (fdd::injected_alloc_failure()) {
    *ptr = nullptr;
    return fail(FDD_ERR_ALLOC, "injected allocation failure");
  }
  cudaError_t e = cudaMalloc(ptr, bytes);
  if (e != cudaSuccess) {
    *ptr = nullptr;
    cudaGetLastError();
    return fail(FDD_ERR_ALLOC, "cudaMalloc(%zu bytes): %s", bytes, cudaGetErrorString(e));
  }
  P->bytes_held += bytes;
  return FDD_OK;
}

// A per-call buffer: from the borrowed workspace when the plan has one.
fdd_status ws_alloc(fdd_plan_s* P, void** ptr, size_t bytes) {
  if (!P->arena) return dev_alloc(P, ptr, bytes);
  const size_t at = (P->arena_used + 255) / 256 * 256;
  if (at + bytes > P->arena_bytes) {
    *ptr = nullptr;
    return fail(FDD_ERR_ALLOC, "borrowed workspace of %zu bytes too small (%zu more needed)",
                P->arena_bytes, at + bytes - P->arena_bytes);
  }
  *ptr = P->arena + at;
  P->arena_used = at + bytes;
  return FDD_OK;
}

fdd_status check_device(const fdd_plan_s* P) {
  int dev = -1;
  FDD_CUDA(cudaGetDevice(&dev));
  if (dev != P->device)
    return fail(FDD_ERR_INVALID_ARG, "plan was made on device %d, current device is %d", P->device,
                dev);
  return FDD_OK;
}

// Where a run's input comes from and where its output goes (the copies of
// Algorithm 1).  fdd_execute: the whole input and output on the device.
// Otherwise input windows and output blocks pass through plan-owned rings of
// two slots each: filled by the caller's source and handed to its sink in
// stream order (fdd_execute_stream), or copied from / to host buffers on the
// plan's two copy streams (fdd_execute_host), so no device buffer is sized by
// the whole input or output.
struct Io {
  const void* d_in = nullptr;
  void* d_out = nullptr;
  fdd_source_fn source = nullptr;
  void* source_user = nullptr;
  fdd_sink_fn sink = nullptr;
  void* sink_user = nullptr;
  const char* h_in = nullptr;
  char* h_out = nullptr;
  bool host() const { return h_in != nullptr; }
  int dm_first = 0, n_dm = 0;  // the trials of this run
};

// Where the unpack of (beam b, chunk c) reads: into *ua.  Streamed input
// fills a window slot with samples [c hop, c hop + L) of beam b first.
fdd_status input_for(fdd_plan_s* P, const Io& io, int b, int64_t c, cudaStream_t s,
                     fdd::UnpackArgs* ua, int* slot_out) {
  const fdd_params& p = P->p;
  const fdd_info& g = P->info;
  const size_t esz = p.in_dtype == FDD_IN_U8 ? 1 : 4;
  *slot_out = -1;
  *ua = fdd::UnpackArgs{nullptr, p.in_dtype, p.in_layout, p.n_chan, p.n_t, c * g.hop,
                        g.fft_len, P->d_xw, g.fft_len};
  if (io.d_in) {
    ua->in = static_cast<const char*>(io.d_in) + esz * static_cast<size_t>(p.n_t) * p.n_chan * b;
    return FDD_OK;
  }
  const int w = static_cast<int>(P->win_next++ & 1);
  const int64_t t0 = c * g.hop;
  const int64_t n = std::min<int64_t>(g.fft_len, p.n_t - t0);
  void* dst = P->d_win[w];
  if (io.host()) {
    if (P->win_used[w]) FDD_CUDA(cudaStreamWaitEvent(P->h2d, P->win_free[w], 0));
    const char* src = io.h_in + esz * static_cast<size_t>(p.n_t) * p.n_chan * b;
    if (p.in_layout == FDD_LAYOUT_TIME_MAJOR) {
      FDD_CUDA(cudaMemcpyAsync(dst, src + esz * static_cast<size_t>(t0) * p.n_chan,
                               esz * static_cast<size_t>(n) * p.n_chan, cudaMemcpyHostToDevice,
                               P->h2d));
    } else {
      FDD_CUDA(cudaMemcpy2DAsync(dst, esz * static_cast<size_t>(n), src + esz * t0,
                                 esz * static_cast<size_t>(p.n_t), esz * static_cast<size_t>(n),
                                 p.n_chan, cudaMemcpyHostToDevice, P->h2d));
    }
    FDD_CUDA(cudaEventRecord(P->win_full[w], P->h2d));
    FDD_CUDA(cudaStreamWaitEvent(s, P->win_full[w], 0));
  } else {
    void* ready = P->win_used[w] ? static_cast<void*>(P->win_free[w]) : nullptr;
    const fdd_status st =
        io.source(io.source_user, b, t0, n, dst, ready, reinterpret_cast<fdd_stream_t>(s));
    if (st != FDD_OK) return fail(st, "the input source failed for beam %d, samples %lld..%lld", b,
                                  (long long)t0, (long long)(t0 + n));
  }
  ua->in = dst;
  ua->n_t = n;
  ua->t_begin = 0;
  *slot_out = w;
  return FDD_OK;
}

// After the unpack that read window slot w (streamed input): the slot may be
// refilled once the unpack is done.
fdd_status input_done(fdd_plan_s* P, const Io& io, int w, cudaStream_t s) {
  (void)io;
  if (w < 0) return FDD_OK;
  FDD_CUDA(cudaEventRecord(P->win_free[w], s));
  P->win_used[w] = true;
  return FDD_OK;
}

// An output block slot for the next block (streamed output); waits until the
// host copy of its previous block is done.
fdd_status block_slot(fdd_plan_s* P, const Io& io, cudaStream_t s, int* slot) {
  const int k = static_cast<int>(P->blk_next++ & 1);
  if (io.host() && P->blk_used[k]) FDD_CUDA(cudaStreamWaitEvent(s, P->blk_free[k], 0));
  if (!io.host() && P->blk_release[k]) {  // the sink's reads of the slot's last block
    FDD_CUDA(cudaStreamWaitEvent(s, static_cast<cudaEvent_t>(P->blk_release[k]), 0));
    P->blk_release[k] = nullptr;
  }
  *slot = k;
  return FDD_OK;
}

// Hand a finished block to the sink, or copy it to the host output.
fdd_status deliver(fdd_plan_s* P, const Io& io, int k, fdd_block& blk, cudaStream_t s) {
  const fdd_params& p = P->p;
  const fdd_info& g = P->info;
  if (!io.host()) {
    blk.release_event = nullptr;
    const fdd_status st = io.sink(io.sink_user, &blk, reinterpret_cast<fdd_stream_t>(s));
    if (st != FDD_OK) return fail(st, "the output sink failed (chunk %lld, trials %d..%d)",
                                  (long long)blk.chunk, blk.dm_first, blk.dm_first + blk.n_dm);
    P->blk_release[k] = blk.release_event;
    return FDD_OK;
  }
  FDD_CUDA(cudaEventRecord(P->blk_done[k], s));
  FDD_CUDA(cudaStreamWaitEvent(P->d2h, P->blk_done[k], 0));
  const int rel = blk.dm_first - io.dm_first;  // row of the first trial in the output
  if (p.output == FDD_OUT_TIME) {
    // rows [beam][trial] of out_len samples; the block holds row_len of them
    const size_t dst_pitch = sizeof(float) * static_cast<size_t>(g.out_len);
    for (int q = 0; q < blk.n_beams; ++q) {
      char* dst = io.h_out + sizeof(float) * ((static_cast<size_t>(blk.beam_first + q) * io.n_dm + rel) *
                                                  g.out_len + blk.out_offset);
      const char* src = static_cast<const char*>(blk.d_data) +
                        sizeof(float) * static_cast<size_t>(q) * blk.n_dm * blk.row_pitch;
      FDD_CUDA(cudaMemcpy2DAsync(dst, dst_pitch, src, sizeof(float) * blk.row_pitch,
                                 sizeof(float) * blk.row_len, blk.n_dm, cudaMemcpyDeviceToHost,
                                 P->d2h));
    }
  } else {
    const size_t esz = p.output == FDD_OUT_SPECTRA ? 8 : 4;
    const size_t rows_beam = static_cast<size_t>(g.n_chunks) * io.n_dm;  // rows per beam
    char* dst = io.h_out + esz * ((static_cast<size_t>(blk.beam_first) * rows_beam +
                                   static_cast<size_t>(blk.chunk) * io.n_dm + rel) *
                                  g.n_bins);
    FDD_CUDA(cudaMemcpy2DAsync(dst, esz * rows_beam * g.n_bins, blk.d_data,
                               esz * static_cast<size_t>(blk.n_dm) * g.n_bins,
                               esz * static_cast<size_t>(blk.n_dm) * g.n_bins, blk.n_beams,
                               cudaMemcpyDeviceToHost, P->d2h));
  }
  FDD_CUDA(cudaEventRecord(P->blk_free[k], P->d2h));
  P->blk_used[k] = true;
  return FDD_OK;
}

// Unpack + forward transforms of (beam b, chunk c) into spectra X (Eq. 3).
fdd_status transform(fdd_plan_s* P, const Io& io, int b, int64_t c, float2* X, cudaStream_t s) {
  fdd::UnpackArgs ua;
  int w;
  fdd_status st = input_for(P, io, b, c, s, &ua, &w);
  if (st != FDD_OK) return st;
  {
    StageTimer t(P, FDD_STAGE_UNPACK, s);
    FDD_CUDA(fdd::launch_unpack(ua, s));
  }
  if ((st = input_done(P, io, w, s)) != FDD_OK) return st;
  StageTimer t(P, FDD_STAGE_R2C, s);
  FDD_CUFFT(cufftExecR2C(P->r2c, P->d_xw, reinterpret_cast<cufftComplex*>(X)));
  return FDD_OK;
}

// Whole rows: one chunk whose kept samples are the whole inverse transform
// (an unchunked series whose length is the transform length).  Then the
// phase-rotate-and-sum applies the 1/L scaling (exact for a power-of-two L)
// and the inverse transforms write the output rows directly: no scatter.
bool whole_rows(const fdd_plan_s* P) {
  const fdd_info& g = P->info;
  return g.n_chunks == 1 && g.out_len == g.fft_len / g.downsample;
}

// The inverse transforms (Eq. 6) of DM batch [j0, j0 + nb) of beam b, chunk c,
// from bins-innermost spectra Y, then the 1/L scaling and valid-sample
// placement (the discard rule of Sect. 2.2): into the output rows, or into a
// block handed on.
fdd_status inverse_and_place(fdd_plan_s* P, const Io& io, int b, int64_t c, int j0, int nb,
                             float2* Y, cudaStream_t s) {
  const fdd_info& g = P->info;
  const int64_t Ls = g.fft_len / g.downsample, hop_o = g.hop / g.downsample;
  const int64_t keep = (g.out_len - c * hop_o) < hop_o ? (g.out_len - c * hop_o) : hop_o;
  const bool tail = P->has_c2r_tail && nb == P->c2r_tail_batch;
  cufftHandle h = tail ? P->c2r_tail : P->c2r;
  const bool direct = whole_rows(P);
  int k = -1;
  float* dst;
  int64_t dst_stride;
  if (io.d_out) {
    dst = static_cast<float*>(io.d_out) +
          (static_cast<int64_t>(b) * io.n_dm + (j0 - io.dm_first)) * g.out_len + c * hop_o;
    dst_stride = g.out_len;
  } else {
    fdd_status st = block_slot(P, io, s, &k);
    if (st != FDD_OK) return st;
    dst = static_cast<float*>(P->d_blk[k]);
    dst_stride = hop_o;
  }
  // (direct: rows of Ls samples at stride Ls, the C2R plan's own output
  // layout; a batch of fewer trials than the plan's writes nb rows only when
  // it is the tail plan, so a short batch goes through d_yt)
  const bool plan_rows = tail || nb == g.dm_batch;
  if (direct && plan_rows) {
    StageTimer t(P, FDD_STAGE_C2R, s);
    FDD_CUFFT(cufftExecC2R(h, reinterpret_cast<cufftComplex*>(Y), dst));
  } else {
    {
      StageTimer t(P, FDD_STAGE_C2R, s);
      FDD_CUFFT(cufftExecC2R(h, reinterpret_cast<cufftComplex*>(Y), P->d_yt));
    }
    fdd::ScatterArgs sa{};
    sa.src = P->d_yt;
    sa.src_stride = Ls;
    sa.n_dm = nb;
    sa.n_keep = keep;
    sa.scale = direct ? 1.0f : static_cast<float>(1.0 / static_cast<double>(g.fft_len));
    sa.dst = dst;
    sa.dst_stride = dst_stride;
    StageTimer t(P, FDD_STAGE_SCATTER, s);
    FDD_CUDA(fdd::launch_scatter(sa, s));
  }
  if (k < 0) return FDD_OK;
  fdd_block blk{b, 1, c, j0, nb, P->d_blk[k], keep, hop_o, c * hop_o, nullptr};
  return deliver(P, io, k, blk, s);
}

fdd_status run_tc(fdd_plan_s* P, const Io& io, cudaStream_t s);

fdd_status run(fdd_plan_s* P, const Io& io, cudaStream_t s) {
  const fdd_params& p = P->p;
  const fdd_info& g = P->info;
  FDD_CUFFT(cufftSetStream(P->r2c, s));
  if (P->has_c2r) FDD_CUFFT(cufftSetStream(P->c2r, s));
  if (P->has_c2r_tail) FDD_CUFFT(cufftSetStream(P->c2r_tail, s));
  if (P->tc) return run_tc(P, io, s);
  fdd_status st;
  const int dm_end = io.dm_first + io.n_dm;
  for (int b = 0; b < p.n_beams; ++b) {
    for (int64_t c = 0; c < g.n_chunks; ++c) {
      if ((st = transform(P, io, b, c, P->d_X, s)) != FDD_OK) return st;
      fdd::MacArgs m{};
      m.X = P->d_X;
      m.x_series_stride = 0;
      m.x_chan_stride = g.bin_pitch;
      m.pc = P->d_pc;
      m.n_chan = p.n_chan;
      m.n_bins = static_cast<int>(g.n_bins);
      m.n_series = 1;
      m.scale = 1.0f;
      m.status = P->d_status;
      if (p.output == FDD_OUT_TIME) {
        // (shortened inverse: only the bins up to Nyquist of length L / f)
        const int64_t Ls = g.fft_len / g.downsample;
        m.n_bins = static_cast<int>(Ls / 2 + 1);
        for (int j0 = io.dm_first; j0 < dm_end; j0 += g.dm_batch) {
          const int nb = (dm_end - j0) < g.dm_batch ? (dm_end - j0) : g.dm_batch;
          m.j_begin = j0;
          m.n_dm = nb;
          m.Y = P->d_Y;
          m.y_series_stride = 0;
          m.y_dm_stride = g.bin_pitch;
          m.out_kind = 1;
          m.real_bin_a = 0;                           // DC and Nyquist of a real
          m.real_bin_b = static_cast<int>(Ls / 2);    // series: real parts only
          m.scale = whole_rows(P) ? static_cast<float>(1.0 / static_cast<double>(g.fft_len)) : 1.0f;
          {
            StageTimer t(P, FDD_STAGE_MAC, s);
            FDD_CUDA(fdd::launch_mac_fp32(m, g.mac_variant, s));
          }
          if ((st = inverse_and_place(P, io, b, c, j0, nb, P->d_Y, s)) != FDD_OK) return st;
        }
      } else {
        m.y_series_stride = 0;
        m.y_dm_stride = g.n_bins;
        m.real_bin_a = -1;
        m.real_bin_b = -1;
        m.out_kind = p.output == FDD_OUT_SPECTRA ? 1 : 2;
        const size_t esz = p.output == FDD_OUT_SPECTRA ? 8 : 4;
        // the whole trial range into the output, or blocks of block_dm trials
        const int step = io.d_out ? io.n_dm : P->block_dm;
        for (int j0 = io.dm_first; j0 < dm_end; j0 += step) {
          const int nb = (dm_end - j0) < step ? (dm_end - j0) : step;
          m.j_begin = j0;
          m.n_dm = nb;
          int k = -1;
          if (io.d_out) {
            const int64_t row0 = (static_cast<int64_t>(b) * g.n_chunks + c) * io.n_dm;
            m.Y = static_cast<char*>(io.d_out) + esz * row0 * g.n_bins;
          } else {
            if ((st = block_slot(P, io, s, &k)) != FDD_OK) return st;
            m.Y = P->d_blk[k];
          }
          {
            StageTimer t(P, FDD_STAGE_MAC, s);
            FDD_CUDA(fdd::launch_mac_fp32(m, g.mac_variant, s));
          }
          if (k >= 0) {
            fdd_block blk{b, 1, c, j0, nb, P->d_blk[k], g.n_bins, g.n_bins, 0, nullptr};
            if ((st = deliver(P, io, k, blk, s)) != FDD_OK) return st;
          }
        }
      }
    }
  }
  return FDD_OK;
}

// Spin-frequency-dependent grids (one beam, tensor cores): per chunk the
// beam's spectra stay bins innermost (d_xb); launch_mac_spin writes the
// dedispersed spectra bins innermost too, so the inverse transforms read
// them directly (time output) or they go straight to the output.
fdd_status run_spin(fdd_plan_s* P, const Io& io, cudaStream_t s) {
  fdd_status st;
  const fdd_params& p = P->p;
  const fdd_info& g = P->info;
  const int dm_end = io.dm_first + io.n_dm;
  for (int64_t c = 0; c < g.n_chunks; ++c) {
    if ((st = transform(P, io, 0, c, P->d_xb, s)) != FDD_OK) return st;
    fdd::MacArgs m{};
    m.X = P->d_xb;
    m.x_chan_stride = g.bin_pitch;
    m.x_series_stride = static_cast<int64_t>(p.n_chan) * g.bin_pitch;
    m.pc = P->d_pc;
    m.n_chan = p.n_chan;
    m.n_series = 1;
    m.status = P->d_status;
    m.scale = 1.0f;
    if (p.output == FDD_OUT_TIME) {
      const int64_t Ls = g.fft_len / g.downsample;
      m.n_bins = static_cast<int>(Ls / 2 + 1);
      m.out_kind = 1;
      m.real_bin_a = 0;
      m.real_bin_b = static_cast<int>(Ls / 2);
      m.scale = whole_rows(P) ? static_cast<float>(1.0 / static_cast<double>(g.fft_len)) : 1.0f;
      for (int j0 = io.dm_first; j0 < dm_end; j0 += g.dm_batch) {
        const int nb = (dm_end - j0) < g.dm_batch ? (dm_end - j0) : g.dm_batch;
        m.j_begin = j0;
        m.n_dm = nb;
        m.Y = P->d_Yb;
        m.y_dm_stride = g.bin_pitch;
        {
          StageTimer t(P, FDD_STAGE_MAC, s);
          FDD_CUDA(fdd::launch_mac_spin(m, P->spin, P->d_pc_spin, P->spin_fp32_variant,
                                        p.precision, P->n_sms, P->d_spin_scratch,
                                        P->spin_scratch_bytes, s));
        }
        if ((st = inverse_and_place(P, io, 0, c, j0, nb, P->d_Yb, s)) != FDD_OK) return st;
      }
    } else {
      m.n_bins = static_cast<int>(g.n_bins);
      m.out_kind = p.output == FDD_OUT_SPECTRA ? 1 : 2;
      m.real_bin_a = -1;
      m.real_bin_b = -1;
      const size_t esz = p.output == FDD_OUT_SPECTRA ? 8 : 4;
      const int step = io.d_out ? io.n_dm : P->block_dm;
      for (int j0 = io.dm_first; j0 < dm_end; j0 += step) {
        const int nb = (dm_end - j0) < step ? (dm_end - j0) : step;
        m.j_begin = j0;
        m.n_dm = nb;
        m.y_dm_stride = g.n_bins;
        int k = -1;
        if (io.d_out) {
          m.Y = static_cast<char*>(io.d_out) +
                esz * ((c * static_cast<int64_t>(io.n_dm) + (j0 - io.dm_first)) * g.n_bins);
        } else {
          if ((st = block_slot(P, io, s, &k)) != FDD_OK) return st;
          m.Y = P->d_blk[k];
        }
        {
          StageTimer t(P, FDD_STAGE_MAC, s);
          FDD_CUDA(fdd::launch_mac_spin(m, P->spin, P->d_pc_spin, P->spin_fp32_variant,
                                        p.precision, P->n_sms, P->d_spin_scratch,
                                        P->spin_scratch_bytes, s));
        }
        if (k >= 0) {
          fdd_block blk{0, 1, c, j0, nb, P->d_blk[k], g.n_bins, g.n_bins, 0, nullptr};
          if ((st = deliver(P, io, k, blk, s)) != FDD_OK) return st;
        }
      }
    }
  }
  return FDD_OK;
}

// Tensor-core form: every beam of a chunk is transformed first, each beam's
// spectra moved into the bin-major X_T[k][beam][chan] the kernel reads (the
// FP16 form's per-bin maxima found on the way), then one launch per DM batch
// dedisperses all of them at once (the beams share each bin's phasors).
fdd_status run_tc(fdd_plan_s* P, const Io& io, cudaStream_t s) {
  fdd_status st;
  const fdd_params& p = P->p;
  const fdd_info& g = P->info;
  const int64_t rows = static_cast<int64_t>(p.n_beams) * p.n_chan;  // X_T row per bin
  unsigned int* absmax = reinterpret_cast<unsigned int*>(P->d_tcx);  // scratch head
  const bool f16 = p.precision == FDD_PREC_FP16 || p.precision == FDD_PREC_FP8;  // scaled
  const int dm_end = io.dm_first + io.n_dm;
  if (P->spin_on) return run_spin(P, io, s);
  for (int64_t c = 0; c < g.n_chunks; ++c) {
    if (f16) FDD_CUDA(cudaMemsetAsync(absmax, 0, sizeof(unsigned int) * g.n_bins, s));
    for (int b = 0; b < p.n_beams; ++b) {
      if ((st = transform(P, io, b, c, P->d_xb, s)) != FDD_OK) return st;
      fdd::BinTransposeArgs t{P->d_xb, g.bin_pitch, p.n_chan, 0, static_cast<int>(g.n_bins),
                              P->d_X + static_cast<int64_t>(b) * p.n_chan, f16 ? absmax : nullptr,
                              rows};
      StageTimer tt(P, FDD_STAGE_TRANSPOSE, s);
      FDD_CUDA(fdd::launch_bin_transpose(t, s));
    }
    fdd::MacArgs m{};
    m.tc_pair = P->info.mac_variant == FDD_MAC_TC_PAIR;
    m.X = P->d_X;
    m.x_bin_stride = rows;
    m.x_series_stride = p.n_chan;
    m.x_chan_stride = 1;
    m.pc = P->d_pc;
    m.n_chan = p.n_chan;
    m.n_bins = static_cast<int>(g.n_bins);
    m.n_series = p.n_beams;
    m.scale = 1.0f;
    m.status = P->d_status;
    m.absmax_ready = 1;  // found by the transposes
    if (p.output == FDD_OUT_TIME) {
      // (shortened inverse: only the bins up to Nyquist of length L / f)
      const int64_t Ls = g.fft_len / g.downsample;
      const int ks = static_cast<int>(Ls / 2 + 1);
      m.n_bins = ks;
      for (int j0 = io.dm_first; j0 < dm_end; j0 += g.dm_batch) {
        const int nb = (dm_end - j0) < g.dm_batch ? (dm_end - j0) : g.dm_batch;
        // bin-major [bin][beam][trial] for every beam of the batch
        m.j_begin = j0;
        m.n_dm = nb;
        m.Y = P->d_Y;
        m.y_bin_stride = static_cast<int64_t>(p.n_beams) * g.dm_batch;
        m.y_series_stride = g.dm_batch;
        m.y_dm_stride = 1;
        m.out_kind = 1;
        m.real_bin_a = 0;
        m.real_bin_b = static_cast<int>(Ls / 2);
        m.scale = whole_rows(P) ? static_cast<float>(1.0 / static_cast<double>(g.fft_len)) : 1.0f;
        {
          StageTimer t(P, FDD_STAGE_MAC, s);
          FDD_CUDA(fdd::launch_mac_tc(m, p.precision, P->n_sms, P->d_tcx, P->tcx_bytes, s));
        }
        for (int b = 0; b < p.n_beams; ++b) {
          // this beam's trials with bins innermost, then its inverse transforms
          fdd::BinUntransposeArgs u{P->d_Y + static_cast<int64_t>(b) * g.dm_batch, 8, 1, nb, ks,
                                    P->d_Yb, 0, g.bin_pitch,
                                    static_cast<int64_t>(p.n_beams) * g.dm_batch};
          {
            StageTimer t(P, FDD_STAGE_TRANSPOSE, s);
            FDD_CUDA(fdd::launch_bin_untranspose(u, s));
          }
          if ((st = inverse_and_place(P, io, b, c, j0, nb, P->d_Yb, s)) != FDD_OK) return st;
        }
      }
    } else {
      m.real_bin_a = -1;
      m.real_bin_b = -1;
      m.out_kind = p.output == FDD_OUT_SPECTRA ? 1 : 2;
      const size_t esz = p.output == FDD_OUT_SPECTRA ? 8 : 4;
      const int step = io.d_out ? io.n_dm : P->block_dm;
      for (int j0 = io.dm_first; j0 < dm_end; j0 += step) {
        const int nb = (dm_end - j0) < step ? (dm_end - j0) : step;
        m.j_begin = j0;
        m.n_dm = nb;
        int k = -1;
        if (io.d_out) {
          m.y_series_stride = g.n_chunks * static_cast<int64_t>(io.n_dm) * g.n_bins;
          m.Y = static_cast<char*>(io.d_out) + esz * (c * static_cast<int64_t>(io.n_dm) * g.n_bins);
        } else {
          if ((st = block_slot(P, io, s, &k)) != FDD_OK) return st;
          m.y_series_stride = static_cast<int64_t>(nb) * g.n_bins;
          m.Y = P->d_blk[k];
        }
        m.y_dm_stride = g.n_bins;
        {
          StageTimer t(P, FDD_STAGE_MAC, s);
          FDD_CUDA(fdd::launch_mac_tc(m, p.precision, P->n_sms, P->d_tcx, P->tcx_bytes, s));
        }
        if (k >= 0) {
          fdd_block blk{0, p.n_beams, c, j0, nb, P->d_blk[k], g.n_bins, g.n_bins, 0, nullptr};
          if ((st = deliver(P, io, k, blk, s)) != FDD_OK) return st;
        }
      }
    }
  }
  return FDD_OK;
}

// The streaming rings (made on the first streamed call): two input windows
// of n_chan x L samples and two output blocks.
fdd_status make_rings(fdd_plan_s* P, bool host) {
  const fdd_params& p = P->p;
  const fdd_info& g = P->info;
  fdd_status st;
  const size_t esz = p.in_dtype == FDD_IN_U8 ? 1 : 4;
  for (int w = 0; w < 2; ++w) {
    if (!P->d_win[w] &&
        (st = ws_alloc(P, &P->d_win[w], esz * static_cast<size_t>(p.n_chan) * g.fft_len)))
      return st;
    if (!P->d_blk[w] && (st = ws_alloc(P, &P->d_blk[w], P->blk_bytes))) return st;
  }
  cudaEvent_t* evs[] = {&P->win_free[0], &P->win_free[1], &P->win_full[0], &P->win_full[1],
                        &P->blk_free[0], &P->blk_free[1], &P->blk_done[0], &P->blk_done[1],
                        &P->pipe_start, &P->pipe_end};
  for (cudaEvent_t* e : evs)
    if (!*e) FDD_CUDA(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
  if (!host) return FDD_OK;
  if (!P->h2d) FDD_CUDA(cudaStreamCreateWithFlags(&P->h2d, cudaStreamNonBlocking));
  if (!P->d2h) FDD_CUDA(cudaStreamCreateWithFlags(&P->d2h, cudaStreamNonBlocking));
  return FDD_OK;
}

}  // namespace

namespace fdd {

fdd_status report_error(fdd_status s, const char* message) { return fail(s, "%s", message); }

std::atomic<long long> g_launches{0};
void note_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
long long launches_so_far() { return g_launches.load(std::memory_order_relaxed); }

// fdd_debug_fail_alloc: allocations to let through before one fails (-1: none).
std::atomic<int> g_fail_alloc{-1};

bool injected_alloc_failure() {
  int k = g_fail_alloc.load();
  while (k >= 0)
    if (g_fail_alloc.compare_exchange_weak(k, k - 1)) return k == 0;  // fails once, then off
  return false;
}


}  // namespace fdd

extern "C" {

int32_t fdd_abi_version(void) { return FDD_ABI_VERSION; }

const char* fdd_status_string(fdd_status s) {
  switch (s) {
    case FDD_OK: return "FDD_OK";
    case FDD_ERR_INVALID_ARG: return "FDD_ERR_INVALID_ARG";
    case FDD_ERR_UNSUPPORTED: return "FDD_ERR_UNSUPPORTED";
    case FDD_ERR_ALLOC: return "FDD_ERR_ALLOC";
    case FDD_ERR_CUDA: return "FDD_ERR_CUDA";
    case FDD_ERR_CUFFT: return "FDD_ERR_CUFFT";
    case FDD_ERR_TIMEOUT: return "FDD_ERR_TIMEOUT";
    case FDD_ERR_DEVICE: return "FDD_ERR_DEVICE";
  }
  return "FDD_ERR_UNKNOWN";
}

const char* fdd_last_error(void) { return g_err; }

void fdd_params_init(fdd_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof *p);
  p->n_beams = 1;
  p->in_dtype = FDD_IN_U8;
  p->in_layout = FDD_LAYOUT_TIME_MAJOR;
  p->output = FDD_OUT_TIME;
  p->precision = FDD_PREC_FP32;
}

fdd_status fdd_plan_geometry(const fdd_params* p, fdd_info* out) {
  return compute_plan(p, out, nullptr);
}

fdd_status fdd_plan(const fdd_params* p, fdd_plan_t* out) {
  return fdd::plan_create(p, nullptr, 0, out);
}

}  // extern "C"

namespace fdd {

fdd_status plan_drain(fdd_plan_t P, cudaStream_t s) {
  for (int k = 0; k < 2; ++k) {
    if (!P->blk_release[k]) continue;
    FDD_CUDA(cudaStreamWaitEvent(s, static_cast<cudaEvent_t>(P->blk_release[k]), 0));
    P->blk_release[k] = nullptr;
  }
  return FDD_OK;
}

size_t plan_arena_used(fdd_plan_t P) { return P->arena_used; }

fdd_status plan_create(const fdd_params* p, void* arena, size_t arena_bytes, fdd_plan_t* out) {
  if (!out) return fail(FDD_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  fdd_plan_s* P = new (std::nothrow) fdd_plan_s();
  if (!P) return fail(FDD_ERR_ALLOC, "host allocation failed");
  std::unique_ptr<fdd_plan_s, void (*)(fdd_plan_s*)> guard(P, release);
  P->arena = static_cast<char*>(arena);
  P->arena_bytes = arena ? arena_bytes : 0;

  fdd_status st = compute_plan(p, &P->info, &P->core);
  if (st != FDD_OK) return st;
  P->rate.resize(p->n_chan);
  for (int c = 0; c < p->n_chan; ++c) P->rate[c] = fdd::delay_rate(*p, P->core, c);
  P->p = *p;
  P->dms.assign(p->dm_list, p->dm_list + p->n_dm);
  P->p.dm_list = nullptr;

  FDD_CUDA(cudaGetDevice(&P->device));
  int major = 0, minor = 0;
  FDD_CUDA(cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, P->device));
  FDD_CUDA(cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, P->device));
  if (major != 10 || minor != 3)
    return fail(FDD_ERR_UNSUPPORTED, "kernels are built for sm_103a; device is sm_%d%d", major,
                minor);
  fdd_info& g = P->info;
  P->tc = p->precision != FDD_PREC_FP32;
  FDD_CUDA(cudaDeviceGetAttribute(&P->n_sms, cudaDevAttrMultiProcessorCount, P->device));
  if (P->tc)
    FDD_CUDA(fdd::mac_tc_prepare());
  else
    FDD_CUDA(fdd::mac_prepare(g.mac_variant, p->n_chan));

  // Exact fixed-point phase rates (see fdd_internal.h).
  P->pc_host.resize(p->n_chan);
  for (int c = 0; c < p->n_chan; ++c)
    P->pc_host[c] = fdd::phase_const(P->rate[c], static_cast<double>(g.fft_len), g.dm0, g.ddm);

  const int nc = p->n_chan;
  if ((st = dev_alloc(P, reinterpret_cast<void**>(&P->d_pc), sizeof(fdd::PhaseConst) * nc)))
    return st;
  if ((st = dev_alloc(P, reinterpret_cast<void**>(&P->d_status), 256))) return st;
  if ((st = ws_alloc(P, reinterpret_cast<void**>(&P->d_xw), sizeof(float) * size_t(nc) * g.fft_len)))
    return st;
  const size_t sets = P->tc ? static_cast<size_t>(p->n_beams) : 1;
  if (P->tc) {
    P->tcx_bytes = fdd::mac_tc_scratch_bytes(p->n_beams, nc, p->n_dm, g.n_bins);
    if ((st = ws_alloc(P, reinterpret_cast<void**>(&P->d_tcx), P->tcx_bytes))) return st;
  }
  if ((st = ws_alloc(P, reinterpret_cast<void**>(&P->d_X),
                     sizeof(float2) * size_t(nc) * g.bin_pitch * sets)))
    return st;
  if (P->tc && (st = ws_alloc(P, reinterpret_cast<void**>(&P->d_xb),
                              sizeof(float2) * size_t(nc) * g.bin_pitch)))
    return st;
  if (P->tc && p->output == FDD_OUT_TIME &&
      (st = ws_alloc(P, reinterpret_cast<void**>(&P->d_Yb),
                     sizeof(float2) * size_t(g.dm_batch) * g.bin_pitch)))
    return st;
  if (p->output == FDD_OUT_TIME) {
    if ((st = ws_alloc(P, reinterpret_cast<void**>(&P->d_Y),
                       sizeof(float2) * size_t(g.dm_batch) * g.bin_pitch * sets)))
      return st;
    if ((st = ws_alloc(P, reinterpret_cast<void**>(&P->d_yt),
                       sizeof(float) * size_t(g.dm_batch) * (g.fft_len / g.downsample))))
      return st;
  }
  FDD_CUDA(cudaMemcpy(P->d_pc, P->pc_host.data(), sizeof(fdd::PhaseConst) * nc,
                      cudaMemcpyHostToDevice));
  if (p->spin_group != 0) {
    // the scaled grid's phase constants (first DM dm0s), its scratch, and the
    // FP32 tile of the bins below the first group
    P->spin_on = true;
    fdd::spin_geometry(g.n_bins, p->n_dm, g.dm0, g.ddm, p->spin_group,
                       p->spin_tol > 0.0 ? p->spin_tol : 0.01, &P->spin);
    std::vector<fdd::PhaseConst> pcs(nc);
    for (int c = 0; c < nc; ++c)
      pcs[c] = fdd::phase_const(P->rate[c], static_cast<double>(g.fft_len), P->spin.dm0s, g.ddm);
    if ((st = dev_alloc(P, reinterpret_cast<void**>(&P->d_pc_spin), sizeof(fdd::PhaseConst) * nc)))
      return st;
    FDD_CUDA(cudaMemcpy(P->d_pc_spin, pcs.data(), sizeof(fdd::PhaseConst) * nc,
                        cudaMemcpyHostToDevice));
    P->spin_scratch_bytes = fdd::spin_scratch_bytes(P->spin, nc, g.n_bins);
    if ((st = ws_alloc(P, &P->d_spin_scratch, P->spin_scratch_bytes))) return st;
    P->spin_fp32_variant = fdd::mac_variant_for(p->n_dm, nc);
    if (fdd::mac_smem_bytes(P->spin_fp32_variant, nc) > kMaxSmem)
      return fail(FDD_ERR_UNSUPPORTED, "n_chan %d needs more shared memory than a CTA has", nc);
    FDD_CUDA(fdd::mac_prepare(P->spin_fp32_variant, nc));
  }
  FDD_CUDA(cudaMemset(P->d_status, 0, 256));

  // cuFFT plans with caller-owned work area (execute never allocates).
  long long n[1] = {g.fft_len};
  long long emb_real[1] = {g.fft_len};
  long long emb_cplx[1] = {g.bin_pitch};
  size_t w_r2c = 0, w_c2r = 0, w_tail = 0;
  FDD_CUFFT(cufftCreate(&P->r2c));
  P->has_r2c = true;
  FDD_CUFFT(cufftSetAutoAllocation(P->r2c, 0));
  FDD_CUFFT(cufftMakePlanMany64(P->r2c, 1, n, emb_real, 1, g.fft_len, emb_cplx, 1, g.bin_pitch,
                                CUFFT_R2C, nc, &w_r2c));
  if (p->output == FDD_OUT_TIME) {
    // inverse transforms of length L / downsample over the first bins of each row
    // (one beam's DM batch, rows of bin_pitch bins, for both forms)
    long long ns[1] = {g.fft_len / g.downsample};
    auto make_c2r = [&](cufftHandle* h, int batch, size_t* work) -> fdd_status {
      FDD_CUFFT(cufftCreate(h));
      FDD_CUFFT(cufftSetAutoAllocation(*h, 0));
      FDD_CUFFT(cufftMakePlanMany64(*h, 1, ns, emb_cplx, 1, g.bin_pitch, ns, 1, ns[0],
                                    CUFFT_C2R, batch, work));
      return FDD_OK;
    };
    P->has_c2r = true;
    if ((st = make_c2r(&P->c2r, g.dm_batch, &w_c2r)) != FDD_OK) return st;
    const int tail = p->n_dm % g.dm_batch;
    if (tail != 0) {
      P->has_c2r_tail = true;
      P->c2r_tail_batch = tail;
      if ((st = make_c2r(&P->c2r_tail, tail, &w_tail)) != FDD_OK) return st;
    }
  }
  size_t w = w_r2c > w_c2r ? w_r2c : w_c2r;
  w = w > w_tail ? w : w_tail;
  if (w > 0) {
    if ((st = ws_alloc(P, &P->d_fftwork, w))) return st;
    FDD_CUFFT(cufftSetWorkArea(P->r2c, P->d_fftwork));
    if (P->has_c2r) FDD_CUFFT(cufftSetWorkArea(P->c2r, P->d_fftwork));
    if (P->has_c2r_tail) FDD_CUFFT(cufftSetWorkArea(P->c2r_tail, P->d_fftwork));
  }
  g.workspace_bytes = static_cast<int64_t>(P->bytes_held);
  P->block_dm = g.block_dm;
  P->blk_bytes = p->output == FDD_OUT_TIME
                     ? sizeof(float) * static_cast<size_t>(g.dm_batch) * (g.hop / g.downsample)
                     : (p->output == FDD_OUT_SPECTRA ? 8 : 4) * sets *
                           static_cast<size_t>(g.n_bins) * g.block_dm;
  *out = guard.release();
  return FDD_OK;
}

}  // namespace fdd

extern "C" {

fdd_status fdd_query(fdd_plan_t plan, fdd_info* out) {
  if (!plan || !out) return fail(FDD_ERR_INVALID_ARG, "NULL plan or info");
  *out = plan->info;
  int word = 0;
  FDD_CUDA(cudaMemcpy(&word, plan->d_status, sizeof word, cudaMemcpyDeviceToHost));
  if (word == 0) return FDD_OK;
  FDD_CUDA(cudaMemset(plan->d_status, 0, sizeof word));  // reported once
  if (word == FDD_ERR_TIMEOUT) return fail(FDD_ERR_TIMEOUT, "a device-side wait timed out");
  return fail(FDD_ERR_DEVICE, "device status word %d", word);
}

fdd_status fdd_debug_fail_alloc(int32_t after) {
  fdd::g_fail_alloc.store(after < 0 ? -1 : after);
  return FDD_OK;
}

fdd_status fdd_debug_stall_test(fdd_plan_t plan, fdd_stream_t stream) {
  if (!plan) return fail(FDD_ERR_INVALID_ARG, "plan is NULL");
  fdd_status st = check_device(plan);
  if (st != FDD_OK) return st;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  // One bin, one trial, one series: a single CTA whose producers withhold
  // every arrival; the plan's spectra buffer serves as (unread-for-value) X.
  void* y = nullptr;
  FDD_CUDA(cudaMalloc(&y, 64));
  fdd::MacArgs m{};
  m.tc_pair = plan->info.mac_variant == FDD_MAC_TC_PAIR;
  m.X = plan->d_X;
  m.x_chan_stride = plan->info.bin_pitch;
  m.x_series_stride = plan->info.bin_pitch * plan->p.n_chan;
  m.pc = plan->d_pc;
  m.n_chan = plan->p.n_chan;
  m.n_bins = 1;
  m.n_series = 1;
  m.j_begin = 0;
  m.n_dm = 1;
  m.Y = y;
  m.y_dm_stride = 1;
  m.y_series_stride = 1;
  m.out_kind = 1;
  m.scale = 1.0f;
  m.real_bin_a = -1;
  m.real_bin_b = -1;
  m.status = plan->d_status;
  m.test_withhold = 1;
  cudaError_t e;
  if (plan->tc) {
    e = fdd::launch_mac_tc(m, plan->p.precision, plan->n_sms, plan->d_tcx,
                           plan->tcx_bytes, s);
  } else {
    e = fdd::mac_prepare(fdd::MAC_W12_8x8, plan->p.n_chan);
    if (e == cudaSuccess) e = fdd::launch_mac_fp32(m, fdd::MAC_W12_8x8, s);
  }
  const cudaError_t es = cudaStreamSynchronize(s);
  cudaFree(y);
  if (e != cudaSuccess) return fail(FDD_ERR_CUDA, "%s", cudaGetErrorString(e));
  if (es != cudaSuccess) return fail(FDD_ERR_CUDA, "%s", cudaGetErrorString(es));
  return FDD_OK;
}

fdd_status fdd_execute_dm_range(fdd_plan_t plan, const void* d_in, int32_t dm_first,
                                int32_t n_dm, void* d_out, fdd_stream_t stream) {
  if (!plan) return fail(FDD_ERR_INVALID_ARG, "plan is NULL");
  if (!d_in || !d_out) return fail(FDD_ERR_INVALID_ARG, "NULL input or output");
  if (dm_first < 0 || n_dm < 1 || dm_first + static_cast<int64_t>(n_dm) > plan->p.n_dm)
    return fail(FDD_ERR_INVALID_ARG, "trial range [%d, %d) outside [0, %d)", dm_first,
                dm_first + n_dm, plan->p.n_dm);
  fdd_status st = check_device(plan);
  if (st != FDD_OK) return st;
  if ((st = need_uniform_grid(plan)) != FDD_OK) return st;
  Io io;
  io.d_in = d_in;
  io.d_out = d_out;
  io.dm_first = dm_first;
  io.n_dm = n_dm;
  return run(plan, io, reinterpret_cast<cudaStream_t>(stream));
}

fdd_status fdd_execute(fdd_plan_t plan, const void* d_in, void* d_out, fdd_stream_t stream) {
  if (!plan) return fail(FDD_ERR_INVALID_ARG, "plan is NULL");
  return fdd_execute_dm_range(plan, d_in, 0, plan->p.n_dm, d_out, stream);
}

fdd_status fdd_execute_stream(fdd_plan_t plan, const void* d_in, fdd_source_fn source,
                              void* source_user, fdd_sink_fn sink, void* sink_user,
                              fdd_stream_t stream) {
  if (!plan) return fail(FDD_ERR_INVALID_ARG, "plan is NULL");
  if (!sink) return fail(FDD_ERR_INVALID_ARG, "NULL sink");
  if ((d_in == nullptr) == (source == nullptr))
    return fail(FDD_ERR_INVALID_ARG, "give exactly one of d_in and source");
  fdd_status st = check_device(plan);
  if (st != FDD_OK) return st;
  if ((st = need_uniform_grid(plan)) != FDD_OK) return st;
  if ((st = make_rings(plan, false)) != FDD_OK) return st;
  Io io;
  io.d_in = d_in;
  io.source = source;
  io.source_user = source_user;
  io.sink = sink;
  io.sink_user = sink_user;
  io.dm_first = 0;
  io.n_dm = plan->p.n_dm;
  return run(plan, io, reinterpret_cast<cudaStream_t>(stream));
}

fdd_status fdd_execute_host(fdd_plan_t plan, const void* h_in, void* h_out, fdd_stream_t stream) {
  if (!plan) return fail(FDD_ERR_INVALID_ARG, "plan is NULL");
  if (!h_in || !h_out) return fail(FDD_ERR_INVALID_ARG, "NULL input or output");
  fdd_status st = check_device(plan);
  if (st != FDD_OK) return st;
  if ((st = need_uniform_grid(plan)) != FDD_OK) return st;
  if ((st = make_rings(plan, true)) != FDD_OK) return st;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  Io io;
  io.h_in = static_cast<const char*>(h_in);
  io.h_out = static_cast<char*>(h_out);
  io.dm_first = 0;
  io.n_dm = plan->p.n_dm;
  // the copy streams start after the work already queued on the caller's stream
  FDD_CUDA(cudaEventRecord(plan->pipe_start, s));
  FDD_CUDA(cudaStreamWaitEvent(plan->h2d, plan->pipe_start, 0));
  FDD_CUDA(cudaStreamWaitEvent(plan->d2h, plan->pipe_start, 0));
  st = run(plan, io, s);
  if (st != FDD_OK) return st;
  // and the caller's stream ends after the last copy back
  FDD_CUDA(cudaEventRecord(plan->pipe_end, plan->d2h));
  FDD_CUDA(cudaStreamWaitEvent(s, plan->pipe_end, 0));
  return FDD_OK;
}

fdd_status fdd_dedisperse_spectra_bins(fdd_plan_t plan, const void* d_X, int64_t x_pitch,
                                       int32_t n_series, int32_t bin_first, int32_t n_bins,
                                       int32_t dm_first, int32_t n_dm, void* d_Y,
                                       int64_t y_pitch, int32_t out_kind, fdd_stream_t stream) {
  if (!plan) return fail(FDD_ERR_INVALID_ARG, "plan is NULL");
  if (!d_X || !d_Y) return fail(FDD_ERR_INVALID_ARG, "NULL spectra pointer");
  const fdd_info& g = plan->info;
  if (bin_first < 0 || n_bins < 1 || bin_first + static_cast<int64_t>(n_bins) > g.n_bins)
    return fail(FDD_ERR_INVALID_ARG, "bin range [%d, %lld) outside [0, %lld)", bin_first,
                static_cast<long long>(bin_first) + n_bins, (long long)g.n_bins);
  if (x_pitch < n_bins || y_pitch < n_bins)
    return fail(FDD_ERR_INVALID_ARG, "pitches must be >= n_bins (%d)", n_bins);
  if (n_series < 1 || n_series > 65535)
    return fail(FDD_ERR_INVALID_ARG, "n_series must be in [1, 65535]");
  if (dm_first < 0 || n_dm < 1 || dm_first + static_cast<int64_t>(n_dm) > plan->p.n_dm)
    return fail(FDD_ERR_INVALID_ARG, "trial range outside the plan's list");
  if (out_kind != FDD_OUT_SPECTRA && out_kind != FDD_OUT_POWER)
    return fail(FDD_ERR_INVALID_ARG, "out_kind must be FDD_OUT_SPECTRA or FDD_OUT_POWER");
  if (plan->tc && fdd::mac_tc_min_scratch(n_series, plan->p.n_chan, n_dm, n_bins) > plan->tcx_bytes)
    return fail(FDD_ERR_UNSUPPORTED,
                "the spectra and outputs of one bin exceed the tensor-core form's scratch");
  fdd_status st = check_device(plan);
  if (st != FDD_OK) return st;
  if ((st = need_uniform_grid(plan)) != FDD_OK) return st;
  fdd::MacArgs m{};
  m.tc_pair = plan->info.mac_variant == FDD_MAC_TC_PAIR;
  m.X = static_cast<const float2*>(d_X);
  m.x_chan_stride = x_pitch;
  m.x_series_stride = x_pitch * plan->p.n_chan;
  m.pc = plan->d_pc;
  m.n_chan = plan->p.n_chan;
  m.n_bins = n_bins;
  m.k_begin = bin_first;
  m.n_series = n_series;
  m.j_begin = dm_first;
  m.n_dm = n_dm;
  m.Y = d_Y;
  m.y_dm_stride = y_pitch;
  m.y_series_stride = y_pitch * n_dm;
  m.out_kind = out_kind == FDD_OUT_SPECTRA ? 1 : 2;
  m.scale = 1.0f;
  m.real_bin_a = -1;
  m.real_bin_b = -1;
  m.status = plan->d_status;
  StageTimer t(plan, FDD_STAGE_MAC, reinterpret_cast<cudaStream_t>(stream));
  if (plan->spin_on) {
    if (bin_first != 0 || n_bins != g.n_bins || n_series != 1)
      return fail(FDD_ERR_UNSUPPORTED,
                  "spin-frequency grids take one series of every bin (no bin windows)");
    FDD_CUDA(fdd::launch_mac_spin(m, plan->spin, plan->d_pc_spin, plan->spin_fp32_variant,
                                  plan->p.precision, plan->n_sms, plan->d_spin_scratch,
                                  plan->spin_scratch_bytes, reinterpret_cast<cudaStream_t>(stream)));
  } else if (plan->tc)
    FDD_CUDA(fdd::launch_mac_tc(m, plan->p.precision, plan->n_sms,
                                plan->d_tcx, plan->tcx_bytes,
                                reinterpret_cast<cudaStream_t>(stream)));
  else
    FDD_CUDA(fdd::launch_mac_fp32(m, g.mac_variant, reinterpret_cast<cudaStream_t>(stream)));
  return FDD_OK;
}

fdd_status fdd_dedisperse_spectra(fdd_plan_t plan, const void* d_X, int64_t x_pitch,
                                  int32_t n_series, int32_t dm_first, int32_t n_dm, void* d_Y,
                                  int64_t y_pitch, int32_t out_kind, fdd_stream_t stream) {
  if (!plan) return fail(FDD_ERR_INVALID_ARG, "plan is NULL");
  return fdd_dedisperse_spectra_bins(plan, d_X, x_pitch, n_series, 0,
                                     static_cast<int32_t>(plan->info.n_bins), dm_first, n_dm,
                                     d_Y, y_pitch, out_kind, stream);
}

fdd_status fdd_tdd_execute(fdd_plan_t plan, const void* d_in, void* d_out, fdd_stream_t stream) {
  if (!plan) return fail(FDD_ERR_INVALID_ARG, "plan is NULL");
  if (!d_in || !d_out) return fail(FDD_ERR_INVALID_ARG, "NULL input or output");
  const fdd_params& p = plan->p;
  const fdd_info& g = plan->info;
  const int64_t out_len = p.n_t - g.d_max;
  if (out_len <= 0)
    return fail(FDD_ERR_INVALID_ARG, "n_t %lld does not exceed the largest delay %lld",
                (long long)p.n_t, (long long)g.d_max);
  if (out_len > int64_t(65535) * fdd::kTdSamp)
    return fail(FDD_ERR_UNSUPPORTED, "more than %lld output samples per trial",
                (long long)int64_t(65535) * fdd::kTdSamp);
  fdd_status st = check_device(plan);
  if (st != FDD_OK) return st;
  const int nc = p.n_chan, nd = p.n_dm;
  if (!plan->d_shift) {
    // Eq. 1 delays in samples (FP64), rounded to the nearest sample (halves
    // away from zero; delays are >= 0), and per block of kTdDms trials the
    // smallest shift of each channel and the widest span.
    std::vector<int> sh(static_cast<size_t>(nd) * nc);
    for (int j = 0; j < nd; ++j)
      for (int c = 0; c < nc; ++c) {
        const double d = plan->dms[j] * plan->rate[c];
        if (!(d >= 0.0) || d > 2.0e9) return fail(FDD_ERR_UNSUPPORTED, "delay out of range");
        sh[static_cast<size_t>(j) * nc + c] = static_cast<int>(std::floor(d + 0.5));
      }
    const int n_blk = (nd + fdd::kTdDms - 1) / fdd::kTdDms;
    std::vector<int> base(static_cast<size_t>(n_blk) * nc);
    std::vector<int> rel(static_cast<size_t>(n_blk) * nc * fdd::kTdDms, 0);
    int span = 0;
    for (int b = 0; b < n_blk; ++b)
      for (int c = 0; c < nc; ++c) {
        int lo = INT_MAX, hi = INT_MIN;
        for (int j = b * fdd::kTdDms; j < nd && j < (b + 1) * fdd::kTdDms; ++j) {
          lo = std::min(lo, sh[static_cast<size_t>(j) * nc + c]);
          hi = std::max(hi, sh[static_cast<size_t>(j) * nc + c]);
        }
        base[static_cast<size_t>(b) * nc + c] = lo;
        span = std::max(span, hi - lo);
        for (int j = b * fdd::kTdDms; j < nd && j < (b + 1) * fdd::kTdDms; ++j)
          rel[(static_cast<size_t>(b) * nc + c) * fdd::kTdDms + (j - b * fdd::kTdDms)] =
              sh[static_cast<size_t>(j) * nc + c] - lo;
      }
    const int win = (fdd::kTdSamp + span + 3) / 4 * 4;
    if (fdd::tdd_smem_bytes(win) > kMaxSmem)
      return fail(FDD_ERR_UNSUPPORTED,
                  "a block of %d trials spans %d samples of delay in one channel", fdd::kTdDms,
                  span);
    if ((st = dev_alloc(plan, reinterpret_cast<void**>(&plan->d_shift), sizeof(int) * rel.size())))
      return st;
    if ((st = dev_alloc(plan, reinterpret_cast<void**>(&plan->d_shift_base),
                        sizeof(int) * base.size())))
      return st;
    if ((st = dev_alloc(plan, reinterpret_cast<void**>(&plan->d_tdd_x),
                        sizeof(float) * static_cast<size_t>(nc) * p.n_t)))
      return st;
    FDD_CUDA(cudaMemcpy(plan->d_shift, rel.data(), sizeof(int) * rel.size(),
                        cudaMemcpyHostToDevice));
    FDD_CUDA(cudaMemcpy(plan->d_shift_base, base.data(), sizeof(int) * base.size(),
                        cudaMemcpyHostToDevice));
    FDD_CUDA(fdd::tdd_prepare(win));
    plan->tdd_win = win;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const size_t esz = p.in_dtype == FDD_IN_U8 ? 1 : 4;
  const int64_t beam_elems = p.n_t * static_cast<int64_t>(nc);
  for (int b = 0; b < p.n_beams; ++b) {
    fdd::UnpackArgs ua{static_cast<const char*>(d_in) + esz * beam_elems * b, p.in_dtype,
                       p.in_layout, nc, p.n_t, 0, p.n_t, plan->d_tdd_x, p.n_t};
    {
      StageTimer t(plan, FDD_STAGE_UNPACK, s);
      FDD_CUDA(fdd::launch_unpack(ua, s));
    }
    fdd::TddArgs ta{plan->d_tdd_x, p.n_t, nc, plan->d_shift, plan->d_shift_base, nd,
                    plan->tdd_win,
                    static_cast<float*>(d_out) + static_cast<int64_t>(b) * nd * out_len, out_len};
    StageTimer t(plan, FDD_STAGE_TDD, s);
    FDD_CUDA(fdd::launch_tdd(ta, s));
  }
  return FDD_OK;
}

fdd_status fdd_profile_enable(fdd_plan_t plan, int32_t on) {
  if (!plan) return fail(FDD_ERR_INVALID_ARG, "plan is NULL");
  if (on) {
    if (plan->prof_ev.empty()) {
      plan->prof_ev.assign(2 * kProfSlots, nullptr);
      plan->prof_stage.assign(kProfSlots, 0);
      for (auto& e : plan->prof_ev) FDD_CUDA(cudaEventCreate(&e));
    }
    plan->prof_n = 0;
    plan->prof_dropped = 0;
    plan->prof_launch0 = fdd::launches_so_far();
  }
  plan->prof_on = on != 0;
  return FDD_OK;
}

fdd_status fdd_profile_read(fdd_plan_t plan, fdd_profile* out) {
  if (!plan || !out) return fail(FDD_ERR_INVALID_ARG, "NULL plan or profile");
  std::memset(out, 0, sizeof *out);
  out->dropped = plan->prof_dropped;
  out->kernels = fdd::launches_so_far() - plan->prof_launch0;
  if (plan->prof_n == 0) return FDD_OK;
  FDD_CUDA(cudaEventSynchronize(plan->prof_ev[2 * (plan->prof_n - 1) + 1]));
  for (int i = 0; i < plan->prof_n; ++i) {
    float ms = 0.f;
    FDD_CUDA(cudaEventElapsedTime(&ms, plan->prof_ev[2 * i], plan->prof_ev[2 * i + 1]));
    const int st = plan->prof_stage[i];
    out->launches[st] += 1;
    out->ms[st] += ms;
  }
  return FDD_OK;
}

fdd_status fdd_destroy(fdd_plan_t plan) {
  if (!plan) return FDD_OK;
  cudaError_t e = cudaDeviceSynchronize();
  release(plan);
  if (e != cudaSuccess)
    return fail(FDD_ERR_CUDA, "cudaDeviceSynchronize: %s", cudaGetErrorString(e));
  return FDD_OK;
}

}  // extern "C"

// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "fdd.h"

namespace fdd {

// Per-channel 64-bit fixed-point phase constants (fractions of a cycle):
//   u = frac(DM_0 * c_nu / L) * 2^64,  v = frac(dDM * c_nu / L) * 2^64,
// with c_nu the delay rate of Eq. 1 in samples per unit DM.  The phase of the
// Eq. 4 phasor for bin k and trial j is then exactly (k u + k j v) mod 2^64.
struct PhaseConst {
  uint32_t u_lo, u_hi, v_lo, v_hi;
};

// Phase-rotate-and-sum launch arguments (Eq. 7 over one set of spectra).
struct MacArgs {
  const float2* X;          // [n_series][n_chan][x_chan_stride]
  int64_t x_series_stride;  // complex elements
  int64_t x_chan_stride;    // complex elements
  int64_t x_bin_stride;     // complex elements between bins; read by the tensor-core
                            // kernel only (the FP32 kernels take bins contiguous)
  const PhaseConst* pc;     // [n_chan]
  int n_chan;
  int n_bins;               // bins handled by this call (local indices 0 .. n_bins-1)
  int k_begin;              // absolute bin index of local bin 0 (phases use k_begin + k)
  int k_step;               // tensor-core kernel only: phases use k_begin + k * k_step
                            // (0 or 1: consecutive bins; G: one reference bin per
                            // group of G bins, the groups' bins being the series)
  int n_series;
  int j_begin;              // first global trial index handled by this call
  int n_dm;                 // trials handled by this call
  void* Y;                  // [n_series][n_dm][y_dm_stride] complex or float
  int64_t y_series_stride;  // elements of the output type
  int64_t y_dm_stride;      // elements of the output type
  int64_t y_bin_stride;     // elements between bins; used by the tensor-core kernel only
                            // (the FP32 kernels write bins contiguous)
  int out_kind;             // 1 = complex spectra, 2 = |Y|^2
  float scale;              // multiplies Y before the store (power: |scale Y|^2)
  int real_bin_a;           // absolute bins whose imaginary part is set to zero, or -1
  int real_bin_b;
  int* status;              // device status word (may be NULL)
  int test_withhold;        // self-test only: producers never announce a filled stage,
                            // so the consumers' bounded waits run out (FDD_ERR_TIMEOUT)
  const float* bin_absmax;  // tensor cores in FP16 only: per local bin, the largest
                            // |re| or |im| of the spectra (sets that bin's data scale)
  int absmax_ready;         // tensor cores in FP16: the scratch already holds the
                            // per-bin maxima of these spectra (a later DM batch)
  int tc_pair;              // tensor cores: the CTA-pair form (the plan's choice)
};

// Kernel variants of the FP32 phasor-MAC (see fdd_mac_fp32.cu and the
// FDD_MAC_* list in fdd.h).
enum MacVariant {
  MAC_W12_8x8 = FDD_MAC_W12_8X8,
  MAC_Q12_8x8 = FDD_MAC_Q12_8X8,
  MAC_Q_4x8 = FDD_MAC_Q_4X8,
  MAC_Q_8x8_512 = FDD_MAC_Q_8X8_512,
  MAC_Q_4x4 = FDD_MAC_Q_4X4,
  MAC_G12_4x8 = FDD_MAC_G12_4X8,
  MAC_NUM_VARIANTS = FDD_MAC_VARIANTS
};
// One set of spectra in a batch (the batching form): its launch arguments
// (n_series 1) and its place in the batch's work-item numbering.
struct BatchSet {
  MacArgs args;
  long long item_begin;  // first work item of this set
  int n_dm_blocks;       // trial blocks (items per bin tile)
  int n_bin_tiles;
  // the three-product tile only, numbered after the n_bin_tiles x
  // n_dm_blocks items: wide items of 1024 trials (twice the bins) from trial
  // j_wide, then wide items of 512 trials (four times the bins) from j_narrow
  int n_wide_tiles;
  int j_wide;
  int n_narrow_tiles;
  int j_narrow;
};

// The FP32 tile with the least time for n_dm trials among those whose
// shared memory holds n_chan channels' phase constants.
int mac_variant_for(int n_dm, int n_chan);
int mac_variant_bins_per_cta(int variant);
bool mac_variant_batchable(int variant);
// CTAs of the persistent batch kernel per SM (occupancy), 0 if unsupported.
int mac_batch_ctas_per_sm(int variant, int n_chan);
cudaError_t launch_mac_batch(const BatchSet* d_sets, int n_sets, long long n_items,
                             unsigned long long* d_counter, int variant, int n_ctas,
                             int n_chan, cudaStream_t s);
int mac_variant_trials_per_block(int variant);
cudaError_t mac_prepare(int variant, int n_chan);  // kernel attributes (host, once)
cudaError_t launch_mac_fp32(const MacArgs& a, int variant, cudaStream_t s);
size_t mac_smem_bytes(int variant, int n_chan);

// Tensor-core phase-rotate-and-sum (fdd_mac_tc.cu): 16-bit (or FP8)
// phasors and data, FP32 accumulation in tensor memory; persistent CTAs (one
// per SM), alone or in pairs (one bin per pair at a time).
size_t mac_tc_smem_bytes();
// trials of one pass over the channels, and of one a (T = 128, or 256 for
// the CTA-pair form)
int mac_tc_trials_per_pass(int n_series, bool pair);
int mac_tc_trials_per_a(bool pair);
// Sets the kernels' shared-memory limit and counts the pairs resident at once
// on the current device (before the first call on it).
cudaError_t mac_tc_prepare();
// Beams per tensor-core group: 16 when a call has at most 16 series (then a
// pass covers 2048 trials, 4096 for a pair), else 32 (1024, 2048).
int mac_tc_beams_per_group(int n_series);
// The tensor-core kernel reads the spectra bin-major, X_T[k][series][chan]
// (a 256-byte row per 32 channels of one beam), and writes Y bin-major,
// Y_T[k][series][trial] (every warp store contiguous).  launch_mac_tc takes
// either layout on each side: a.x_bin_stride > 0 means X is bin-major at the
// given strides (x_chan_stride 1) and is read in place, 0 means X is
// [series][chan][pitch] with bins innermost (x_series_stride = n_chan x
// x_chan_stride) and is moved bin-major into `scratch` a block of bins at a
// time; likewise a.y_bin_stride > 0 writes Y in place bin-major, 0 writes a
// block bin-major into the scratch and moves it into the caller's layout
// (bins innermost).  The FP16 form first finds each bin's largest component.
// mac_tc_scratch_bytes: the scratch a plan allocates for calls of up to n_dm
// trials on n_series x n_chan spectra of n_bins bins in the caller's layouts
// (per-bin maxima, blocks of at most 3 GiB, at least one bin);
// mac_tc_min_scratch: the least scratch such a call needs.
size_t mac_tc_scratch_bytes(int n_series, int n_chan, int n_dm, int64_t n_bins);
size_t mac_tc_min_scratch(int n_series, int n_chan, int n_dm, int64_t n_bins);
// precision: FDD_PREC_BF16_HILO, FDD_PREC_BF16 or FDD_PREC_FP16.
cudaError_t launch_mac_tc(const MacArgs& a, int precision, int n_sms, float2* scratch,
                          size_t scratch_bytes, cudaStream_t s);

// Bins k0 .. k0 + n_bins - 1 of `rows` complex rows of stride in_stride into
// out[k][row] (bin-major), for the tensor-core kernel.
struct BinTransposeArgs {
  const float2* in;      // row r, bin k at in + r * in_stride + k
  int64_t in_stride;
  int64_t rows;
  int64_t k0;
  int n_bins;
  float2* out;           // bin k, row r at out + k * out_bin_stride + r
  unsigned int* absmax;  // optional: per bin, atomic max of the bits of max(|re|, |im|)
                         // over the rows (non-negative floats order as their bits);
                         // the caller zeroes it first
  int64_t out_bin_stride = 0;  // 0: rows
};
cudaError_t launch_bin_transpose(const BinTransposeArgs& a, cudaStream_t s);

// Per bin k < n_bins of bin-major spectra (rows contiguous: in[k * bin_stride
// + r], r < rows), the bits of the largest |re| or |im| into absmax[k]: the
// FP16 tensor-core form's per-bin data scale.
struct BinAbsmaxArgs {
  const float2* in;
  int64_t bin_stride;
  int rows;
  int n_bins;
  unsigned int* absmax;
};
cudaError_t launch_bin_absmax(const BinAbsmaxArgs& a, cudaStream_t s);

// The way back for the output: in[k][series][trial] (bin-major, n_bins bins)
// into out + series * out_series_stride + trial * out_dm_stride + k.
struct BinUntransposeArgs {
  const void* in;
  int elem_bytes;        // 8 (complex) or 4 (power)
  int n_series;
  int n_dm;
  int n_bins;
  void* out;
  int64_t out_series_stride;  // elements
  int64_t out_dm_stride;      // elements
  int64_t in_bin_stride = 0;  // elements between bins of `in`; 0: n_series * n_dm
};
cudaError_t launch_bin_untranspose(const BinUntransposeArgs& a, cudaStream_t s);

// The tensor-core kernel on bin-major spectra and output at the strides in a
// (x_bin_stride, y_bin_stride > 0), with a.bin_absmax already holding the FP16
// form's per-bin maxima: no scratch, one launch.
cudaError_t launch_mac_tc_direct(const MacArgs& a, int precision, int n_sms, cudaStream_t s);

// A plan whose per-call buffers (spectra, scratch, transform staging, FFT
// work area, streaming rings) are taken from a caller's device block
// [arena, arena + arena_bytes) instead of its own allocations (arena NULL:
// fdd_plan).  Plans sharing one block must run one after another on one
// stream, each drained (plan_drain) before the next starts.
fdd_status plan_create(const fdd_params* p, void* arena, size_t arena_bytes, fdd_plan_t* out);
// Bytes of the borrowed block in use (after the first streamed call: with
// its rings).
size_t plan_arena_used(fdd_plan_t plan);
// Make stream s wait for the sink release events the plan still holds.
fdd_status plan_drain(fdd_plan_t plan, cudaStream_t s);

// Spin-frequency-dependent DM grids (fdd_spin.cu; Sect. 2.3, Eqs. 8 and 9).
struct SpinGeometry {
  int G;             // bins per group (16 or 32)
  double eps;        // largest relative DM contraction within a group
  int k_min;         // first grouped bin: max(1, ceil((G - 1) / eps)), at most K
  int j_lo;          // the scaled grid starts at trial j_lo of the plan's grid (<= 0)
  int n_s;           // trials of the scaled grid, n_dm - j_lo
  double dm0, ddm;   // the plan's grid
  double dm0s;       // first DM of the scaled grid, dm0 + j_lo ddm
};
void spin_geometry(int64_t K, int n_dm, double dm0, double ddm, int G, double eps,
                   SpinGeometry* out);
// Scratch of launch_mac_spin: blocks of groups of at most 3 GiB.
size_t spin_scratch_bytes(const SpinGeometry& sg, int n_chan, int64_t K);
// Eq. 7 of one beam on the spin-frequency-dependent grids: a.X bins
// innermost [chan][x_chan_stride], a.Y bins innermost (y_dm_stride), all K
// = a.n_bins bins (k_begin 0), trials a.j_begin .. + a.n_dm of the plan's
// grid; a.pc the plan's phase table (bins below k_min, on the FP32 tile
// fp32_variant), pc_spin that of the scaled grid (first DM dm0s).
cudaError_t launch_mac_spin(const MacArgs& a, const SpinGeometry& sg, const PhaseConst* pc_spin,
                            int fp32_variant, int precision, int n_sms, void* scratch,
                            size_t scratch_bytes, cudaStream_t s);

// Allocation-failure injection (fdd_debug_fail_alloc): true when this device
// allocation is to fail; every library allocator asks before cudaMalloc.
bool injected_alloc_failure();

// Kernels this library has launched (process wide): every launch wrapper
// adds to it; the profiling calls report the count over a profiled region.
void note_launches(int n);
long long launches_so_far();

// The last-error setter shared by every translation unit (never allocates).
fdd_status report_error(fdd_status s, const char* message);

// The plan constants every entry point derives from fdd_params, validated and
// computed without allocating (fdd_plan, fdd_plan_geometry, fdd_batch_plan
// per beam, and the allocation-free entry point all use these):
//   Eq. 1 reference frequency and dispersion constant, the largest delay,
//   the DM grid, the transform length and the overlap-save chunking
//   (Sect. 2.2 discard rule, Sect. 3 zero padding), down-sampling.
struct CoreGeometry {
  double nu_ref;     // Eq. 1 reference frequency nu_0, MHz
  double k_dm;       // dispersion constant in use, MHz^2 pc^-1 cm^3 s
  double rate_max;   // largest delay per unit DM over the channels, samples
  double dm0, ddm;   // first trial and step of the list
  int uniform;       // 1 when the list is an arithmetic progression
  int downsample;    // factor of the shortened inverse transform (1: none)
  int64_t d_max;     // ceil of the largest delay, samples
  int64_t L, n_bins, hop, n_chunks, out_len, valid_len;
};
fdd_status core_geometry(const fdd_params* p, CoreGeometry* out);
// Eq. 1: the delay of channel c per unit DM, in samples.
double delay_rate(const fdd_params& p, const CoreGeometry& g, int c);
// The exact fixed-point phase constants of a channel with delay rate `rate`
// (samples per unit DM) for transform length L and the trial grid dm0 + j ddm.
PhaseConst phase_const(double rate, double L, double dm0, double ddm);

// Unpack / transpose / chunk / zero-pad (Sect. 3: transpose_and_unpack and
// zero_pad of Algorithm 1) of one beam into channel-major float series.
struct UnpackArgs {
  const void* in;        // one beam of input
  int in_dtype;          // FDD_IN_U8 | FDD_IN_F32
  int in_layout;         // FDD_LAYOUT_*
  int n_chan;
  int64_t n_t;
  int64_t t_begin;       // first input sample of the chunk
  int64_t L;             // samples per output series
  float* out;            // [n_chan][out_stride]
  int64_t out_stride;
};
cudaError_t launch_unpack(const UnpackArgs& a, cudaStream_t s);

// Scale by 1/L and place the first n_keep samples of each DM series of one
// chunk into the time-domain output (the discard rule of Sect. 2.2).
struct ScatterArgs {
  const float* src;      // [n_dm][src_stride]
  int64_t src_stride;
  float* dst;            // row r of the output at dst + r * dst_stride
  int64_t dst_stride;
  int n_dm;
  int64_t n_keep;
  float scale;
};
cudaError_t launch_scatter(const ScatterArgs& a, cudaStream_t s);

// Brute-force time-domain dedispersion (fdd_tdd.cu), Eq. 2.
constexpr int kTdDms = 32;   // trials per CTA
constexpr int kTdSamp = 256;  // output samples per CTA
constexpr int kTdCh = 8;     // channels per shared-memory stage
struct TddArgs {
  const float* x;     // one beam, channel-major [n_chan][n_t]
  int64_t n_t;
  int n_chan;
  const int* rel;     // [blocks of kTdDms trials][n_chan][kTdDms]: the delays of Eq. 1
                      // rounded to the nearest sample, minus the block's smallest
                      // (0 for trials beyond n_dm)
  const int* base;    // [blocks of kTdDms trials][n_chan] smallest shift of the block
  int n_dm;
  int win;            // window floats per channel: kTdSamp + the largest shift span
                      // of a block, rounded up to a multiple of 4
  float* y;           // [n_dm][out_len]
  int64_t out_len;    // valid samples, n_t - D_max
};
size_t tdd_smem_bytes(int win);
cudaError_t tdd_prepare(int win);
cudaError_t launch_tdd(const TddArgs& a, cudaStream_t s);

}  // namespace fdd

/*
 * fdd.h -- C ABI of the GB300 (sm_103a) Fourier-domain dedispersion library.
 *
 * Fourier-domain dedispersion (FDD; Bassa et al., arXiv 2110.03482) replaces
 * the per-channel time shifts of brute-force dedispersion (Sect. 2.1, Eq. 2)
 * by phase rotations of each channel's Fourier transform (Sect. 2.2):
 *
 *   X[nu][k]  = sum_n x_nu[n] exp(-2 pi i k n / L)                  (Eq. 3)
 *   d(nu, DM) = DM k_DM (nu^-2 - nu_ref^-2) / t_samp  [samples]      (Eq. 1)
 *   Y[DM][k]  = sum_nu exp(+2 pi i k d(nu, DM) / L) X[nu][k]          (Eqs. 4, 7)
 *   y[DM][n]  = (1/L) inverse real transform of Y[DM][.]             (Eq. 6)
 *
 * The phasor sign is the one that ADVANCES low channels so that a dispersed
 * pulse lines up at its arrival time at nu_ref (the discard rule of Sect. 2.2
 * puts the wrapped-around samples at the end of each series).
 *
 * Conventions for every entry point:
 *  - Pointers named d_* are device pointers (memory of the current CUDA
 *    device); h_* are host pointers.  The caller owns every buffer it passes
 *    and the stream; the plan owns its workspace, its FFT plans and tables.
 *  - Streams are CUDA runtime streams (cudaStream_t); NULL means the legacy
 *    default stream.  Execute calls are asynchronous on that stream, launch
 *    only, never synchronise and never allocate.
 *  - Every call returns an fdd_status.  Nothing aborts.  On failure a message
 *    is kept per thread and returned by fdd_last_error().
 *  - A plan must not be executed concurrently from two streams or threads.
 *  - All complex data are interleaved single-precision (re, im) pairs.
 */
#ifndef FDD_H_
#define FDD_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FDD_ABI_VERSION 2

struct CUstream_st;
typedef struct CUstream_st* fdd_stream_t; /* same type as cudaStream_t */

typedef struct fdd_plan_s* fdd_plan_t;

typedef enum fdd_status {
  FDD_OK = 0,
  FDD_ERR_INVALID_ARG = 1, /* a parameter or pointer is out of its domain   */
  FDD_ERR_UNSUPPORTED = 2, /* valid, but not implemented by this library    */
  FDD_ERR_ALLOC = 3,       /* device or host allocation failed (plan time)  */
  FDD_ERR_CUDA = 4,        /* a CUDA runtime call failed                    */
  FDD_ERR_CUFFT = 5,       /* a cuFFT call failed                           */
  FDD_ERR_TIMEOUT = 6,     /* a bounded device-side wait gave up            */
  FDD_ERR_DEVICE = 7       /* a kernel reported an error in its status word */
} fdd_status;

/* fdd_params.in_dtype: sample type of the input dynamic spectrum (Sect. 3:
 * packed 8-bit data; float32 also accepted). */
#define FDD_IN_U8 0
#define FDD_IN_F32 1

/* fdd_params.in_layout */
#define FDD_LAYOUT_TIME_MAJOR 0 /* [beam][n_t][n_chan], filterbank order (Sect. 3) */
#define FDD_LAYOUT_CHAN_MAJOR 1 /* [beam][n_chan][n_t]                              */

/* fdd_params.output */
#define FDD_OUT_TIME 0    /* float  [beam][n_dm][out_len]: back to time (Eq. 6) */
#define FDD_OUT_SPECTRA 1 /* complex[beam][chunk][n_dm][n_bins]: Y of Eq. 7     */
#define FDD_OUT_POWER 2   /* float  [beam][chunk][n_dm][n_bins]: |Y|^2 for
                             periodicity searches (Sect. 5)                     */

/* Kernel tiles of the FP32 phase-rotate-and-sum (fdd_params.mac_variant - 1,
 * fdd_info.mac_variant).  All issue paired f32x2 FMAs on an A x B register
 * tile per lane (a warp covers 2048, 1024, 4 x 512 or 4 x 128 trials of its
 * bins); W12 and G12 split phasor evaluation (4 warps) from the
 * multiply-accumulates (8 warps), the others let every warp do both.  With
 * mac_variant 0 a plan takes the tile with the least time for its trial
 * count whose shared memory holds the channels' phase table: G12_4X8 from
 * 257 trials, Q_4X4 below; above 8381 channels G12_4X8 no longer fits and
 * the fastest of the others that do is taken. */
#define FDD_MAC_W12_8X8 0   /* warp-specialised, 2048-trial blocks, four real
                               products per complex MAC                         */
#define FDD_MAC_Q12_8X8 1   /* 2048-trial blocks, 12 warps, plain schedule       */
#define FDD_MAC_Q_4X8 2     /* 1024-trial blocks                                 */
#define FDD_MAC_Q_8X8_512 3 /* 8x8 lane tile, 8 lanes per bin, four bins per
                               warp: 512-trial blocks                           */
#define FDD_MAC_Q_4X4 4     /* 4x4 lane tile, four bins per warp: 128-trial
                               blocks (small trial counts, ragged tails)        */
#define FDD_MAC_G12_4X8 5   /* warp-specialised, 2048-trial blocks, three real
                               products per complex MAC (Gauss's form): 4 phasor
                               warps feed 8 MAC warps, two per bin; a last block
                               of <= 1024 / <= 512 trials runs as wide items of
                               8 / 16 bins (default from 257 trials)            */
#define FDD_MAC_VARIANTS 6
#define FDD_MAC_TC 100      /* fdd_info.mac_variant of the tensor-core form: one
                               CTA per SM, a pass over the channels covering
                               1024 trials with more than 16 beams, else 2048   */
#define FDD_MAC_TC_PAIR 101 /* the same on pairs of CTAs (two SMs, one MMA of
                               M = 256, T = 256), each building half of the data
                               operand; a pass covers 2048 trials with more than
                               16 beams, else 4096.  Plans whose calls end in a
                               pass of this form that is full or more than half
                               full take it: time output only in DM batches of
                               whole passes, spectra and power only while an
                               output block of one pass fits a quarter of
                               workspace_limit                                 */

/* fdd_params.precision */
#define FDD_PREC_FP32 0      /* FP32 phasors and accumulation (CUDA cores)       */
#define FDD_PREC_BF16_HILO 1 /* tensor cores (tcgen05), the direction of Sect. 5:
                                BF16 hi+lo phasors, BF16 data, FP32 accumulation;
                                all beams of a chunk share each bin's phasors    */
#define FDD_PREC_BF16 2      /* the same with BF16 phasors only (half the tensor
                                work of hi+lo, larger error)                     */
#define FDD_PREC_FP16 3      /* tensor cores with FP16 phasors and FP16 data, each
                                bin's data scaled by a power of two into FP16's
                                range (the tensor work of BF16, smaller error)   */
#define FDD_PREC_FP8 4       /* tensor cores with FP8 E4M3 phasors and data (the
                                8-bit direction of Sect. 5), per-bin data scaling
                                as FP16, 64 channels per K stage; three mantissa
                                bits give a relative error of a few percent, far
                                above the 16-bit forms (measured, opt-in)        */

typedef struct fdd_params {
  int32_t n_chan;         /* observing channels N_nu, >= 1                          */
  int32_t n_beams;        /* independent beams sharing the setup, >= 1              */
  double nu_lo_mhz;       /* centre frequency of channel 0, MHz, > 0                */
  double dnu_mhz;         /* channel spacing, MHz, nonzero, may be negative         */
  double t_samp_s;        /* sampling time, s, > 0                                  */
  int64_t n_t;            /* samples per channel and beam, >= 2                     */
  const double* dm_list;  /* host array of n_dm trial DMs (pc cm^-3), >= 0; copied  */
  int32_t n_dm;           /* number of trial DMs, >= 1                              */
  int32_t in_dtype;       /* FDD_IN_U8 | FDD_IN_F32                                  */
  int64_t chunk_len;      /* 0: whole series zero padded to a power of two (Sect. 3);
                             L > 0: overlap-save chunks of L samples, even          */
  double k_dm;            /* dispersion constant, MHz^2 pc^-1 cm^3 s; 0 selects the
                             paper's (2.41e-4)^-1 (Sect. 2.1)                       */
  double nu_ref_mhz;      /* reference frequency nu_0 of Eq. 1; 0 selects the
                             highest channel centre; must be >= every channel centre */
  int32_t in_layout;      /* FDD_LAYOUT_*                                            */
  int32_t output;         /* FDD_OUT_*                                               */
  int32_t precision;      /* FDD_PREC_*                                              */
  int32_t mac_variant;    /* phase-rotate-and-sum kernel: 0 chooses automatically;
                             1 + FDD_MAC_* forces that variant                      */
  size_t workspace_limit; /* device bytes the plan may hold; 0 = library default    */
  int32_t downsample;     /* FDD_OUT_TIME: shorten the inverse transform by this
                             power-of-two factor f (0 or 1: none; Sect. 2.2, last
                             paragraph): only the bins k <= L/(2f) are dedispersed
                             and inverted with length L/f, scaled by 1/L, giving
                             the series low-passed to those bins and sampled every
                             f native samples; with chunking the hop is rounded
                             down to a multiple of f.  L must be divisible by 2f. */
  int32_t spin_group;     /* tensor-core form, one beam: 0 (off), 16 or 32 -- the
                             spin-frequency-dependent DM grids of Sect. 2.3
                             (Eqs. 8, 9): bins from k_min on are taken in groups of
                             this many consecutive bins that share the phasors of
                             their highest bin k_ref, i.e. bin k is dedispersed at
                             the DMs DM_j k_ref / k, and is then re-sampled to the
                             plan's trials by linear interpolation along the
                             trial axis.  An approximation: its error against
                             Eq. 7 grows with the DM step and the bin.          */
  double spin_tol;        /* largest relative DM contraction 1 - k / k_ref within a
                             group (0: 0.01); bins below k_min = max(1,
                             ceil((spin_group - 1) / spin_tol)) follow Eq. 7 exactly */
} fdd_params;

typedef struct fdd_info {
  int64_t fft_len;         /* L, transform length                                  */
  int64_t n_bins;          /* L/2 + 1                                              */
  int64_t bin_pitch;       /* complex elements between spectra rows in workspace   */
  int64_t n_chunks;        /* chunks per beam                                      */
  int64_t hop;             /* output samples kept per chunk                        */
  int64_t d_max;           /* ceil(largest delay) in samples (Sect. 2.2)           */
  int64_t out_len;         /* time samples per DM in FDD_OUT_TIME output (down-
                              sampled: ceil of the native count / downsample)        */
  int64_t valid_len;       /* leading output samples free of wrap-around           */
  int64_t in_elems;        /* elements of the input buffer                         */
  int64_t out_elems;       /* elements (float or complex) of a full output buffer  */
  int64_t out_bytes;       /* bytes of a full output buffer                        */
  int64_t workspace_bytes; /* device bytes held by the plan                        */
  double dm0;              /* first trial DM                                       */
  double ddm;              /* DM step of the (uniform) trial list                  */
  int32_t dm_uniform;      /* 1 when the list is an arithmetic progression         */
  int32_t dm_batch;        /* trials per internal batch (bounded by workspace)     */
  int32_t mac_variant;     /* phasor-MAC kernel chosen for this plan: an FP32 tile
                              (FDD_MAC_*) or FDD_MAC_TC / FDD_MAC_TC_PAIR         */
  int32_t downsample;      /* factor of the shortened inverse transform (1: none)    */
  int32_t block_dm;        /* trials per output block of the streamed calls        */
  int64_t stream_bytes;    /* device bytes the first streamed call adds to the plan
                              (two input windows and two output blocks)           */
  int32_t spin_group;      /* bins per group of the spin-frequency grids (0: off)  */
  int32_t spin_k_min;      /* first grouped bin                                    */
  int32_t spin_j_lo;       /* the scaled grid's first trial, relative to the plan's */
  int32_t spin_n_s;        /* trials of the scaled grid                            */
} fdd_info;

/* ABI version of the loaded library (FDD_ABI_VERSION at build time). */
int32_t fdd_abi_version(void);

/* Human-readable name of a status code.  Never NULL. */
const char* fdd_status_string(fdd_status s);

/* Last error message of the calling thread ("" if none).  Never NULL; valid
 * until the next failing call on this thread. */
const char* fdd_last_error(void);

/* Fill *p with defaults: one beam, FP32, time-major u8 input, time output,
 * paper k_DM, nu_ref at the top channel, no chunking.  Sizes stay zero. */
void fdd_params_init(fdd_params* p);

/*
 * Host-only plan geometry (no CUDA call): validates *p and fills *out with
 * the transform length, chunking (hop, d_max, out_len), DM-grid description
 * and buffer sizes, exactly as fdd_plan would.  The chunking follows
 * Sect. 2.2 (discard the last Delta t_max samples) and Sect. 3 (zero pad to
 * a power of two): chunk_len == 0 gives one circular transform of
 * L = next power of two >= n_t and out_len = n_t, of which the first
 * valid_len = n_t - d_max are free of wrap-around; chunk_len == L gives
 * hop = L - d_max, out_len = n_t - d_max and ceil(out_len / hop) chunks.
 * Errors: FDD_ERR_INVALID_ARG (bad parameter), FDD_ERR_UNSUPPORTED.
 */
fdd_status fdd_plan_geometry(const fdd_params* p, fdd_info* out);

/*
 * Create a plan on the current CUDA device (Algorithm 1, initialisation:
 * delay table, spin-frequency grid, FFT plans, device buffers).  Computes in
 * FP64 the per-channel delay rate of Eq. 1 and, for a uniform DM list, the
 * exact 64-bit fixed-point phase rates used by the kernels.  Allocates all
 * device workspace here; execute calls never allocate.  Any DM list makes a
 * plan; the Fourier-domain calls need a uniform one (fdd_info.dm_uniform),
 * the time-domain call takes any.
 * Errors: FDD_ERR_INVALID_ARG, FDD_ERR_UNSUPPORTED (unsupported precision or
 * sizes), FDD_ERR_ALLOC, FDD_ERR_CUDA, FDD_ERR_CUFFT.
 * On error *out is set to NULL and nothing is leaked.
 */
fdd_status fdd_plan(const fdd_params* p, fdd_plan_t* out);

/* Copy the plan's geometry into *out.  Also reports (FDD_ERR_DEVICE or
 * FDD_ERR_TIMEOUT) a status word left by an earlier kernel, once: reading it
 * clears it.  This call synchronises the plan's status read with the device. */
fdd_status fdd_query(fdd_plan_t plan, fdd_info* out);

/*
 * Whole path for every trial DM (Algorithm 1 on device-resident data):
 * unpack and transpose the input to channel-major float, zero pad / cut the
 * overlap-save chunks, forward real FFT per channel (Eq. 3), phase-rotate-
 * and-sum over channels (Eqs. 4, 7), then per the plan's output either the
 * inverse real FFT scaled by 1/L with the valid samples of each chunk placed
 * in order (Eq. 6), the spectra Y, or |Y|^2.
 *   d_in : input, layout and type per the plan, info.in_elems elements.
 *   d_out: output, info.out_elems elements of the output type:
 *          TIME    float [beam][n_dm][out_len]
 *          SPECTRA complex float [beam][chunk][n_dm][n_bins]
 *          POWER   float [beam][chunk][n_dm][n_bins]
 * Asynchronous on `stream`; never synchronises or allocates, so with
 * profiling off a caller may capture the call into a CUDA graph and replay it
 * (the graph keeps d_in and d_out).
 * Errors: FDD_ERR_INVALID_ARG (NULL plan or pointer), FDD_ERR_CUDA,
 * FDD_ERR_CUFFT.
 */
fdd_status fdd_execute(fdd_plan_t plan, const void* d_in, void* d_out, fdd_stream_t stream);

/*
 * The same for the trial DMs dm_first .. dm_first + n_dm - 1 only (the
 * DM-outer batching of Sect. 3 / Algorithm 1).  d_out has the layout of
 * fdd_execute with n_dm in place of the plan's trial count.
 * Errors: as fdd_execute; FDD_ERR_INVALID_ARG for a range outside the list.
 */
fdd_status fdd_execute_dm_range(fdd_plan_t plan, const void* d_in, int32_t dm_first,
                                int32_t n_dm, void* d_out, fdd_stream_t stream);

/*
 * Streaming: inputs and outputs larger than device memory (Algorithm 1's
 * per-chunk copies and DM-outer batches, Sect. 3).  The path runs chunk by
 * chunk; each (beam, chunk) input window passes through a plan-owned ring of
 * two windows, and the output leaves in blocks through a ring of two output
 * blocks, so no device buffer is sized by the whole input or output.
 *
 * A source fills one input window: samples t_begin .. t_begin + n_samples - 1
 * (n_samples <= fdd_info.fft_len) of beam `beam`, into d_window, in the
 * plan's input type and layout restricted to those samples ([n_samples]
 * [n_chan] time-major, or [n_chan][n_samples] channel-major).  The window's
 * previous contents may still be read by work queued on `stream` before the
 * call: work on another stream that writes the window must first wait for
 * `ready_event` (a cudaEvent_t; NULL when the slot is new).  The source must
 * order its writes before later work on `stream` (enqueue them there, or make
 * the stream wait for them).  It returns FDD_OK, or a status that ends the
 * call.
 *
 * A sink receives one output block (its d_data is device memory of the plan):
 *   FDD_OUT_TIME:    [n_dm][row_pitch] float for one beam (n_beams 1); row r
 *                    holds samples out_offset .. out_offset + row_len - 1 of
 *                    trial dm_first + r (the kept samples of this chunk, 1/L
 *                    scaled; down-sampled when the plan down-samples);
 *   FDD_OUT_SPECTRA / FDD_OUT_POWER: [n_beams][n_dm][n_bins] complex / float
 *                    of chunk `chunk` (row_len = row_pitch = n_bins,
 *                    out_offset 0), for beams beam_first .. + n_beams - 1.
 * The block is complete for work enqueued on `stream` after the sink is
 * called.  Its slot is rewritten two blocks later: a sink that reads it on
 * `stream` needs nothing more; one that reads it on another stream stores in
 * release_event a cudaEvent_t recorded after those reads, and the library
 * makes `stream` wait for it before rewriting the slot.  Blocks come
 * chunk-outer for the tensor-core form, beam-outer for the FP32 form; within
 * a (beam, chunk) in increasing trial order.
 */
typedef struct fdd_block {
  int32_t beam_first;  /* first beam of the block                                   */
  int32_t n_beams;     /* beams in the block                                        */
  int64_t chunk;       /* chunk index                                               */
  int32_t dm_first;    /* first trial of the block (index into the DM list)         */
  int32_t n_dm;        /* trials in the block                                       */
  const void* d_data;  /* the block (device memory owned by the plan)               */
  int64_t row_len;     /* valid elements per (beam, trial) row                      */
  int64_t row_pitch;   /* elements between consecutive rows                         */
  int64_t out_offset;  /* FDD_OUT_TIME: sample index of row element 0 in the whole
                          output row; 0 otherwise                                    */
  void* release_event; /* set by the sink (optional): see above; NULL on entry      */
} fdd_block;

typedef fdd_status (*fdd_source_fn)(void* user, int32_t beam, int64_t t_begin,
                                    int64_t n_samples, void* d_window, void* ready_event,
                                    fdd_stream_t stream);
typedef fdd_status (*fdd_sink_fn)(void* user, fdd_block* block, fdd_stream_t stream);

/*
 * The whole path for every trial DM with streamed output, and input either
 * resident on the device (d_in, layout of fdd_execute; source NULL) or
 * streamed from a source (d_in NULL): the source is called once per (beam,
 * chunk) window, the sink once per output block; the computation is that of
 * fdd_execute.  Both callbacks run on the calling thread, inside this call.
 * The first call allocates the rings (fdd_info.stream_bytes); later calls
 * reuse them.  Asynchronous on `stream` apart from what the callbacks do.
 * Errors: as fdd_execute; FDD_ERR_INVALID_ARG (NULL sink, or not exactly one
 * of d_in and source); FDD_ERR_ALLOC on the first call; a callback's own
 * status.
 */
fdd_status fdd_execute_stream(fdd_plan_t plan, const void* d_in, fdd_source_fn source,
                              void* source_user, fdd_sink_fn sink, void* sink_user,
                              fdd_stream_t stream);

/*
 * End-to-end call with HOST buffers: h_in (layout of fdd_execute's d_in) to
 * the device, the path, and the result back into h_out (layout of d_out),
 * streamed as fdd_execute_stream streams: each (beam, chunk) input window
 * goes up on a plan-owned copy stream into the window ring, and each output
 * block comes back on a second copy stream, so copies overlap the
 * computation of the neighbouring windows and blocks and the device holds
 * only the two rings, whatever the sizes of h_in and h_out.  Events order the
 * copy streams with `stream`: they start after the work already queued on
 * it, and `stream` waits for the last copy, so synchronising `stream` covers
 * the whole call.  Page-locked host buffers make the copies asynchronous
 * (the call returns after enqueueing); both buffers must stay valid until
 * then.  The rings, copy streams and events are created on the first
 * streamed call for the plan and reused.
 * Errors: as fdd_execute, plus FDD_ERR_ALLOC on the first call.
 */
fdd_status fdd_execute_host(fdd_plan_t plan, const void* h_in, void* h_out, fdd_stream_t stream);

/*
 * The hot path alone: phase-rotate-and-sum (Eqs. 4, 7) of given spectra.
 *   d_X      : complex float [n_series][n_chan][x_pitch], bins 0 .. n_bins-1
 *              of each row used (n_bins from the plan; x_pitch >= n_bins).
 *   n_series : independent spectra sets (beams x chunks), >= 1.
 *   dm_first, n_dm : trial range of the plan's DM list.
 *   d_Y      : out_kind FDD_OUT_SPECTRA: complex float [n_series][n_dm][y_pitch];
 *              out_kind FDD_OUT_POWER:   float [n_series][n_dm][y_pitch] (|Y|^2).
 * No scaling is applied (Y is the plain sum of Eq. 7).
 * Errors: FDD_ERR_INVALID_ARG, FDD_ERR_CUDA.
 */
fdd_status fdd_dedisperse_spectra(fdd_plan_t plan, const void* d_X, int64_t x_pitch,
                                  int32_t n_series, int32_t dm_first, int32_t n_dm,
                                  void* d_Y, int64_t y_pitch, int32_t out_kind,
                                  fdd_stream_t stream);

/*
 * The hot path on a window of bins: bins bin_first .. bin_first + n_bins - 1
 * of the plan's transform (Eqs. 4, 7 with k the absolute bin index).  Bins
 * are independent through the phase-rotate-and-sum, so a window is the unit
 * for splitting bins across calls, streams or devices, and for checking
 * chosen bins of a full-size transform.
 *   d_X      : complex float [n_series][n_chan][x_pitch]; element i of a row
 *              is bin bin_first + i (x_pitch >= n_bins).
 *   bin_first, n_bins : the window, inside [0, plan n_bins).
 *   d_Y      : as fdd_dedisperse_spectra, element i of a row = bin bin_first + i
 *              (y_pitch >= n_bins).
 * The other arguments, ownership and errors are those of
 * fdd_dedisperse_spectra; FDD_ERR_INVALID_ARG also for a window outside the
 * plan's bins.  fdd_dedisperse_spectra is this call with the whole range.
 */
fdd_status fdd_dedisperse_spectra_bins(fdd_plan_t plan, const void* d_X, int64_t x_pitch,
                                       int32_t n_series, int32_t bin_first, int32_t n_bins,
                                       int32_t dm_first, int32_t n_dm, void* d_Y,
                                       int64_t y_pitch, int32_t out_kind,
                                       fdd_stream_t stream);

/*
 * Brute-force time-domain dedispersion (Eq. 2), the method the paper
 * measures Fourier-domain dedispersion against (Sect. 4), with the plan's
 * channels, sampling time, k_DM, reference frequency and DM list (any list:
 * uniform or not):
 *   y[beam][j][n] = sum_nu x[beam][nu][n + s[j][nu]],  n < n_t - d_max,
 * where s[j][nu] is the delay of Eq. 1 in samples, computed in FP64 and
 * rounded to the nearest sample (halves away from zero), and d_max is
 * fdd_info.d_max (ceil of the largest delay), so every sample read exists.
 *   d_in  : as fdd_execute (u8 or f32, either layout, n_beams beams).
 *   d_out : float [n_beams][n_dm][n_t - d_max].
 * The first call builds the shift tables and a channel-major copy of one
 * beam (n_chan x n_t floats) in plan memory; later calls reuse them.
 * Asynchronous on the stream.  Errors: FDD_ERR_INVALID_ARG (NULL pointers,
 * n_t <= d_max), FDD_ERR_UNSUPPORTED (a block of 32 trials spans more than
 * ~3300 samples of delay in one channel, or more than 2^24 output samples),
 * FDD_ERR_ALLOC, FDD_ERR_CUDA.
 */
fdd_status fdd_tdd_execute(fdd_plan_t plan, const void* d_in, void* d_out, fdd_stream_t stream);

/*
 * Failure-detection self-tests (no counterpart in the paper).  Nothing here
 * faults or hangs a GPU: every wait in the kernels is bounded (about 2 s of
 * SM clock), after which the kernel records FDD_ERR_TIMEOUT in the plan's
 * status word, releases what it holds and returns.
 *
 * fdd_debug_stall_test runs the plan's waiting phase-rotate-and-sum kernel
 * (the warp-specialised FP32 tile, or the tensor-core kernel) on one bin,
 * one trial and one series, with its producers withholding every "stage
 * filled" arrival, so the consumers' waits run out.  It blocks until the
 * kernel has returned (about 2 s); the next fdd_query then reports
 * FDD_ERR_TIMEOUT once (reading a device status clears it), and the plan
 * stays usable.  Errors: FDD_ERR_INVALID_ARG, FDD_ERR_CUDA.
 *
 * fdd_debug_fail_alloc makes the library's device allocations after the
 * next `after` ones fail once with FDD_ERR_ALLOC (plans and batch plans
 * release what they hold and report it); after < 0 turns it off.  Process
 * wide.  Always FDD_OK.
 */
fdd_status fdd_debug_stall_test(fdd_plan_t plan, fdd_stream_t stream);
fdd_status fdd_debug_fail_alloc(int32_t after);

/* Stages of the path timed by the profiling calls below. */
#define FDD_STAGE_UNPACK 0  /* transpose_and_unpack + zero_pad (Algorithm 1)   */
#define FDD_STAGE_R2C 1     /* channel transforms, Eq. 3 (cuFFT)                */
#define FDD_STAGE_MAC 2     /* phase-rotate-and-sum, Eqs. 4 and 7               */
#define FDD_STAGE_C2R 3     /* inverse transforms, Eq. 6 (cuFFT)                */
#define FDD_STAGE_SCATTER 4 /* 1/L scaling and valid-sample placement           */
#define FDD_STAGE_TDD 5     /* brute-force time-domain shift-and-sum (Eq. 2)    */
#define FDD_STAGE_TRANSPOSE 6 /* tensor-core form: spectra to bin-major, and each
                                 beam's output back to bins innermost            */
#define FDD_STAGE_COUNT 7

typedef struct fdd_profile {
  int64_t launches[FDD_STAGE_COUNT]; /* timed launches per stage               */
  double ms[FDD_STAGE_COUNT];        /* summed device time per stage, ms        */
  int64_t dropped;                   /* launches not timed (event ring full)    */
  int64_t kernels;                   /* kernels of this library launched since
                                        profiling was enabled on this plan (all
                                        plans and threads of the process)        */
} fdd_profile;

/*
 * Profiling (no counterpart in the paper beyond its per-component runtime
 * breakdown, Sect. 4.1): when enabled, execute calls record a CUDA event pair
 * on the launching stream around every stage launch.  on != 0 creates the
 * events (host-side, at this call), clears the counters and starts
 * recording; on == 0 stops recording.  Up to 8192 launches are kept per
 * reset; later ones are counted as dropped.
 * Errors: FDD_ERR_INVALID_ARG, FDD_ERR_CUDA.
 */
fdd_status fdd_profile_enable(fdd_plan_t plan, int32_t on);

/* Sum the recorded event pairs into *out.  Waits for the last recorded event
 * (host synchronisation), so call it outside timed regions.
 * Errors: FDD_ERR_INVALID_ARG, FDD_ERR_CUDA. */
fdd_status fdd_profile_read(fdd_plan_t plan, fdd_profile* out);

/* ------------------------------------------------------------------------
 * Batching form: many beams of uneven length and uneven trial grids (the
 * batch dimensions of Sect. 3 / Algorithm 1, and the autotuning suggested in
 * Sect. 5).  Every beam shares the channel set, sampling time, k_DM, nu_ref,
 * input type and layout of the common parameters; each has its own series
 * length, uniform trial grid and chunk length: a beam is transformed whole
 * (L = next power of two >= n_t, as chunk_len 0) or in overlap-save chunks
 * of its own length (Sect. 2.2, as a plan with that chunk_len), and the
 * batch emits spectra or |Y|^2 (output FDD_OUT_SPECTRA or FDD_OUT_POWER),
 * in the FP32 form or on tensor cores (Sect. 5: beams that share their
 * phasors make each bin a GEMM).
 * ---------------------------------------------------------------------- */
typedef struct fdd_beam_desc {
  int64_t n_t;       /* samples of this beam, >= 2                                  */
  double dm0;        /* first trial DM (pc cm^-3), >= 0                             */
  double ddm;        /* trial step, >= 0                                            */
  int32_t n_dm;      /* trials, >= 1                                                */
  int32_t chunk_len; /* 0: one transform of the whole series; else the overlap-save
                        chunk length of this beam, a power of two above its largest
                        delay (fdd_params.chunk_len's rules)                          */
} fdd_beam_desc;

typedef struct fdd_batch_s* fdd_batch_t;

typedef struct fdd_batch_info {
  int64_t in_elems;        /* elements of the concatenated input                 */
  int64_t out_elems;       /* elements of the concatenated output                */
  int64_t out_bytes;
  int64_t workspace_bytes; /* device bytes held by the batch plan                */
  int64_t work_items;      /* (beam, chunk, bin tile, trial block) items per
                              execute, tail items included                       */
  int32_t n_waves;         /* waves (one or two persistent launches each)        */
  int32_t mac_variant;     /* kernel tile in use (FDD_MAC_*)                     */
  int32_t ctas;            /* CTAs of each persistent launch of that tile        */
  int32_t tail_variant;    /* tile of the ragged last trial blocks (FDD_MAC_*), or
                              -1 (none).  With the W12_8X8 tile a beam's last
                              block of 1024 or fewer trials runs in a second
                              persistent launch on this tile's 128-trial blocks;
                              the G12_4X8 tile runs such a block in its own
                              launch as wide items (eight bins x 1024 trials)  */
  double autotune_ms[FDD_MAC_VARIANTS]; /* timed candidates (ms), -1 if untimed */
} fdd_batch_info;

/*
 * Plan a batch.  *p supplies the common fields (n_chan, nu_lo_mhz, dnu_mhz,
 * t_samp_s, k_dm, nu_ref_mhz, in_dtype, in_layout, output, precision,
 * workspace_limit, mac_variant); its n_t, dm_list, n_dm, n_beams are not
 * read and chunk_len must be 0 (each beam gives its own).  beams[0 ..
 * n_beams-1] describe the beams.  Beams are grouped in order into waves
 * whose spectra (n_chunks x n_chan x (L/2+1 rounded up to 64) complex each)
 * fit in workspace_limit (default 16 GiB) minus the
 * fixed part (n_chan x max L floats of staging, the phase tables and a
 * 64 MiB reserve for the FFT work area);
 * each wave is one persistent launch of the phase-rotate-and-sum whose CTAs
 * take (beam, chunk, bin tile, trial block) work items from a counter.  With
 * mac_variant 0 and autotune != 0 the candidate kernel tiles are timed on the
 * batch's own shapes and the fastest is kept (remembered per shape in the
 * process, and in the text file named by the FDD_AUTOTUNE_CACHE environment
 * variable when set); mac_variant 0 without autotune selects G12_4X8.
 * With a tensor-core precision (FDD_PREC_BF16_HILO .. FDD_PREC_FP8) the
 * beams are grouped by what their phasors share: whole-series beams by
 * transform length and trial grid origin and step, chunked beams also by
 * chunk length and trial count (which set the overlap); each group, sorted
 * by trial count and cut into plans of up to 16 beams (fewer where such a
 * plan, with its streaming rings, would exceed workspace_limit), runs as one
 * tensor-core plan (fdd_plan with that precision) over its largest series
 * and trial count, shorter beams reading zeros beyond their samples and
 * keeping their own trials and chunks.  The plans are made here, each with
 * its own workspace when those fit workspace_limit together, else all
 * taking their per-call buffers (spectra, scratch, FFT work area, streaming
 * rings) from one shared device block of the largest plan's size, which
 * works because they run one after another; if even that block cannot be
 * had, each execute makes each plan for its turn and destroys it after.
 * fdd_batch_info then gives mac_variant FDD_MAC_TC and n_waves the number of
 * plans.
 * Allocates all device memory (and, while autotuning, a temporary output).
 * Layouts: the input is the beams' inputs concatenated in order (each
 * [n_t][n_chan] or [n_chan][n_t]); the output is, per beam in order,
 * [n_chunks][n_dm][L/2+1] complex (spectra) or float (power), with n_chunks
 * and L those fdd_plan_geometry gives for the beam's n_t and chunk_len
 * (n_chunks 1 for a whole series); fdd_batch_query gives the offsets.
 * Errors: FDD_ERR_INVALID_ARG, FDD_ERR_UNSUPPORTED (time output,
 * fdd_params.chunk_len != 0, a tile without batched form), FDD_ERR_ALLOC,
 * FDD_ERR_CUDA, FDD_ERR_CUFFT.
 */
fdd_status fdd_batch_plan(const fdd_params* p, const fdd_beam_desc* beams, int32_t n_beams,
                          int32_t autotune, fdd_batch_t* out);

/* Sizes, waves, chosen tile and autotune timings; in_offsets / out_offsets
 * (arrays of n_beams, or NULL) receive each beam's element offset in the
 * concatenated input / output.  Waits for the device; returns
 * FDD_ERR_TIMEOUT (once, with *info filled) when a device-side wait of an
 * execute since the last query timed out (its output is incomplete). */
fdd_status fdd_batch_query(fdd_batch_t b, fdd_batch_info* info, int64_t* in_offsets,
                           int64_t* out_offsets);

/*
 * Execute the batch: unpack and transform every beam (Eq. 3), then the
 * phase-rotate-and-sum (Eqs. 4, 7) of each wave in one persistent launch.
 * The sequence is captured once as a CUDA graph for a given (d_in, d_out)
 * pair and replayed on the stream by later calls with the same buffers; a
 * call with other buffers re-captures (synchronising the stream first).
 * The tensor-core batch runs its plans streamed instead (fdd_execute_stream,
 * windows copied from d_in, blocks copied into d_out), not as a graph; with
 * plans made per execute it waits for the device after each.
 * Errors: FDD_ERR_INVALID_ARG, FDD_ERR_ALLOC (plans made per execute),
 * FDD_ERR_CUDA, FDD_ERR_CUFFT.
 */
fdd_status fdd_batch_execute(fdd_batch_t b, const void* d_in, void* d_out, fdd_stream_t stream);

/*
 * Execute the batch streamed (fdd_execute_stream's callbacks and contracts):
 * the source fills one window per beam (t_begin 0, the beam's n_t samples,
 * the common layout) through a ring of two windows of the longest beam, so
 * the concatenated input never has to be on the device; per wave the
 * persistent launch writes into one of two output slots of the wave's size,
 * and the sink receives one block per beam and chunk (n_beams 1, the chunk
 * index, dm_first 0, the beam's n_dm trials x n_bins, row_len = row_pitch =
 * n_bins).  A sink
 * that reads a wave's blocks on another stream returns a release event for
 * its last block of the wave (an event recorded after all of them).  The
 * first call allocates the rings and binds the work sets to them.  Not
 * captured as a graph.  The tensor-core batch (time-major input only) calls
 * the source per (beam, chunk) window of its plans (t_begin, n_samples within
 * the beam's own samples) and the sink per (beam, chunk, block of trials) in
 * each plan's block order (the blocks of one plan block — same chunk and
 * first trial, consecutive beams — come one after another); a sink reading
 * on another stream may return a release event with any block, recorded
 * after its reads of every block handed over so far: the last one returned
 * within a plan block guards that plan block's device memory.  Errors:
 * FDD_ERR_INVALID_ARG, FDD_ERR_ALLOC (first
 * call), FDD_ERR_UNSUPPORTED (tensor-core batch with channel-major input),
 * FDD_ERR_CUDA, FDD_ERR_CUFFT, a callback's own status.
 */
fdd_status fdd_batch_execute_stream(fdd_batch_t b, fdd_source_fn source, void* source_user,
                                    fdd_sink_fn sink, void* sink_user, fdd_stream_t stream);

/* Release the batch plan (synchronises the device first).  NULL is ignored. */
fdd_status fdd_batch_destroy(fdd_batch_t b);

/* Largest channel count accepted by fdd_dedisperse_spectra_static. */
#define FDD_STATIC_MAX_CHAN 8192

/*
 * Phase-rotate-and-sum for callers that cannot allocate device memory (the
 * paper has no counterpart: this entry point exists for such callers).
 * Applications that hand all of a GPU's memory to their own pool, or
 * real-time pipelines that forbid allocation once running, cannot create a
 * plan, because fdd_plan allocates workspace.  This call takes the plan
 * parameters *p directly (the fields that the phase-rotate-and-sum uses --
 * channels, frequencies, t_samp, n_t and chunk_len for the transform length,
 * the DM list, k_dm, nu_ref -- are checked exactly as fdd_plan checks them;
 * precision must be FDD_PREC_FP32) and computes bit for bit what
 * fdd_dedisperse_spectra computes for a plan made from *p, with the same
 * arguments and layouts.  It allocates nothing, on the device or the host,
 * and calls no allocating library routine.  The per-channel phase table the
 * kernel reads lives in a file-scope device array of FDD_STATIC_MAX_CHAN
 * entries (128 KiB), which every GPU that loads the library holds until the
 * process exits; every call rewrites it, in stream order, with small kernel
 * launches that carry the constants in their parameters.  Calls share that
 * one array, so calls that overlap on the GPU (on different streams, or from
 * different threads) race and must be serialised by the caller; calls queued
 * on one stream are ordered and need nothing more.  The first call on each
 * device looks up the array's device address (a one-time set-up); make that
 * first call before any stream capture.  Without a plan there is no status
 * word: a bounded device-side wait that runs out (reported as FDD_ERR_TIMEOUT
 * by the planned calls) is not reported here, and the output is then
 * incomplete.
 * Errors: FDD_ERR_INVALID_ARG (NULL pointers, n_chan above
 * FDD_STATIC_MAX_CHAN, bad ranges or pitches, the parameter errors of
 * fdd_plan), FDD_ERR_UNSUPPORTED (non-uniform DM list, precision other than
 * FP32, transform length above 2^30), FDD_ERR_CUDA.
 */
fdd_status fdd_dedisperse_spectra_static(const fdd_params* p, const void* d_X, int64_t x_pitch,
                                         int32_t n_series, int32_t dm_first, int32_t n_dm,
                                         void* d_Y, int64_t y_pitch, int32_t out_kind,
                                         fdd_stream_t stream);

/* Release the plan and everything it owns (synchronises the device first).
 * NULL is accepted and ignored. */
fdd_status fdd_destroy(fdd_plan_t plan);

#ifdef __cplusplus
}
#endif

#endif /* FDD_H_ */

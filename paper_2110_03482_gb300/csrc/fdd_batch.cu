// fdd_batch.cu -- the batching form: many beams of uneven length and uneven
// trial grids dedispersed together (the batch dimensions of Sect. 3 /
// Algorithm 1 and the autotuning suggestion of Sect. 5).
//
// Beams are grouped into waves whose spectra fit the workspace.  For each
// wave the beams are unpacked and transformed one by one (one cuFFT plan per
// distinct transform length), then ONE persistent launch of the FP32
// phase-rotate-and-sum serves the whole wave: its CTAs pull (beam, bin tile,
// trial block) items from a counter.  The whole execute is captured once as a
// CUDA graph and replayed.  At plan time an autotuner times the candidate
// kernel tiles on the batch's real shapes and keeps the fastest.
#include <cufft.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <limits>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "fdd.h"
#include "fdd_internal.h"

struct fdd_batch_s {
  fdd_params p{};
  std::vector<fdd_beam_desc> beams;
  int device = -1;
  int n_sms = 0;
  int variant = 0;
  int ctas = 0;
  int tail_variant = -1;  // tile of the ragged last trial blocks, -1: none
  int tail_ctas = 0;
  double tune_ms[FDD_MAC_VARIANTS];
  // per beam
  std::vector<int64_t> L, n_bins, pitch, in_off, out_off, spec_off;
  std::vector<int> wave_of;
  // per wave
  struct Wave {
    int first = 0, count = 0;
    long long n_items = 0;
    fdd::BatchSet* d_sets = nullptr;
    std::vector<fdd::BatchSet> h_sets;
    // ragged last trial blocks of 1024 or fewer trials, on the tail tile
    long long n_tail_items = 0;
    fdd::BatchSet* d_tail = nullptr;
    std::vector<fdd::BatchSet> h_tail;
    std::vector<int> tail_beam;  // beam of each tail set
  };
  std::vector<Wave> waves;
  int64_t in_elems = 0, out_elems = 0;
  // device memory
  fdd::PhaseConst* d_pc = nullptr;  // [beam][n_chan]
  float* d_xw = nullptr;            // [n_chan][L_max]
  float2* d_pool = nullptr;         // spectra of one wave
  unsigned long long* d_counter = nullptr;  // one per wave
  void* d_fftwork = nullptr;
  size_t bytes_held = 0;
  std::map<int64_t, cufftHandle> r2c;  // by transform length
  // streamed execute (fdd_batch_execute_stream, made on its first call): two
  // input windows (the longest beam), and per wave two output slots (the
  // wave's whole output) with the work sets bound to each
  void* d_win[2] = {nullptr, nullptr};
  void* d_wout[2] = {nullptr, nullptr};
  size_t wout_bytes = 0;
  std::vector<fdd::BatchSet*> d_sets_slot[2];
  unsigned win_next = 0, out_next = 0;
  bool win_used[2] = {false, false};
  cudaEvent_t win_free[2] = {nullptr, nullptr};
  void* out_release[2] = {nullptr, nullptr};
  // CUDA graph of the whole execute, for the buffers it was captured with
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t graph = nullptr;
  const void* graph_in = nullptr;
  void* graph_out = nullptr;
};

namespace {

#define B_CUDA(call)                                                                    \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess) {                                                            \
      cudaGetLastError();                                                               \
      return fdd::report_error(FDD_ERR_CUDA, (std::string(#call) + ": " + cudaGetErrorString(e_)).c_str()); \
    }                                                                                   \
  } while (0)

#define B_CUFFT(call)                                                                   \
  do {                                                                                  \
    cufftResult r_ = (call);                                                            \
    if (r_ != CUFFT_SUCCESS)                                                            \
      return fdd::report_error(FDD_ERR_CUFFT, (std::string(#call) + " failed").c_str()); \
  } while (0)

void release(fdd_batch_s* B) {
  if (!B) return;
  if (B->graph) cudaGraphExecDestroy(B->graph);
  if (B->cap_stream) cudaStreamDestroy(B->cap_stream);
  for (auto& kv : B->r2c) cufftDestroy(kv.second);
  for (auto& w : B->waves) {
    if (w.d_sets) cudaFree(w.d_sets);
    if (w.d_tail) cudaFree(w.d_tail);
  }
  for (int k = 0; k < 2; ++k) {
    for (fdd::BatchSet* p : B->d_sets_slot[k])
      if (p) cudaFree(p);
    if (B->d_win[k]) cudaFree(B->d_win[k]);
    if (B->d_wout[k]) cudaFree(B->d_wout[k]);
    if (B->win_free[k]) cudaEventDestroy(B->win_free[k]);
  }
  void* ptrs[] = {B->d_pc, B->d_xw, B->d_pool, B->d_counter, B->d_fftwork};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  delete B;
}

fdd_status alloc(fdd_batch_s* B, void** p, size_t bytes) {
  if (fdd::injected_alloc_failure()) {
    *p = nullptr;
    return fdd::report_error(FDD_ERR_ALLOC, "injected allocation failure");
  }
  const cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return fdd::report_error(FDD_ERR_ALLOC, cudaGetErrorString(e));
  }
  B->bytes_held += bytes;
  return FDD_OK;
}

// Sets the output pointers of every work set for the given output buffer: a
// set's row 0 is trial j_begin of its beam.
// (`origin`: output element at d_out, nonzero for a buffer that holds only
// the beams from some beam on)
void bind_set(const fdd_batch_s* B, fdd::BatchSet& bs, int b, void* d_out, int64_t origin = 0) {
  fdd::MacArgs& m = bs.args;
  const int64_t off = B->out_off[b] - origin + static_cast<int64_t>(m.j_begin) * B->n_bins[b];
  if (B->p.output == FDD_OUT_SPECTRA)
    m.Y = static_cast<float2*>(d_out) + off;
  else
    m.Y = static_cast<float*>(d_out) + off;
}

void bind_output(fdd_batch_s* B, void* d_out) {
  for (auto& w : B->waves) {
    for (int i = 0; i < w.count; ++i) bind_set(B, w.h_sets[i], w.first + i, d_out);
    for (size_t i = 0; i < w.h_tail.size(); ++i) bind_set(B, w.h_tail[i], w.tail_beam[i], d_out);
  }
}

// All work of one execute, issued on stream s (also used under capture).
fdd_status issue(fdd_batch_s* B, const void* d_in, cudaStream_t s) {
  const size_t esz = B->p.in_dtype == FDD_IN_U8 ? 1 : 4;
  for (auto& kv : B->r2c) B_CUFFT(cufftSetStream(kv.second, s));
  for (size_t wi = 0; wi < B->waves.size(); ++wi) {
    const auto& w = B->waves[wi];
    for (int i = 0; i < w.count; ++i) {
      const int b = w.first + i;
      fdd::UnpackArgs ua{static_cast<const char*>(d_in) + esz * B->in_off[b], B->p.in_dtype,
                         B->p.in_layout, B->p.n_chan, B->beams[b].n_t, 0, B->L[b], B->d_xw,
                         B->L[b]};
      B_CUDA(fdd::launch_unpack(ua, s));
      B_CUFFT(cufftExecR2C(B->r2c.at(B->L[b]), B->d_xw,
                           reinterpret_cast<cufftComplex*>(B->d_pool + B->spec_off[b])));
    }
    B_CUDA(cudaMemsetAsync(B->d_counter + 2 * wi, 0, 2 * sizeof(unsigned long long), s));
    B_CUDA(fdd::launch_mac_batch(w.d_sets, w.count, w.n_items, B->d_counter + 2 * wi,
                                 B->variant, B->ctas, B->p.n_chan, s));
    if (w.n_tail_items)
      B_CUDA(fdd::launch_mac_batch(w.d_tail, static_cast<int>(w.h_tail.size()), w.n_tail_items,
                                   B->d_counter + 2 * wi + 1, B->tail_variant, B->tail_ctas,
                                   B->p.n_chan, s));
  }
  return FDD_OK;
}

fdd_status upload_wave(const fdd_batch_s::Wave& w, cudaStream_t s) {
  B_CUDA(cudaMemcpyAsync(w.d_sets, w.h_sets.data(), sizeof(fdd::BatchSet) * w.count,
                         cudaMemcpyHostToDevice, s));
  if (!w.h_tail.empty())
    B_CUDA(cudaMemcpyAsync(w.d_tail, w.h_tail.data(), sizeof(fdd::BatchSet) * w.h_tail.size(),
                           cudaMemcpyHostToDevice, s));
  return FDD_OK;
}

fdd_status upload_sets(fdd_batch_s* B, cudaStream_t s) {
  for (auto& w : B->waves) {
    fdd_status st = upload_wave(w, s);
    if (st != FDD_OK) return st;
  }
  return FDD_OK;
}

// Autotune cache: shape signature -> variant, in process and optionally in a
// text file named by FDD_AUTOTUNE_CACHE (one "signature variant" per line).
std::mutex g_tune_mutex;
std::map<std::string, int> g_tune_cache;

std::string signature(const fdd_batch_s* B) {
  std::string sig = "c" + std::to_string(B->p.n_chan) + "o" + std::to_string(B->p.output);
  for (size_t b = 0; b < B->beams.size(); ++b)
    sig += "|" + std::to_string(B->L[b]) + "x" + std::to_string(B->beams[b].n_dm);
  // keep the key short: hash the per-beam list
  unsigned long long h = 1469598103934665603ull;
  for (char c : sig) h = (h ^ static_cast<unsigned char>(c)) * 1099511628211ull;
  char buf[64];
  snprintf(buf, sizeof buf, "fdd-batch-%d-%zu-%016llx", B->p.n_chan, B->beams.size(), h);
  return buf;
}

int cache_lookup(const std::string& key) {
  std::lock_guard<std::mutex> lk(g_tune_mutex);
  auto it = g_tune_cache.find(key);
  if (it != g_tune_cache.end()) return it->second;
  const char* path = std::getenv("FDD_AUTOTUNE_CACHE");
  if (!path) return -1;
  FILE* f = std::fopen(path, "r");
  if (!f) return -1;
  char k[128];
  int v = -1, found = -1;
  while (std::fscanf(f, "%127s %d", k, &v) == 2)
    if (key == k) found = v;
  std::fclose(f);
  if (found >= 0) g_tune_cache[key] = found;
  return found;
}

void cache_store(const std::string& key, int v) {
  std::lock_guard<std::mutex> lk(g_tune_mutex);
  g_tune_cache[key] = v;
  const char* path = std::getenv("FDD_AUTOTUNE_CACHE");
  if (!path) return;
  FILE* f = std::fopen(path, "a");
  if (!f) return;
  std::fprintf(f, "%s %d\n", key.c_str(), v);
  std::fclose(f);
}

}  // namespace

extern "C" {

fdd_status fdd_batch_plan(const fdd_params* p, const fdd_beam_desc* beams, int32_t n_beams,
                          int32_t autotune, fdd_batch_t* out) {
  using fdd::report_error;
  if (!out) return report_error(FDD_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!p || !beams || n_beams < 1)
    return report_error(FDD_ERR_INVALID_ARG, "NULL params or beams, or no beams");
  if (p->output != FDD_OUT_SPECTRA && p->output != FDD_OUT_POWER)
    return report_error(FDD_ERR_UNSUPPORTED,
                        "the batching form emits spectra or power (time output: per-beam plans)");
  if (p->precision != FDD_PREC_FP32)
    return report_error(FDD_ERR_UNSUPPORTED, "the batching form runs the FP32 form");
  if (p->chunk_len != 0)
    return report_error(FDD_ERR_UNSUPPORTED, "the batching form transforms whole series (chunk_len 0)");
  if (p->mac_variant < 0 || p->mac_variant > FDD_MAC_VARIANTS)
    return report_error(FDD_ERR_INVALID_ARG, "mac_variant out of range");

  fdd_batch_s* B = new (std::nothrow) fdd_batch_s();
  if (!B) return report_error(FDD_ERR_ALLOC, "host allocation failed");
  std::unique_ptr<fdd_batch_s, void (*)(fdd_batch_s*)> guard(B, release);
  B->p = *p;
  B->p.dm_list = nullptr;
  B->beams.assign(beams, beams + n_beams);

  // Geometry and phase tables per beam; plan-time validation through
  // fdd_plan_geometry with this beam's series and trial grid.
  std::vector<fdd::PhaseConst> pc(static_cast<size_t>(n_beams) * p->n_chan);
  int64_t L_max = 0, in_acc = 0, out_acc = 0;
  for (int b = 0; b < n_beams; ++b) {
    const fdd_beam_desc& d = beams[b];
    if (d.n_dm < 1 || d.n_t < 2 || !(d.dm0 >= 0.0) || !(d.ddm >= 0.0) ||
        !std::isfinite(d.dm0) || !std::isfinite(d.ddm) || d.reserved != 0)
      return report_error(FDD_ERR_INVALID_ARG, "invalid beam description");
    std::vector<double> dms(d.n_dm);
    for (int j = 0; j < d.n_dm; ++j) dms[j] = d.dm0 + d.ddm * j;
    fdd_params q = *p;
    q.n_t = d.n_t;
    q.n_beams = 1;
    q.dm_list = dms.data();
    q.n_dm = d.n_dm;
    fdd_info g;
    fdd_status st = fdd_plan_geometry(&q, &g);
    if (st != FDD_OK) return st;
    B->L.push_back(g.fft_len);
    B->n_bins.push_back(g.n_bins);
    B->pitch.push_back(g.bin_pitch);
    B->in_off.push_back(in_acc);
    B->out_off.push_back(out_acc);
    in_acc += d.n_t * static_cast<int64_t>(p->n_chan);
    out_acc += g.n_bins * static_cast<int64_t>(d.n_dm);
    L_max = std::max(L_max, g.fft_len);
    fdd::CoreGeometry cg;
    if ((st = fdd::core_geometry(&q, &cg)) != FDD_OK) return st;
    for (int c = 0; c < p->n_chan; ++c)
      pc[static_cast<size_t>(b) * p->n_chan + c] = fdd::phase_const(
          fdd::delay_rate(q, cg, c), static_cast<double>(g.fft_len), g.dm0, g.ddm);
  }
  B->in_elems = in_acc;
  B->out_elems = out_acc;

  B_CUDA(cudaGetDevice(&B->device));
  B_CUDA(cudaDeviceGetAttribute(&B->n_sms, cudaDevAttrMultiProcessorCount, B->device));

  // Waves: consecutive beams whose spectra fit the pool.
  const size_t limit = p->workspace_limit ? p->workspace_limit : (size_t(16) << 30);
  const size_t fixed = sizeof(float) * size_t(p->n_chan) * L_max +
                       sizeof(fdd::PhaseConst) * pc.size() + (size_t(64) << 20);
  if (fixed >= limit) return report_error(FDD_ERR_INVALID_ARG, "workspace_limit too small");
  const size_t pool_cap = limit - fixed;
  size_t pool_need = 0, cur = 0;
  fdd_batch_s::Wave w;
  for (int b = 0; b < n_beams; ++b) {
    const size_t spec = sizeof(float2) * size_t(p->n_chan) * B->pitch[b];
    if (spec > pool_cap)
      return report_error(FDD_ERR_INVALID_ARG, "one beam's spectra exceed workspace_limit");
    if (cur + spec > pool_cap) {
      B->waves.push_back(w);
      w = fdd_batch_s::Wave();
      w.first = b;
      cur = 0;
    }
    B->spec_off.push_back(static_cast<int64_t>(cur / sizeof(float2)));
    B->wave_of.push_back(static_cast<int>(B->waves.size()));
    cur += spec;
    w.count += 1;
    pool_need = std::max(pool_need, cur);
  }
  B->waves.push_back(w);

  // Device buffers.
  fdd_status st;
  if ((st = alloc(B, reinterpret_cast<void**>(&B->d_pc), sizeof(fdd::PhaseConst) * pc.size())))
    return st;
  if ((st = alloc(B, reinterpret_cast<void**>(&B->d_xw), sizeof(float) * size_t(p->n_chan) * L_max)))
    return st;
  if ((st = alloc(B, reinterpret_cast<void**>(&B->d_pool), pool_need))) return st;
  if ((st = alloc(B, reinterpret_cast<void**>(&B->d_counter),
                  2 * sizeof(unsigned long long) * B->waves.size())))
    return st;
  B_CUDA(cudaMemcpy(B->d_pc, pc.data(), sizeof(fdd::PhaseConst) * pc.size(),
                    cudaMemcpyHostToDevice));

  // cuFFT plans per distinct length, sharing one work area.
  size_t work = 0;
  for (int b = 0; b < n_beams; ++b) {
    if (B->r2c.count(B->L[b])) continue;
    cufftHandle h;
    B_CUFFT(cufftCreate(&h));
    B->r2c[B->L[b]] = h;
    B_CUFFT(cufftSetAutoAllocation(h, 0));
    long long n[1] = {B->L[b]}, er[1] = {B->L[b]}, ec[1] = {B->pitch[b]};
    size_t ws = 0;
    B_CUFFT(cufftMakePlanMany64(h, 1, n, er, 1, B->L[b], ec, 1, B->pitch[b], CUFFT_R2C,
                                p->n_chan, &ws));
    work = std::max(work, ws);
  }
  if (work) {
    if ((st = alloc(B, &B->d_fftwork, work))) return st;
    for (auto& kv : B->r2c) B_CUFFT(cufftSetWorkArea(kv.second, B->d_fftwork));
  }

  // Work sets per wave (output pointers bound at execute).  With a tile of
  // 2048-trial blocks, a beam's last block of 1024 or fewer trials goes to the
  // tail tile's 128-trial blocks instead (less padding beyond the trial grid).
  auto base_args = [&](int b) {
    fdd::MacArgs m{};
    m.X = B->d_pool + B->spec_off[b];
    m.x_series_stride = 0;
    m.x_chan_stride = B->pitch[b];
    m.pc = B->d_pc + static_cast<size_t>(b) * p->n_chan;
    m.n_chan = p->n_chan;
    m.n_bins = static_cast<int>(B->n_bins[b]);
    m.n_series = 1;
    m.y_series_stride = 0;
    m.y_dm_stride = B->n_bins[b];
    m.out_kind = p->output == FDD_OUT_SPECTRA ? 1 : 2;
    m.scale = 1.0f;
    m.real_bin_a = -1;
    m.real_bin_b = -1;
    return m;
  };
  auto build_sets = [&](int variant) -> fdd_status {
    const int bins_per_cta = fdd::mac_variant_bins_per_cta(variant);
    const int dms = fdd::mac_variant_trials_per_block(variant);
    const int tv = B->tail_variant;
    const int tail_dms = tv >= 0 ? fdd::mac_variant_trials_per_block(tv) : 0;
    // (the three-product tile runs a ragged last block of up to half its
    // trials in the same launch, at half its work: no second launch)
    const bool tails = tv >= 0 && dms >= 2048 && tail_dms < dms && variant != FDD_MAC_G12_4X8;
    for (auto& wv : B->waves) {
      wv.h_sets.assign(wv.count, fdd::BatchSet{});
      wv.h_tail.clear();
      wv.tail_beam.clear();
      long long items = 0, t_items = 0;
      for (int i = 0; i < wv.count; ++i) {
        const int b = wv.first + i;
        const int n_dm = B->beams[b].n_dm;
        const int full = n_dm / dms, rem = n_dm % dms;
        const bool tail = tails && rem > 0 && rem <= dms / 2;
        const int blocks = full + (rem > 0 && !tail ? 1 : 0);
        fdd::BatchSet& bs = wv.h_sets[i];
        bs.args = base_args(b);
        bs.args.j_begin = 0;
        bs.args.n_dm = tail ? full * dms : n_dm;
        bs.n_bin_tiles = static_cast<int>((B->n_bins[b] + bins_per_cta - 1) / bins_per_cta);
        bs.n_dm_blocks = blocks;
        bs.item_begin = items;
        items += static_cast<long long>(bs.n_bin_tiles) * blocks;
        if (tail) {
          fdd::BatchSet ts{};
          ts.args = base_args(b);
          ts.args.j_begin = full * dms;
          ts.args.n_dm = rem;
          const int tb = fdd::mac_variant_bins_per_cta(tv);
          ts.n_bin_tiles = static_cast<int>((B->n_bins[b] + tb - 1) / tb);
          ts.n_dm_blocks = (rem + tail_dms - 1) / tail_dms;
          ts.item_begin = t_items;
          t_items += static_cast<long long>(ts.n_bin_tiles) * ts.n_dm_blocks;
          wv.h_tail.push_back(ts);
          wv.tail_beam.push_back(b);
        }
      }
      wv.n_items = items;
      wv.n_tail_items = t_items;
    }
    return FDD_OK;
  };
  for (auto& wv : B->waves) {
    if ((st = alloc(B, reinterpret_cast<void**>(&wv.d_sets), sizeof(fdd::BatchSet) * wv.count)))
      return st;
    if ((st = alloc(B, reinterpret_cast<void**>(&wv.d_tail), sizeof(fdd::BatchSet) * wv.count)))
      return st;
  }
  // the tail tile (128-trial blocks, four bins per warp)
  {
    const int tv = FDD_MAC_Q_4X4;
    B_CUDA(fdd::mac_prepare(tv, p->n_chan));
    const int per_sm = fdd::mac_batch_ctas_per_sm(tv, p->n_chan);
    if (per_sm >= 1) {
      B->tail_variant = tv;
      B->tail_ctas = per_sm * B->n_sms;
    }
  }

  auto use_variant = [&](int v) -> fdd_status {
    B->variant = v;
    B_CUDA(fdd::mac_prepare(v, p->n_chan));
    const int per_sm = fdd::mac_batch_ctas_per_sm(v, p->n_chan);
    if (per_sm < 1) return report_error(FDD_ERR_UNSUPPORTED, "kernel tile does not fit an SM");
    B->ctas = per_sm * B->n_sms;
    return build_sets(v);
  };

  for (double& t : B->tune_ms) t = -1.0;
  int variant = p->mac_variant ? p->mac_variant - 1 : -1;
  if (variant >= 0 && !fdd::mac_variant_batchable(variant))
    return report_error(FDD_ERR_UNSUPPORTED, "this kernel variant has no batched form");
  const std::string key = signature(B);
  if (variant < 0 && autotune) variant = cache_lookup(key);
  if (variant < 0 && autotune) {
    // Time each candidate on wave 0's real shapes (spectra and output scratch
    // are this plan's; values do not affect the timing).
    const int cands[] = {FDD_MAC_W12_8X8, FDD_MAC_G12_4X8, FDD_MAC_Q12_8X8, FDD_MAC_Q_4X8,
                         FDD_MAC_Q_4X4};
    const auto& w0 = B->waves[0];
    int64_t w0_out = 0;
    for (int i = 0; i < w0.count; ++i)
      w0_out += B->n_bins[w0.first + i] * static_cast<int64_t>(B->beams[w0.first + i].n_dm);
    void* scratch = nullptr;
    B_CUDA(cudaMalloc(&scratch, (p->output == FDD_OUT_SPECTRA ? 8 : 4) * size_t(w0_out)));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double best = std::numeric_limits<double>::infinity();
    fdd_status tst = FDD_OK;
    for (int v : cands) {
      if ((tst = use_variant(v))) break;
      // output of wave 0 into the scratch, laid out like the real output
      auto& w0m = B->waves[0];
      const int64_t origin = B->out_off[w0.first];
      for (int i = 0; i < w0.count; ++i) bind_set(B, w0m.h_sets[i], w0.first + i, scratch, origin);
      for (size_t i = 0; i < w0.h_tail.size(); ++i)
        bind_set(B, w0m.h_tail[i], w0.tail_beam[i], scratch, origin);
      if ((tst = upload_wave(w0, nullptr))) break;
      // Each launch times a bounded share of wave 0's items (eight rounds of
      // the persistent grid rank the tiles whatever the wave's size), scaled
      // to the whole wave: main launch plus, for a tile with one, tail launch.
      auto timed = [&](fdd::BatchSet* sets, int n_sets, long long n_items, int tile, int ctas,
                       unsigned long long* counter) -> double {
        const long long part = std::min<long long>(n_items, 8LL * ctas);
        float ms = 0.f;
        for (int rep = 0; rep < 2; ++rep) {  // the first launch is a warm-up
          cudaMemset(counter, 0, sizeof(unsigned long long));
          cudaEventRecord(e0);
          fdd::launch_mac_batch(sets, n_sets, part, counter, tile, ctas, p->n_chan, nullptr);
          cudaEventRecord(e1);
          cudaEventSynchronize(e1);
          cudaEventElapsedTime(&ms, e0, e1);
        }
        return static_cast<double>(ms) * static_cast<double>(n_items) / static_cast<double>(part);
      };
      double tot = timed(w0.d_sets, w0.count, w0.n_items, v, B->ctas, B->d_counter);
      if (w0.n_tail_items)
        tot += timed(w0.d_tail, static_cast<int>(w0.h_tail.size()), w0.n_tail_items,
                     B->tail_variant, B->tail_ctas, B->d_counter + 1);
      if (cudaGetLastError() != cudaSuccess) {
        tst = report_error(FDD_ERR_CUDA, "autotune launch failed");
        break;
      }
      B->tune_ms[v] = tot;
      if (tot < best) {
        best = tot;
        variant = v;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(scratch);
    if (tst != FDD_OK) return tst;
    cache_store(key, variant);
  }
  if (variant < 0) variant = FDD_MAC_G12_4X8;
  if ((st = use_variant(variant))) return st;
  B_CUDA(cudaStreamCreateWithFlags(&B->cap_stream, cudaStreamNonBlocking));
  *out = guard.release();
  return FDD_OK;
}

fdd_status fdd_batch_query(fdd_batch_t b, fdd_batch_info* info, int64_t* in_offsets,
                           int64_t* out_offsets) {
  if (!b || !info) return fdd::report_error(FDD_ERR_INVALID_ARG, "NULL batch or info");
  std::memset(info, 0, sizeof *info);
  info->in_elems = b->in_elems;
  info->out_elems = b->out_elems;
  info->out_bytes = b->out_elems * (b->p.output == FDD_OUT_SPECTRA ? 8 : 4);
  info->workspace_bytes = static_cast<int64_t>(b->bytes_held);
  info->n_waves = static_cast<int32_t>(b->waves.size());
  info->mac_variant = b->variant;
  long long items = 0;
  bool any_tail = false;
  for (auto& w : b->waves) {
    items += w.n_items + w.n_tail_items;
    any_tail = any_tail || w.n_tail_items > 0;
  }
  info->work_items = items;
  info->ctas = b->ctas;
  info->tail_variant = any_tail ? b->tail_variant : -1;
  for (int v = 0; v < FDD_MAC_VARIANTS; ++v) info->autotune_ms[v] = b->tune_ms[v];
  for (size_t i = 0; i < b->beams.size(); ++i) {
    if (in_offsets) in_offsets[i] = b->in_off[i];
    if (out_offsets) out_offsets[i] = b->out_off[i];
  }
  return FDD_OK;
}

fdd_status fdd_batch_execute(fdd_batch_t b, const void* d_in, void* d_out, fdd_stream_t stream) {
  if (!b) return fdd::report_error(FDD_ERR_INVALID_ARG, "batch is NULL");
  if (!d_in || !d_out) return fdd::report_error(FDD_ERR_INVALID_ARG, "NULL input or output");
  int dev = -1;
  B_CUDA(cudaGetDevice(&dev));
  if (dev != b->device)
    return fdd::report_error(FDD_ERR_INVALID_ARG, "batch plan belongs to another device");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (!b->graph || b->graph_in != d_in || b->graph_out != d_out) {
    // (Re)build the graph for these buffers: bind and upload the work sets,
    // then capture one execute on the plan's private stream.
    if (b->graph) {
      B_CUDA(cudaStreamSynchronize(s));
      cudaGraphExecDestroy(b->graph);
      b->graph = nullptr;
    }
    bind_output(b, d_out);
    fdd_status st = upload_sets(b, s);
    if (st != FDD_OK) return st;
    B_CUDA(cudaStreamSynchronize(s));
    B_CUDA(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
    st = issue(b, d_in, b->cap_stream);
    cudaGraph_t g = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(b->cap_stream, &g);
    if (st != FDD_OK) {
      if (g) cudaGraphDestroy(g);
      return st;
    }
    if (ec != cudaSuccess) {
      cudaGetLastError();
      return fdd::report_error(FDD_ERR_CUDA, cudaGetErrorString(ec));
    }
    const cudaError_t ei = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) {
      cudaGetLastError();
      b->graph = nullptr;
      return fdd::report_error(FDD_ERR_CUDA, cudaGetErrorString(ei));
    }
    b->graph_in = d_in;
    b->graph_out = d_out;
  }
  B_CUDA(cudaGraphLaunch(b->graph, s));
  return FDD_OK;
}

fdd_status fdd_batch_execute_stream(fdd_batch_t b, fdd_source_fn source, void* source_user,
                                    fdd_sink_fn sink, void* sink_user, fdd_stream_t stream) {
  using fdd::report_error;
  if (!b) return report_error(FDD_ERR_INVALID_ARG, "batch is NULL");
  if (!source || !sink) return report_error(FDD_ERR_INVALID_ARG, "NULL source or sink");
  int dev = -1;
  B_CUDA(cudaGetDevice(&dev));
  if (dev != b->device)
    return report_error(FDD_ERR_INVALID_ARG, "batch plan belongs to another device");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  fdd_status st;
  const size_t esz = b->p.in_dtype == FDD_IN_U8 ? 1 : 4;
  const size_t oesz = b->p.output == FDD_OUT_SPECTRA ? 8 : 4;
  if (!b->d_win[0]) {
    // rings: windows of the longest beam, output slots of the largest wave,
    // and each wave's work sets bound to each output slot
    int64_t nt_max = 0;
    for (auto& d : b->beams) nt_max = std::max<int64_t>(nt_max, d.n_t);
    size_t wmax = 0;
    for (auto& w : b->waves) {
      size_t o = 0;
      for (int i = 0; i < w.count; ++i)
        o += oesz * static_cast<size_t>(b->n_bins[w.first + i]) * b->beams[w.first + i].n_dm;
      wmax = std::max(wmax, o);
    }
    b->wout_bytes = wmax;
    for (int k = 0; k < 2; ++k) {
      if ((st = alloc(b, &b->d_win[k], esz * static_cast<size_t>(b->p.n_chan) * nt_max)))
        return st;
      if ((st = alloc(b, &b->d_wout[k], wmax))) return st;
      B_CUDA(cudaEventCreateWithFlags(&b->win_free[k], cudaEventDisableTiming));
      for (size_t wi = 0; wi < b->waves.size(); ++wi) {
        auto& w = b->waves[wi];
        const int64_t origin = b->out_off[w.first];
        std::vector<fdd::BatchSet> sets = w.h_sets, tails = w.h_tail;
        for (int i = 0; i < w.count; ++i) bind_set(b, sets[i], w.first + i, b->d_wout[k], origin);
        for (size_t i = 0; i < tails.size(); ++i)
          bind_set(b, tails[i], w.tail_beam[i], b->d_wout[k], origin);
        fdd::BatchSet* d = nullptr;
        const size_t n = sets.size() + tails.size();
        if ((st = alloc(b, reinterpret_cast<void**>(&d), sizeof(fdd::BatchSet) * n))) return st;
        b->d_sets_slot[k].push_back(d);
        B_CUDA(cudaMemcpy(d, sets.data(), sizeof(fdd::BatchSet) * sets.size(),
                          cudaMemcpyHostToDevice));
        if (!tails.empty())
          B_CUDA(cudaMemcpy(d + sets.size(), tails.data(), sizeof(fdd::BatchSet) * tails.size(),
                            cudaMemcpyHostToDevice));
      }
    }
  }
  for (auto& kv : b->r2c) B_CUFFT(cufftSetStream(kv.second, s));
  for (size_t wi = 0; wi < b->waves.size(); ++wi) {
    const auto& w = b->waves[wi];
    for (int i = 0; i < w.count; ++i) {
      const int bm = w.first + i;
      const int slot = static_cast<int>(b->win_next++ & 1);
      void* ready = b->win_used[slot] ? static_cast<void*>(b->win_free[slot]) : nullptr;
      st = source(source_user, bm, 0, b->beams[bm].n_t, b->d_win[slot], ready, stream);
      if (st != FDD_OK) return report_error(st, "the input source failed");
      fdd::UnpackArgs ua{b->d_win[slot], b->p.in_dtype, b->p.in_layout, b->p.n_chan,
                         b->beams[bm].n_t, 0, b->L[bm], b->d_xw, b->L[bm]};
      B_CUDA(fdd::launch_unpack(ua, s));
      B_CUDA(cudaEventRecord(b->win_free[slot], s));
      b->win_used[slot] = true;
      B_CUFFT(cufftExecR2C(b->r2c.at(b->L[bm]), b->d_xw,
                           reinterpret_cast<cufftComplex*>(b->d_pool + b->spec_off[bm])));
    }
    const int k = static_cast<int>(b->out_next++ & 1);
    if (b->out_release[k]) {  // the sink's reads of this slot's last wave
      B_CUDA(cudaStreamWaitEvent(s, static_cast<cudaEvent_t>(b->out_release[k]), 0));
      b->out_release[k] = nullptr;
    }
    fdd::BatchSet* d_sets = b->d_sets_slot[k][wi];
    B_CUDA(cudaMemsetAsync(b->d_counter + 2 * wi, 0, 2 * sizeof(unsigned long long), s));
    B_CUDA(fdd::launch_mac_batch(d_sets, w.count, w.n_items, b->d_counter + 2 * wi, b->variant,
                                 b->ctas, b->p.n_chan, s));
    if (w.n_tail_items)
      B_CUDA(fdd::launch_mac_batch(d_sets + w.count, static_cast<int>(w.h_tail.size()),
                                   w.n_tail_items, b->d_counter + 2 * wi + 1, b->tail_variant,
                                   b->tail_ctas, b->p.n_chan, s));
    const int64_t origin = b->out_off[w.first];
    void* release = nullptr;
    for (int i = 0; i < w.count; ++i) {
      const int bm = w.first + i;
      fdd_block blk{bm, 1, 0, 0, b->beams[bm].n_dm,
                    static_cast<char*>(b->d_wout[k]) + oesz * (b->out_off[bm] - origin),
                    b->n_bins[bm], b->n_bins[bm], 0, nullptr};
      st = sink(sink_user, &blk, stream);
      if (st != FDD_OK) return report_error(st, "the output sink failed");
      if (blk.release_event) release = blk.release_event;  // the wave's last one counts
    }
    b->out_release[k] = release;
  }
  return FDD_OK;
}

fdd_status fdd_batch_destroy(fdd_batch_t b) {
  if (!b) return FDD_OK;
  const cudaError_t e = cudaDeviceSynchronize();
  release(b);
  if (e != cudaSuccess)
    return fdd::report_error(FDD_ERR_CUDA, cudaGetErrorString(e));
  return FDD_OK;
}

}  // extern "C"

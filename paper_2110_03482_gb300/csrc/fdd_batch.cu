// fdd_batch.cu -- the batching form: many beams of uneven length and uneven
// trial grids dedispersed together (the batch dimensions of Sect. 3 /
// Algorithm 1 and the autotuning suggestion of Sect. 5).
//
// Beams are grouped into waves whose spectra fit the workspace.  For each
// wave the beams are unpacked and transformed one by one, whole or in their
// own overlap-save chunks (one cuFFT plan per distinct transform length),
// then ONE persistent launch of the FP32 phase-rotate-and-sum serves the
// whole wave: its CTAs pull (beam, chunk, bin tile, trial block) items from a
// counter.  The whole execute is captured once as a
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
#include <tuple>
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
  // per beam (a chunk's spectra are n_chan x pitch, its output n_dm x n_bins)
  std::vector<int64_t> L, n_bins, pitch, n_chunks, hop, in_off, out_off, spec_off;
  std::vector<int> wave_of;
  // per wave
  struct Wave {
    int first = 0, count = 0;  // beams
    long long n_items = 0;
    fdd::BatchSet* d_sets = nullptr;
    std::vector<fdd::BatchSet> h_sets;   // one per (beam, chunk)
    std::vector<int> set_beam, set_chunk;
    // ragged last trial blocks of 1024 or fewer trials, on the tail tile
    long long n_tail_items = 0;
    fdd::BatchSet* d_tail = nullptr;
    std::vector<fdd::BatchSet> h_tail;
    std::vector<int> tail_beam, tail_chunk;
  };
  std::vector<Wave> waves;
  int64_t in_elems = 0, out_elems = 0;
  // device memory
  fdd::PhaseConst* d_pc = nullptr;  // [beam][n_chan]
  float* d_xw = nullptr;            // [n_chan][L_max]
  float2* d_pool = nullptr;         // spectra of one wave
  unsigned long long* d_counter = nullptr;  // one per wave
  int* d_status = nullptr;  // device-side timeouts of the persistent launches
  fdd_status tc_status = FDD_OK;  // a timeout seen in a made-and-destroyed plan
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
  // tensor-core form: beams grouped by what their phasors share (transform
  // length, trial grid origin and step; with chunks also the trial count,
  // which sets the overlap), one plan per group of up to 16 beams, run
  // through fdd_execute_stream.  Plans are kept while their workspaces fit
  // the limit together, else each is made for its turn and destroyed after.
  struct TcGroup {
    fdd_params q{};
    std::vector<double> dms;
    std::vector<int> beams;  // batch beams in the plan's beam order
    fdd_plan_t plan = nullptr;
  };
  bool tc = false;
  std::vector<TcGroup> tc_groups;
  // plans whose workspaces exceed the limit together share one block of the
  // largest one's size for their per-call buffers (run one after another)
  void* tc_arena = nullptr;
  cudaEvent_t tc_ready = nullptr;  // recorded before each plan of a shared block
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
  for (auto& g : B->tc_groups)
    if (g.plan) fdd_destroy(g.plan);
  if (B->tc_arena) cudaFree(B->tc_arena);
  if (B->tc_ready) cudaEventDestroy(B->tc_ready);
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
  void* ptrs[] = {B->d_pc, B->d_xw, B->d_pool, B->d_counter, B->d_fftwork, B->d_status};
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

// Output element of trial 0 of chunk c of beam b.
int64_t chunk_out(const fdd_batch_s* B, int b, int64_t c) {
  return B->out_off[b] + c * B->beams[b].n_dm * B->n_bins[b];
}

// Sets the output pointers of a work set for the given output buffer: a
// set's row 0 is trial j_begin of its beam's chunk c.
// (`origin`: output element at d_out, nonzero for a buffer that holds only
// the beams from some beam on)
void bind_set(const fdd_batch_s* B, fdd::BatchSet& bs, int b, int c, void* d_out,
              int64_t origin = 0) {
  fdd::MacArgs& m = bs.args;
  const int64_t off = chunk_out(B, b, c) - origin + static_cast<int64_t>(m.j_begin) * B->n_bins[b];
  if (B->p.output == FDD_OUT_SPECTRA)
    m.Y = static_cast<float2*>(d_out) + off;
  else
    m.Y = static_cast<float*>(d_out) + off;
}

void bind_wave(const fdd_batch_s* B, std::vector<fdd::BatchSet>& sets,
               std::vector<fdd::BatchSet>& tails, const fdd_batch_s::Wave& w, void* d_out,
               int64_t origin) {
  for (size_t i = 0; i < sets.size(); ++i)
    bind_set(B, sets[i], w.set_beam[i], w.set_chunk[i], d_out, origin);
  for (size_t i = 0; i < tails.size(); ++i)
    bind_set(B, tails[i], w.tail_beam[i], w.tail_chunk[i], d_out, origin);
}

void bind_output(fdd_batch_s* B, void* d_out) {
  for (auto& w : B->waves) bind_wave(B, w.h_sets, w.h_tail, w, d_out, 0);
}

// Unpack chunk c of beam b from its input and transform it into the pool.
fdd_status transform_chunk(fdd_batch_s* B, const void* beam_in, int b, int64_t c,
                           cudaStream_t s) {
  fdd::UnpackArgs ua{beam_in, B->p.in_dtype, B->p.in_layout, B->p.n_chan, B->beams[b].n_t,
                     c * B->hop[b], B->L[b], B->d_xw, B->L[b]};
  B_CUDA(fdd::launch_unpack(ua, s));
  B_CUFFT(cufftExecR2C(B->r2c.at(B->L[b]), B->d_xw,
                       reinterpret_cast<cufftComplex*>(
                           B->d_pool + B->spec_off[b] + c * B->p.n_chan * B->pitch[b])));
  return FDD_OK;
}

// All work of one execute, issued on stream s (also used under capture).
fdd_status issue(fdd_batch_s* B, const void* d_in, cudaStream_t s) {
  const size_t esz = B->p.in_dtype == FDD_IN_U8 ? 1 : 4;
  for (auto& kv : B->r2c) B_CUFFT(cufftSetStream(kv.second, s));
  for (size_t wi = 0; wi < B->waves.size(); ++wi) {
    const auto& w = B->waves[wi];
    for (int i = 0; i < w.count; ++i) {
      const int b = w.first + i;
      for (int64_t c = 0; c < B->n_chunks[b]; ++c) {
        const fdd_status st =
            transform_chunk(B, static_cast<const char*>(d_in) + esz * B->in_off[b], b, c, s);
        if (st != FDD_OK) return st;
      }
    }
    B_CUDA(cudaMemsetAsync(B->d_counter + 2 * wi, 0, 2 * sizeof(unsigned long long), s));
    B_CUDA(fdd::launch_mac_batch(w.d_sets, static_cast<int>(w.h_sets.size()), w.n_items,
                                 B->d_counter + 2 * wi, B->variant, B->ctas, B->p.n_chan, s));
    if (w.n_tail_items)
      B_CUDA(fdd::launch_mac_batch(w.d_tail, static_cast<int>(w.h_tail.size()), w.n_tail_items,
                                   B->d_counter + 2 * wi + 1, B->tail_variant, B->tail_ctas,
                                   B->p.n_chan, s));
  }
  return FDD_OK;
}

fdd_status upload_wave(const fdd_batch_s::Wave& w, cudaStream_t s) {
  B_CUDA(cudaMemcpyAsync(w.d_sets, w.h_sets.data(), sizeof(fdd::BatchSet) * w.h_sets.size(),
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

// ------------------------------------------------ tensor-core batch
// The callbacks of one group's fdd_execute_stream: windows come from the
// resident input (d_in) or the caller's source, blocks go to the resident
// output (d_out) or the caller's sink, one (beam, chunk) at a time.  A beam
// shorter than the group's longest reads zeros beyond its own samples, which
// is its own zero padding (whole series) or its own last chunks' zero fill;
// chunks and trials beyond its own are dropped.
struct TcCtx {
  fdd_batch_s* B;
  const fdd_batch_s::TcGroup* g;
  const void* d_in;
  void* d_out;
  fdd_source_fn source;
  void* source_user;
  fdd_sink_fn sink;
  void* sink_user;
  fdd_status inner = FDD_OK;  // a callback's own failure
  void* arena_ready = nullptr;  // shared block: recorded before this plan's work
};

fdd_status tc_source(void* user, int32_t beam, int64_t t_begin, int64_t n, void* d_window,
                     void* ready, fdd_stream_t stream) {
  TcCtx* x = static_cast<TcCtx*>(user);
  const fdd_batch_s* B = x->B;
  const int bm = x->g->beams[beam];
  const int64_t nc = B->p.n_chan;
  const size_t esz = B->p.in_dtype == FDD_IN_U8 ? 1 : 4;
  const bool tmaj = B->p.in_layout == FDD_LAYOUT_TIME_MAJOR;
  const int64_t nb = std::max<int64_t>(0, std::min<int64_t>(n, B->beams[bm].n_t - t_begin));
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  char* win = static_cast<char*>(d_window);
  if (nb < n) {  // samples beyond the beam: zeros
    cudaError_t e = cudaSuccess;
    if (tmaj)
      e = cudaMemsetAsync(win + esz * nb * nc, 0, esz * (n - nb) * nc, s);
    else
      e = cudaMemset2DAsync(win + esz * nb, esz * n, 0, esz * (n - nb), nc, s);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fdd::report_error(FDD_ERR_CUDA, cudaGetErrorString(e));
    }
  }
  if (nb == 0) return FDD_OK;
  if (x->d_in) {
    const char* src = static_cast<const char*>(x->d_in) + esz * B->in_off[bm];
    cudaError_t e;
    if (tmaj)
      e = cudaMemcpyAsync(win, src + esz * t_begin * nc, esz * nb * nc, cudaMemcpyDeviceToDevice,
                          s);
    else
      e = cudaMemcpy2DAsync(win, esz * n, src + esz * t_begin, esz * B->beams[bm].n_t, esz * nb,
                            nc, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fdd::report_error(FDD_ERR_CUDA, cudaGetErrorString(e));
    }
    return FDD_OK;
  }
  // (a window in a shared block may still hold an earlier plan's buffers)
  if (!ready) ready = x->arena_ready;
  const fdd_status st = x->source(x->source_user, bm, t_begin, nb, d_window, ready, stream);
  if (st != FDD_OK) x->inner = st;
  return st;
}

fdd_status tc_sink(void* user, fdd_block* blk, fdd_stream_t stream) {
  TcCtx* x = static_cast<TcCtx*>(user);
  const fdd_batch_s* B = x->B;
  const size_t esz = B->p.output == FDD_OUT_SPECTRA ? 8 : 4;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  void* release = nullptr;
  for (int i = 0; i < blk->n_beams; ++i) {
    const int bm = x->g->beams[blk->beam_first + i];
    if (blk->chunk >= B->n_chunks[bm]) continue;
    const int rows = std::min(blk->n_dm, B->beams[bm].n_dm - blk->dm_first);
    if (rows <= 0) continue;
    const char* src = static_cast<const char*>(blk->d_data) +
                      esz * static_cast<size_t>(i) * blk->n_dm * blk->row_pitch;
    if (x->d_out) {
      const int64_t o = chunk_out(B, bm, blk->chunk) +
                        static_cast<int64_t>(blk->dm_first) * B->n_bins[bm];
      const cudaError_t e =
          cudaMemcpyAsync(static_cast<char*>(x->d_out) + esz * o, src,
                          esz * static_cast<size_t>(rows) * B->n_bins[bm],
                          cudaMemcpyDeviceToDevice, s);
      if (e != cudaSuccess) {
        cudaGetLastError();
        return fdd::report_error(FDD_ERR_CUDA, cudaGetErrorString(e));
      }
      continue;
    }
    fdd_block ub{bm, 1, blk->chunk, blk->dm_first, rows, src, B->n_bins[bm], B->n_bins[bm], 0,
                 nullptr};
    const fdd_status st = x->sink(x->sink_user, &ub, stream);
    if (st != FDD_OK) {
      x->inner = st;
      return st;
    }
    if (ub.release_event) release = ub.release_event;  // the last one counts
  }
  blk->release_event = release;
  return FDD_OK;
}

fdd_status run_tc_batch(fdd_batch_s* B, TcCtx ctx, cudaStream_t s) {
  for (auto& g : B->tc_groups) {
    fdd_plan_t plan = g.plan;
    fdd_status st;
    if (!plan && (st = fdd_plan(&g.q, &plan)) != FDD_OK) return st;
    ctx.g = &g;
    if (B->tc_arena) {
      B_CUDA(cudaEventRecord(B->tc_ready, s));
      ctx.arena_ready = B->tc_ready;
    }
    st = fdd_execute_stream(plan, nullptr, tc_source, &ctx, tc_sink, &ctx,
                            reinterpret_cast<fdd_stream_t>(s));
    // the next plan of a shared block starts after the sink's reads of this one's blocks
    if (st == FDD_OK && B->tc_arena) st = fdd::plan_drain(plan, s);
    if (!g.plan) {
      fdd_info gi;
      if (st == FDD_OK && fdd_query(plan, &gi) == FDD_ERR_TIMEOUT) B->tc_status = FDD_ERR_TIMEOUT;
      const fdd_status sd = fdd_destroy(plan);  // waits for the device
      if (st == FDD_OK) st = sd;
    }
    if (st != FDD_OK) return ctx.inner != FDD_OK ? ctx.inner : st;
  }
  return FDD_OK;
}

// Groups and plans of the tensor-core form.
fdd_status plan_tc_groups(fdd_batch_s* B, const fdd_params* p) {
  using fdd::report_error;
  // key: (transform length, chunk length, trial count for chunked beams,
  // dm0, ddm); whole-series beams of one length share a group whatever
  // their trial counts and lengths (the group runs to its largest)
  std::map<std::tuple<int64_t, int32_t, int32_t, double, double>, std::vector<int>> keyed;
  for (size_t b = 0; b < B->beams.size(); ++b) {
    const fdd_beam_desc& d = B->beams[b];
    keyed[std::make_tuple(B->L[b], d.chunk_len, d.chunk_len ? d.n_dm : 0, d.dm0, d.ddm)]
        .push_back(static_cast<int>(b));
  }
  constexpr int kGroup = 16;  // beams per plan (the 16-beam tensor-core groups)
  const size_t limit = p->workspace_limit ? p->workspace_limit : (size_t(16) << 30);
  auto with_margin = [](size_t bytes) { return bytes + bytes / 16 + (size_t(256) << 20); };
  // a plan of beams v[i0 .. i0 + n - 1] and the device bytes it would hold
  // with its streaming rings
  auto make_group = [&](const std::vector<int>& v, size_t i0, size_t n,
                        fdd_batch_s::TcGroup* g, size_t* bytes) -> fdd_status {
    g->beams.assign(v.begin() + i0, v.begin() + i0 + n);
    int64_t n_t = 0;
    int n_dm = 0;
    for (int b : g->beams) {
      n_t = std::max(n_t, B->beams[b].n_t);
      n_dm = std::max(n_dm, B->beams[b].n_dm);
    }
    const fdd_beam_desc& d0 = B->beams[g->beams[0]];
    g->dms.resize(n_dm);
    for (int j = 0; j < n_dm; ++j) g->dms[j] = d0.dm0 + d0.ddm * j;
    g->q = *p;
    g->q.n_t = n_t;
    g->q.n_beams = static_cast<int32_t>(g->beams.size());
    g->q.dm_list = g->dms.data();
    g->q.n_dm = n_dm;
    g->q.chunk_len = d0.chunk_len;
    g->q.mac_variant = 0;
    fdd_info gi;
    const fdd_status st = fdd_plan_geometry(&g->q, &gi);
    *bytes = st == FDD_OK ? static_cast<size_t>(gi.workspace_bytes + gi.stream_bytes) : 0;
    return st;
  };
  size_t need = 0;
  for (auto& kv : keyed) {
    std::vector<int>& v = kv.second;
    std::stable_sort(v.begin(), v.end(), [&](int a, int c) {
      return B->beams[a].n_dm != B->beams[c].n_dm ? B->beams[a].n_dm > B->beams[c].n_dm
                                                  : B->beams[a].n_t > B->beams[c].n_t;
    });
    for (size_t i0 = 0; i0 < v.size();) {
      // up to 16 beams, fewer while the plan (with a margin for its FFT work
      // area, which the estimate leaves out) would exceed the limit alone
      size_t n = std::min<size_t>(kGroup, v.size() - i0), bytes = 0;
      fdd_batch_s::TcGroup g;
      fdd_status st = make_group(v, i0, n, &g, &bytes);
      while ((st != FDD_OK || with_margin(bytes) > limit) && n > 1)
        st = make_group(v, i0, --n, &g, &bytes);
      if (st != FDD_OK) return st;
      if (bytes > limit)
        return report_error(FDD_ERR_INVALID_ARG,
                            "workspace_limit too small for one beam's tensor-core plan");
      need += bytes;
      B->tc_groups.push_back(std::move(g));
      i0 += n;
    }
  }
  for (auto& g : B->tc_groups) g.q.dm_list = g.dms.data();  // after the moves
  // keep every plan with its own workspace when they fit the limit together
  if (need <= limit) {
    for (auto& g : B->tc_groups) {
      fdd_status st = fdd_plan(&g.q, &g.plan);
      if (st != FDD_OK) return st;
      fdd_info gi;
      fdd_query(g.plan, &gi);
      B->bytes_held += static_cast<size_t>(gi.workspace_bytes + gi.stream_bytes);
    }
    return FDD_OK;
  }
  // else one shared block for the per-call buffers, sized to the largest
  // plan (estimated; the whole limit if that proves short)
  size_t big = 0;
  for (auto& g : B->tc_groups) {
    fdd_info gi;
    fdd_plan_geometry(&g.q, &gi);
    big = std::max(big, static_cast<size_t>(gi.workspace_bytes + gi.stream_bytes));
  }
  size_t a = std::min(limit, with_margin(big));
  for (int attempt = 0; attempt < 2; ++attempt) {
    fdd_status st = alloc(B, &B->tc_arena, a);
    bool short_block = false;
    for (size_t i = 0; st == FDD_OK && i < B->tc_groups.size(); ++i) {
      auto& g = B->tc_groups[i];
      st = fdd::plan_create(&g.q, B->tc_arena, a, &g.plan);
      if (st == FDD_OK) {
        fdd_info gi;
        fdd_query(g.plan, &gi);
        // the streaming rings come from the block at the first streamed call
        if (fdd::plan_arena_used(g.plan) + 1024 + static_cast<size_t>(gi.stream_bytes) > a)
          st = report_error(FDD_ERR_ALLOC, "shared workspace too small for the streaming rings");
      }
      short_block = st == FDD_ERR_ALLOC;
    }
    if (st == FDD_OK) {
      for (auto& g : B->tc_groups) {  // the plans' own (constant) allocations
        fdd_info gi;
        fdd_query(g.plan, &gi);
        B->bytes_held += static_cast<size_t>(gi.workspace_bytes);
      }
      break;
    }
    for (auto& g : B->tc_groups)
      if (g.plan) {
        fdd_destroy(g.plan);
        g.plan = nullptr;
      }
    cudaFree(B->tc_arena);
    B->bytes_held -= a;
    B->tc_arena = nullptr;
    if (!short_block || a >= limit || attempt == 1) {
      // no shared block: each execute makes each plan for its turn
      if (st != FDD_ERR_ALLOC) return st;
      cudaGetLastError();
      return FDD_OK;
    }
    a = limit;
  }
  if (cudaEventCreateWithFlags(&B->tc_ready, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    return report_error(FDD_ERR_CUDA, "event creation failed");
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
    sig += "|" + std::to_string(B->L[b]) + "x" + std::to_string(B->beams[b].n_dm) + "x" +
           std::to_string(B->n_chunks[b]);
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
  if (p->precision < FDD_PREC_FP32 || p->precision > FDD_PREC_FP8)
    return report_error(FDD_ERR_INVALID_ARG, "unknown precision");
  if (p->chunk_len != 0)
    return report_error(FDD_ERR_UNSUPPORTED,
                        "the batching form takes each beam's chunk length from its description");
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
        !std::isfinite(d.dm0) || !std::isfinite(d.ddm) || d.chunk_len < 0)
      return report_error(FDD_ERR_INVALID_ARG, "invalid beam description");
    std::vector<double> dms(d.n_dm);
    for (int j = 0; j < d.n_dm; ++j) dms[j] = d.dm0 + d.ddm * j;
    fdd_params q = *p;
    q.n_t = d.n_t;
    q.n_beams = 1;
    q.dm_list = dms.data();
    q.n_dm = d.n_dm;
    q.chunk_len = d.chunk_len;
    fdd_info g;
    fdd_status st = fdd_plan_geometry(&q, &g);
    if (st != FDD_OK) return st;
    B->L.push_back(g.fft_len);
    B->n_bins.push_back(g.n_bins);
    B->pitch.push_back(g.bin_pitch);
    B->n_chunks.push_back(g.n_chunks);
    B->hop.push_back(g.hop);
    B->in_off.push_back(in_acc);
    B->out_off.push_back(out_acc);
    in_acc += d.n_t * static_cast<int64_t>(p->n_chan);
    out_acc += g.n_chunks * g.n_bins * static_cast<int64_t>(d.n_dm);
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

  if (p->precision != FDD_PREC_FP32) {
    B->tc = true;
    B->variant = FDD_MAC_TC;
    for (double& t : B->tune_ms) t = -1.0;
    fdd_status st = plan_tc_groups(B, p);
    if (st != FDD_OK) return st;
    *out = guard.release();
    return FDD_OK;
  }

  // Waves: consecutive beams whose spectra fit the pool.
  const size_t limit = p->workspace_limit ? p->workspace_limit : (size_t(16) << 30);
  const size_t fixed = sizeof(float) * size_t(p->n_chan) * L_max +
                       sizeof(fdd::PhaseConst) * pc.size() + (size_t(64) << 20);
  if (fixed >= limit) return report_error(FDD_ERR_INVALID_ARG, "workspace_limit too small");
  const size_t pool_cap = limit - fixed;
  size_t pool_need = 0, cur = 0;
  fdd_batch_s::Wave w;
  for (int b = 0; b < n_beams; ++b) {
    const size_t spec = sizeof(float2) * size_t(p->n_chan) * B->pitch[b] * B->n_chunks[b];
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
  if ((st = alloc(B, reinterpret_cast<void**>(&B->d_status), 256))) return st;
  B_CUDA(cudaMemset(B->d_status, 0, 256));
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
  auto base_args = [&](int b, int64_t c) {
    fdd::MacArgs m{};
    m.X = B->d_pool + B->spec_off[b] + c * p->n_chan * B->pitch[b];
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
    m.status = B->d_status;
    return m;
  };
  auto build_sets = [&](int variant) -> fdd_status {
    const int bins_per_cta = fdd::mac_variant_bins_per_cta(variant);
    const int dms = fdd::mac_variant_trials_per_block(variant);
    const int tv = B->tail_variant;
    const int tail_dms = tv >= 0 ? fdd::mac_variant_trials_per_block(tv) : 0;
    // (the three-product tile runs a ragged last block of up to half its
    // trials in the same launch, as wide items: no second launch)
    const bool tails = tv >= 0 && dms >= 2048 && tail_dms < dms && variant != FDD_MAC_G12_4X8;
    for (auto& wv : B->waves) {
      wv.h_sets.clear();
      wv.set_beam.clear();
      wv.set_chunk.clear();
      wv.h_tail.clear();
      wv.tail_beam.clear();
      wv.tail_chunk.clear();
      long long items = 0, t_items = 0;
      for (int i = 0; i < wv.count; ++i) {
        const int b = wv.first + i;
        const int n_dm = B->beams[b].n_dm;
        const int full = n_dm / dms, rem = n_dm % dms;
        const bool tail = tails && rem > 0 && rem <= dms / 2;
        // the three-product tile's last trials as wide items: up to 512 one
        // 512-trial item, up to 1024 one 1024-trial item, up to 1536 both
        // (cheaper than a full block at the measured rates), else a full block
        const bool g12 = variant == FDD_MAC_G12_4X8;
        const bool wide = g12 && rem > dms / 4 && rem <= 3 * dms / 4;
        const bool narrow = g12 && rem > 0 && (rem <= dms / 4 || (rem > dms / 2 && rem <= 3 * dms / 4));
        const int blocks = full + (rem > 0 && !tail && !wide && !narrow ? 1 : 0);
        for (int64_t c = 0; c < B->n_chunks[b]; ++c) {
          fdd::BatchSet bs{};
          bs.args = base_args(b, c);
          bs.args.j_begin = 0;
          bs.args.n_dm = tail ? full * dms : n_dm;
          bs.n_bin_tiles = static_cast<int>((B->n_bins[b] + bins_per_cta - 1) / bins_per_cta);
          bs.n_dm_blocks = blocks;
          bs.item_begin = items;
          bs.n_wide_tiles = wide ? static_cast<int>((B->n_bins[b] + 2 * bins_per_cta - 1) /
                                                    (2 * bins_per_cta))
                                 : 0;
          bs.j_wide = full * dms;
          bs.n_narrow_tiles = narrow ? static_cast<int>((B->n_bins[b] + 4 * bins_per_cta - 1) /
                                                        (4 * bins_per_cta))
                                     : 0;
          bs.j_narrow = full * dms + (wide ? dms / 2 : 0);
          items += static_cast<long long>(bs.n_bin_tiles) * blocks + bs.n_wide_tiles +
                   bs.n_narrow_tiles;
          wv.h_sets.push_back(bs);
          wv.set_beam.push_back(b);
          wv.set_chunk.push_back(static_cast<int>(c));
          if (tail) {
            fdd::BatchSet ts{};
            ts.args = base_args(b, c);
            ts.args.j_begin = full * dms;
            ts.args.n_dm = rem;
            const int tb = fdd::mac_variant_bins_per_cta(tv);
            ts.n_bin_tiles = static_cast<int>((B->n_bins[b] + tb - 1) / tb);
            ts.n_dm_blocks = (rem + tail_dms - 1) / tail_dms;
            ts.item_begin = t_items;
            t_items += static_cast<long long>(ts.n_bin_tiles) * ts.n_dm_blocks;
            wv.h_tail.push_back(ts);
            wv.tail_beam.push_back(b);
            wv.tail_chunk.push_back(static_cast<int>(c));
          }
        }
      }
      wv.n_items = items;
      wv.n_tail_items = t_items;
    }
    return FDD_OK;
  };
  for (auto& wv : B->waves) {
    int64_t n_sets = 0;
    for (int i = 0; i < wv.count; ++i) n_sets += B->n_chunks[wv.first + i];
    if ((st = alloc(B, reinterpret_cast<void**>(&wv.d_sets), sizeof(fdd::BatchSet) * n_sets)))
      return st;
    if ((st = alloc(B, reinterpret_cast<void**>(&wv.d_tail), sizeof(fdd::BatchSet) * n_sets)))
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

  auto tile_fits = [&](int v) {
    if (fdd::mac_smem_bytes(v, p->n_chan) > 227 * 1024) return false;
    if (fdd::mac_prepare(v, p->n_chan) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    return fdd::mac_batch_ctas_per_sm(v, p->n_chan) >= 1;
  };
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
    const int64_t w0_out = (w0.first + w0.count < n_beams ? B->out_off[w0.first + w0.count]
                                                           : B->out_elems) -
                           B->out_off[w0.first];
    void* scratch = nullptr;
    B_CUDA(cudaMalloc(&scratch, (p->output == FDD_OUT_SPECTRA ? 8 : 4) * size_t(w0_out)));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double best = std::numeric_limits<double>::infinity();
    fdd_status tst = FDD_OK;
    for (int v : cands) {
      if (!tile_fits(v)) continue;  // its shared memory does not hold the phase table
      if ((tst = use_variant(v))) break;
      // output of wave 0 into the scratch, laid out like the real output
      auto& w0m = B->waves[0];
      bind_wave(B, w0m.h_sets, w0m.h_tail, w0, scratch, B->out_off[w0.first]);
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
      double tot = timed(w0.d_sets, static_cast<int>(w0.h_sets.size()), w0.n_items, v, B->ctas,
                         B->d_counter);
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
  if (variant < 0) {  // G12, unless the channels' phase table leaves it no room
    const int order[] = {FDD_MAC_G12_4X8, FDD_MAC_W12_8X8, FDD_MAC_Q12_8X8, FDD_MAC_Q_4X8,
                         FDD_MAC_Q_8X8_512, FDD_MAC_Q_4X4};
    for (int v : order)
      if (tile_fits(v)) {
        variant = v;
        break;
      }
    if (variant < 0) return report_error(FDD_ERR_UNSUPPORTED, "no kernel tile fits an SM");
  }
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
  info->n_waves = static_cast<int32_t>(b->tc ? b->tc_groups.size() : b->waves.size());
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
  // a device-side wait that timed out since the last query, reported once
  bool timeout = b->tc_status == FDD_ERR_TIMEOUT;
  b->tc_status = FDD_OK;
  for (auto& g : b->tc_groups) {
    fdd_info gi;
    if (g.plan && fdd_query(g.plan, &gi) == FDD_ERR_TIMEOUT) timeout = true;
  }
  if (b->d_status) {
    int word = 0;
    B_CUDA(cudaMemcpy(&word, b->d_status, sizeof word, cudaMemcpyDeviceToHost));
    if (word != 0) {
      B_CUDA(cudaMemset(b->d_status, 0, sizeof word));
      timeout = true;
    }
  }
  if (timeout) return fdd::report_error(FDD_ERR_TIMEOUT, "a device-side wait timed out");
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
  if (b->tc) return run_tc_batch(b, TcCtx{b, nullptr, d_in, d_out, nullptr, nullptr, nullptr,
                                          nullptr}, s);
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
  if (b->tc) {
    if (b->p.in_layout != FDD_LAYOUT_TIME_MAJOR)
      return report_error(FDD_ERR_UNSUPPORTED,
                          "the streamed tensor-core batch takes time-major input");
    return run_tc_batch(b, TcCtx{b, nullptr, nullptr, nullptr, source, source_user, sink,
                                 sink_user}, s);
  }
  fdd_status st;
  const size_t esz = b->p.in_dtype == FDD_IN_U8 ? 1 : 4;
  const size_t oesz = b->p.output == FDD_OUT_SPECTRA ? 8 : 4;
  if (!b->d_win[0]) {
    // rings: windows of the longest beam, output slots of the largest wave,
    // and each wave's work sets bound to each output slot
    int64_t nt_max = 0;
    for (auto& d : b->beams) nt_max = std::max<int64_t>(nt_max, d.n_t);
    size_t wmax = 0;
    for (size_t wi = 0; wi < b->waves.size(); ++wi) {
      const auto& w = b->waves[wi];
      const int64_t end = wi + 1 < b->waves.size() ? b->out_off[b->waves[wi + 1].first]
                                                   : b->out_elems;
      wmax = std::max(wmax, oesz * static_cast<size_t>(end - b->out_off[w.first]));
    }
    b->wout_bytes = wmax;
    for (int k = 0; k < 2; ++k) {
      if ((st = alloc(b, &b->d_win[k], esz * static_cast<size_t>(b->p.n_chan) * nt_max)))
        return st;
      if ((st = alloc(b, &b->d_wout[k], wmax))) return st;
      B_CUDA(cudaEventCreateWithFlags(&b->win_free[k], cudaEventDisableTiming));
      for (size_t wi = 0; wi < b->waves.size(); ++wi) {
        auto& w = b->waves[wi];
        std::vector<fdd::BatchSet> sets = w.h_sets, tails = w.h_tail;
        bind_wave(b, sets, tails, w, b->d_wout[k], b->out_off[w.first]);
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
      for (int64_t c = 0; c < b->n_chunks[bm]; ++c)
        if ((st = transform_chunk(b, b->d_win[slot], bm, c, s)) != FDD_OK) return st;
      B_CUDA(cudaEventRecord(b->win_free[slot], s));
      b->win_used[slot] = true;
    }
    const int k = static_cast<int>(b->out_next++ & 1);
    if (b->out_release[k]) {  // the sink's reads of this slot's last wave
      B_CUDA(cudaStreamWaitEvent(s, static_cast<cudaEvent_t>(b->out_release[k]), 0));
      b->out_release[k] = nullptr;
    }
    fdd::BatchSet* d_sets = b->d_sets_slot[k][wi];
    B_CUDA(cudaMemsetAsync(b->d_counter + 2 * wi, 0, 2 * sizeof(unsigned long long), s));
    const int n_sets = static_cast<int>(w.h_sets.size());
    B_CUDA(fdd::launch_mac_batch(d_sets, n_sets, w.n_items, b->d_counter + 2 * wi, b->variant,
                                 b->ctas, b->p.n_chan, s));
    if (w.n_tail_items)
      B_CUDA(fdd::launch_mac_batch(d_sets + n_sets, static_cast<int>(w.h_tail.size()),
                                   w.n_tail_items, b->d_counter + 2 * wi + 1, b->tail_variant,
                                   b->tail_ctas, b->p.n_chan, s));
    const int64_t origin = b->out_off[w.first];
    void* release = nullptr;
    for (int i = 0; i < w.count; ++i) {
      const int bm = w.first + i;
      for (int64_t c = 0; c < b->n_chunks[bm]; ++c) {
        fdd_block blk{bm, 1, c, 0, b->beams[bm].n_dm,
                      static_cast<char*>(b->d_wout[k]) + oesz * (chunk_out(b, bm, c) - origin),
                      b->n_bins[bm], b->n_bins[bm], 0, nullptr};
        st = sink(sink_user, &blk, stream);
        if (st != FDD_OK) return report_error(st, "the output sink failed");
        if (blk.release_event) release = blk.release_event;  // the wave's last one counts
      }
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

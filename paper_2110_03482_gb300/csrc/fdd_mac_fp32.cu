// fdd_mac_fp32.cu -- FP32 phase-rotate-and-sum on CUDA cores (Sect. 2.2,
// Eqs. 4 and 7):
//
//   Y[j][k] = sum_nu W(k, nu, j) X[nu][k],   W = exp(+2 pi i k d(nu, DM_j) / L)
//
// for a uniform trial grid DM_j = DM_0 + j dDM.  The phase of W in cycles is
// k DM_0 c_nu / L + k j dDM c_nu / L with c_nu the per-channel delay rate of
// Eq. 1; both terms are held as exact 64-bit fixed-point fractions of a cycle
// (u_nu, v_nu, computed on the host), so the reduction "modulo one cycle" of
// the phase is exact integer wrap-around and needs no FP64 on the device.
//
// Because the phase is linear in j, the phasor factorises over a split of
// the trial index j = a T + b:
//
//   W(k, nu, aT + b) = Q_a(k, nu) P_b(k, nu),
//   Q_a = exp(2 pi i (k u + k aT v) 2^-64),  P_b = exp(2 pi i k b v 2^-64).
//
// Hence for each bin, Y[aT + b] = sum_nu (X Q_a) P_b is a complex
// (A x N_nu)(N_nu x T) matrix product whose operands are generated on the
// fly.  A warp owns one bin (or a few bins) and a block of A*T trials.  For
// every channel, each lane evaluates a few Z_a = X Q_a and P_b directly from
// the exact phase (MUFU sin/cos, no recurrence), the warp swaps them through
// shared memory, and each lane accumulates an AT x BT register tile with four
// FP32 FMAs per complex multiply-accumulate, the FP32-pipe minimum for 8
// flops.
//
// The arithmetic uses Blackwell's paired FMA (__ffma2_rn: two FMAs per issued
// instruction at the single-FMA pipe rate), pairs running along b:
//   re[a][b:b+2] += (zr, zr)(pr_b, pr_b+1) + (-zi, -zi)(pi_b, pi_b+1)
//   im[a][b:b+2] += (zr, zr)(pi_b, pi_b+1) + (zi, zi)(pr_b, pr_b+1)
// with Z swapped as (zr, zi) pairs and P as planes pr, pi; the broadcast
// pairs are formed in registers.  Two schedules share it: the plain one
// (every warp evaluates its phasors, synchronises, loads and accumulates,
// per channel), used by the smaller tiles, and the warp-specialised one
// below, used by the 2048-trial tile.
// Lanes are numbered lane = ga * GB + gb, so each quarter warp reads a single
// Z row (a broadcast) and GB distinct P rows; the P rows are padded so that
// those reads fall in distinct shared-memory banks.
#include "fdd_device.cuh"
#include "fdd_internal.h"

namespace fdd {
namespace {

using dev::top32_mul;
using dev::unit_phasor;

constexpr int kWarps = 8;
constexpr int kUnroll = 4;  // channels per unrolled group (X loads run one group ahead)

template <int AT_, int BT_, int GA_, int GB_>
struct Geom {
  static constexpr int AT = AT_;        // Z_a values per lane
  static constexpr int BT = BT_;        // P_b values per lane
  static constexpr int GA = GA_;        // lanes along a in a bin group
  static constexpr int GB = GB_;        // lanes along b in a bin group
  static constexpr int G = GA * GB;     // lanes per bin group
  static constexpr int NG = 32 / G;     // bin groups per warp
  static constexpr int AW = GA * AT;    // A: super-steps of the trial block
  static constexpr int TW = GB * BT;    // T: sub-steps of the trial block
  static constexpr int DMS = AW * TW;   // trials per block
  static constexpr int ZGEN = (AW + G - 1) / G;  // Z_a evaluated per lane
  static constexpr int PGEN = (TW + G - 1) / G;  // P_b evaluated per lane
  static_assert(32 % G == 0, "bin group must divide a warp");
};

using G8x8 = Geom<8, 8, 4, 8>;  // 32 x 64 = 2048 trials per bin and warp
using G4x8 = Geom<4, 8, 4, 8>;  // 16 x 64 = 1024
using G4x4 = Geom<4, 4, 2, 4>;  //  8 x 16 =  128, four bins per warp
using G8x8q = Geom<8, 8, 2, 4>; // 16 x 32 =  512, four bins per warp

// ------------------------------------------------- paired-FMA tile, compact swap
// Z swapped as (zr, zi) pairs and P as planes pr, pi; the broadcast pairs
// (zr, zr), (zi, zi), (-zi, -zi) are formed in registers.
template <class Gm>
struct PackedCompact {
  static constexpr int AT = Gm::AT, BT = Gm::BT;
  static constexpr int ZROW = 2 * AT + 4;   // padded a-rows of (zr, zi) pairs
  static constexpr int PSTR = BT + 4;       // padded b-rows of a plane
  static constexpr int ZFL = Gm::GA * ZROW;
  static constexpr int PFL = Gm::GB * PSTR;
  static constexpr int GFL = ZFL + 2 * PFL;
  static_assert(AT % 2 == 0 && BT % 4 == 0, "rows are read as float4");

  struct Ops {
    float zr[AT], zi[AT];
    float2 pr[BT / 2], pi[BT / 2];
  };
  struct Acc {
    float2 re[AT][BT / 2], im[AT][BT / 2];
  };
  static __device__ __forceinline__ void zero(Acc& c) {
#pragma unroll
    for (int i = 0; i < AT; ++i)
#pragma unroll
      for (int j = 0; j < BT / 2; ++j) c.re[i][j] = c.im[i][j] = make_float2(0.f, 0.f);
  }
  static __device__ __forceinline__ int z_off(int a) { return (a / AT) * ZROW + 2 * (a % AT); }
  static __device__ __forceinline__ int p_off(int b) { return ZFL + (b / BT) * PSTR + (b % BT); }
  static __device__ __forceinline__ void put_z(float* grp, int off, float zr, float zi) {
    *reinterpret_cast<float2*>(grp + off) = make_float2(zr, zi);
  }
  static __device__ __forceinline__ void put_p(float* grp, int off, float pr, float pi) {
    grp[off] = pr;
    grp[off + PFL] = pi;
  }
  static __device__ __forceinline__ void load(const float* grp, int ga, int gb, Ops& o) {
    const float4* z = reinterpret_cast<const float4*>(grp + ga * ZROW);
#pragma unroll
    for (int h = 0; h < AT / 2; ++h) {
      const float4 v = z[h];
      o.zr[2 * h] = v.x;
      o.zi[2 * h] = v.y;
      o.zr[2 * h + 1] = v.z;
      o.zi[2 * h + 1] = v.w;
    }
    const float* row = grp + ZFL + gb * PSTR;
#pragma unroll
    for (int h = 0; h < BT / 4; ++h) {
      const float4 r = *reinterpret_cast<const float4*>(row + 4 * h);
      const float4 i = *reinterpret_cast<const float4*>(row + PFL + 4 * h);
      o.pr[2 * h] = make_float2(r.x, r.y);
      o.pr[2 * h + 1] = make_float2(r.z, r.w);
      o.pi[2 * h] = make_float2(i.x, i.y);
      o.pi[2 * h + 1] = make_float2(i.z, i.w);
    }
  }
  static __device__ __forceinline__ void mac(Acc& c, const Ops& o) {
#pragma unroll
    for (int i = 0; i < AT; ++i) {
      const float2 zr = make_float2(o.zr[i], o.zr[i]);
      const float2 zi = make_float2(o.zi[i], o.zi[i]);
      const float2 zn = make_float2(-o.zi[i], -o.zi[i]);
#pragma unroll
      for (int j = 0; j < BT / 2; ++j) {
        c.re[i][j] = __ffma2_rn(zr, o.pr[j], c.re[i][j]);
        c.im[i][j] = __ffma2_rn(zr, o.pi[j], c.im[i][j]);
      }
#pragma unroll
      for (int j = 0; j < BT / 2; ++j) {
        c.re[i][j] = __ffma2_rn(zn, o.pi[j], c.re[i][j]);
        c.im[i][j] = __ffma2_rn(zi, o.pr[j], c.im[i][j]);
      }
    }
  }
  static __device__ __forceinline__ float2 get(const Acc& c, int i, int j) {
    const float2 r = c.re[i][j / 2], m = c.im[i][j / 2];
    return (j & 1) ? make_float2(r.y, m.y) : make_float2(r.x, m.x);
  }
};

template <class Gm, class M>
struct Generator {
  uint32_t mz[Gm::ZGEN], mp[Gm::PGEN];
  int zoff[Gm::ZGEN], poff[Gm::PGEN];
  bool zon[Gm::ZGEN], pon[Gm::PGEN];
  uint32_t ku;

  __device__ __forceinline__ void init(uint32_t k, int lg, int j_first) {
    ku = k;
#pragma unroll
    for (int q = 0; q < Gm::ZGEN; ++q) {
      const int ai = lg + q * Gm::G;
      zon[q] = ai < Gm::AW;
      mz[q] = k * static_cast<uint32_t>(j_first + ai * Gm::TW);
      zoff[q] = M::z_off(ai);
    }
#pragma unroll
    for (int q = 0; q < Gm::PGEN; ++q) {
      const int bi = lg + q * Gm::G;
      pon[q] = bi < Gm::TW;
      mp[q] = k * static_cast<uint32_t>(bi);
      poff[q] = M::p_off(bi);
    }
  }
  __device__ __forceinline__ void run(const PhaseConst& p, float2 x, float* grp) const {
    const uint32_t base = top32_mul(ku, p.u_lo, p.u_hi);
#pragma unroll
    for (int q = 0; q < Gm::ZGEN; ++q) {
      if (zon[q]) {
        const float2 w = unit_phasor(base + top32_mul(mz[q], p.v_lo, p.v_hi));
        M::put_z(grp, zoff[q], x.x * w.x - x.y * w.y, x.x * w.y + x.y * w.x);
      }
    }
#pragma unroll
    for (int q = 0; q < Gm::PGEN; ++q) {
      if (pon[q]) {
        const float2 w = unit_phasor(top32_mul(mp[q], p.v_lo, p.v_hi));
        M::put_p(grp, poff[q], w.x, w.y);
      }
    }
  }
};

// One CTA's block of work: bins (bin_tile * W + warp) * NG + g and trials
// dm_block * DMS + .. of one set of spectra, with the phase table already in
// shared memory (pcs) and the swap area behind it.
template <class Gm, class M, int W>
__device__ __forceinline__ void mac_block(const MacArgs& a, const PhaseConst* pcs,
                                          float* swap_all, int bin_tile, int dm_block,
                                          int series) {
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int g = lane / Gm::G;
  const int lg = lane % Gm::G;
  const int ga = lg / Gm::GB;
  const int gb = lg % Gm::GB;
  const int k = (bin_tile * W + warp) * Gm::NG + g;  // local bin
  const bool k_ok = k < a.n_bins;
  const int kl = k_ok ? k : 0;  // idle groups run local bin 0, store nothing
  const uint32_t ku = static_cast<uint32_t>(a.k_begin + kl);
  const int jblk = dm_block * Gm::DMS;
  const int nc = a.n_chan;

  constexpr int kStage = Gm::NG * M::GFL;  // floats per warp per stage
  float* grp0 = swap_all + warp * 2 * kStage + g * M::GFL;

  Generator<Gm, M> gen;
  gen.init(ku, lg, a.j_begin + jblk);

  const float2* xp = a.X + static_cast<int64_t>(series) * a.x_series_stride + kl;
  const int64_t xs = a.x_chan_stride;
  typename M::Acc acc;
  M::zero(acc);

  float2 xcur[kUnroll];
#pragma unroll
  for (int i = 0; i < kUnroll; ++i) xcur[i] = (i < nc) ? __ldg(xp + i * xs) : make_float2(0.f, 0.f);

  // per channel c: generate(c) -> sync -> load(c) -> MAC(c); two swap stages,
  // so generate(c + 1) writes the stage that load(c - 1) read before the sync
  // that closed channel c.
  int stage = 0;
  for (int c0 = 0; c0 < nc; c0 += kUnroll) {
    float2 xnext[kUnroll];
#pragma unroll
    for (int i = 0; i < kUnroll; ++i) {
      const int c = c0 + kUnroll + i;
      xnext[i] = (c < nc) ? __ldg(xp + c * xs) : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int i = 0; i < kUnroll; ++i) {
      const int c = c0 + i;
      if (c < nc) {
        float* cur = grp0 + stage * kStage;
        typename M::Ops ops;
        gen.run(pcs[c], xcur[i], cur);
        __syncwarp();
        M::load(cur, ga, gb, ops);
        M::mac(acc, ops);
        stage ^= 1;
      }
    }
#pragma unroll
    for (int i = 0; i < kUnroll; ++i) xcur[i] = xnext[i];
  }

  if (!k_ok) return;
  const bool real_only = (a.k_begin + k == a.real_bin_a) || (a.k_begin + k == a.real_bin_b);
#pragma unroll
  for (int ii = 0; ii < Gm::AT; ++ii) {
#pragma unroll
    for (int jj = 0; jj < Gm::BT; ++jj) {
      const int jl = jblk + (ga * Gm::AT + ii) * Gm::TW + gb * Gm::BT + jj;
      if (jl < a.n_dm) {
        const float2 v = M::get(acc, ii, jj);
        const float re = v.x * a.scale;
        const float im = real_only ? 0.f : v.y * a.scale;
        const int64_t o = static_cast<int64_t>(series) * a.y_series_stride +
                          static_cast<int64_t>(jl) * a.y_dm_stride + k;
        if (a.out_kind == 2)
          static_cast<float*>(a.Y)[o] = re * re + im * im;
        else
          static_cast<float2*>(a.Y)[o] = make_float2(re, im);
      }
    }
  }
}

template <class Gm, class M, int W = kWarps>
__global__ void __launch_bounds__(W * 32, 1) mac_kernel(const MacArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  PhaseConst* pcs = reinterpret_cast<PhaseConst*>(smem_raw);
  float* swap_all = reinterpret_cast<float*>(smem_raw + sizeof(PhaseConst) * a.n_chan);
  for (int i = threadIdx.x; i < a.n_chan; i += W * 32) pcs[i] = a.pc[i];
  __syncthreads();
  mac_block<Gm, M, W>(a, pcs, swap_all, blockIdx.x, blockIdx.y, blockIdx.z);
}

// --------------------------------------------- warp-specialised schedule
// The plain schedule makes every warp alternate between the
// latency-bound phasor evaluation (integer phase, MUFU sin/cos, the swap) and
// its block of paired FMAs; with three warps per scheduler the FMA pipe idles
// whenever all of them are evaluating.  Here the two jobs go to different
// warps: kCons consumer warps each own one bin of the CTA's tile and only read
// Z and P from shared memory and accumulate, while kProd producer warps
// evaluate Z_a = X Q_a and P_b for every consumer's bin, kWsCh channels at a
// time, into a ring of kWsStages stages.  A pair of mbarriers per stage orders
// the two sides (full: every producer warp has written the stage; empty:
// every consumer warp has read it; one arrive per warp).  Every wait is
// bounded; a timeout stops both sides and is reported in the status word.
template <class Gm, class M, int kCons, int kProd, int kWsCh = 4, int kWsStages = 3>
struct WsLayout {
  static_assert(Gm::NG == 1, "one bin per consumer warp");
  static_assert(kCons % kProd == 0, "producers share the consumers' bins evenly");
  static constexpr int kBinsPerProd = kCons / kProd;
  static constexpr int kStageFloats = kWsCh * kCons * M::GFL;  // [channel][consumer][GFL]
  // 2 kWsStages mbarriers and the abort flag, rounded up to 16 bytes
  static constexpr size_t kBarBytes = (2 * kWsStages * 8 + 4 + 15) / 16 * 16;
  static constexpr size_t kSwapBytes =
      kBarBytes + sizeof(float) * static_cast<size_t>(kWsStages) * kStageFloats;
  static_assert(2 * kWsStages * 8 + 4 <= kBarBytes, "barrier area");
};

// One work item of the warp-specialised schedule: the CTA's kCons bins
// starting at local bin bin_tile * kCons and the trials dm_block * DMS + ..
// of one set of spectra, with the phase table already in shared memory.
// Stages and barrier phases continue from iteration it0 of the ring (items
// of a persistent CTA follow one another).  Returns false after a timeout.
template <class Gm, class M, int kCons, int kProd, int kWsCh, int kWsStages>
__device__ __forceinline__ bool ws_item(const MacArgs& a, const PhaseConst* pcs, float* stages,
                                        uint64_t* full, uint64_t* empty,
                                        volatile int* abort_flag, int bin_tile, int dm_block,
                                        int series, uint32_t it0) {
  using Ly = WsLayout<Gm, M, kCons, kProd, kWsCh, kWsStages>;
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int n_iter = (a.n_chan + kWsCh - 1) / kWsCh;
  const int jblk = dm_block * Gm::DMS;
  const int k_tile = bin_tile * kCons;  // first local bin of the item
  bool ok = true;

  if (warp >= kCons) {
    // ------------------------------------------------------------ producers
    const int pw = warp - kCons;
    constexpr int NB = Ly::kBinsPerProd;
    Generator<Gm, M> gen[NB];
    const float2* xp[NB];
#pragma unroll
    for (int q = 0; q < NB; ++q) {
      const int k = k_tile + pw * NB + q;
      const int kl = k < a.n_bins ? k : 0;  // idle bins evaluate local bin 0, stored by nobody
      gen[q].init(static_cast<uint32_t>(a.k_begin + kl), lane, a.j_begin + jblk);
      xp[q] = a.X + static_cast<int64_t>(series) * a.x_series_stride + kl;
    }
    const int64_t xs = a.x_chan_stride;
    float2 xn[NB][kWsCh];
#pragma unroll
    for (int q = 0; q < NB; ++q)
#pragma unroll
      for (int ch = 0; ch < kWsCh; ++ch)
        xn[q][ch] = ch < a.n_chan ? __ldg(xp[q] + ch * xs) : make_float2(0.f, 0.f);
    for (int it = 0; it < n_iter; ++it) {
      const uint32_t g = it0 + it;
      const int s = g % kWsStages;
      float2 x[NB][kWsCh];
#pragma unroll
      for (int q = 0; q < NB; ++q)
#pragma unroll
        for (int ch = 0; ch < kWsCh; ++ch) {
          x[q][ch] = xn[q][ch];
          const int c = (it + 1) * kWsCh + ch;  // prefetch the next stage's X
          xn[q][ch] = c < a.n_chan ? __ldg(xp[q] + c * xs) : make_float2(0.f, 0.f);
        }
      ok = __all_sync(0xffffffffu,
                      dev::mbar_wait(&empty[s], ((g / kWsStages) & 1) ^ 1, abort_flag));
      if (!ok) break;
      float* st = stages + s * Ly::kStageFloats + (pw * NB) * M::GFL;
#pragma unroll
      for (int ch = 0; ch < kWsCh; ++ch) {
        const int c = it * kWsCh + ch;
        if (c < a.n_chan) {
          const PhaseConst p = pcs[c];
#pragma unroll
          for (int q = 0; q < NB; ++q) gen[q].run(p, x[q][ch], st + (ch * kCons + q) * M::GFL);
        }
      }
      if (!a.test_withhold) dev::mbar_arrive_warp(&full[s]);
    }
  } else {
    // ------------------------------------------------------------ consumers
    const int k = k_tile + warp;  // local bin
    const int ga = lane / Gm::GB;
    const int gb = lane % Gm::GB;
    typename M::Acc acc;
    M::zero(acc);
    for (int it = 0; it < n_iter; ++it) {
      const uint32_t g = it0 + it;
      const int s = g % kWsStages;
      ok = __all_sync(0xffffffffu, dev::mbar_wait(&full[s], (g / kWsStages) & 1, abort_flag));
      if (!ok) break;
      const float* st = stages + s * Ly::kStageFloats + warp * M::GFL;
      const int nc = a.n_chan - it * kWsCh;
#pragma unroll
      for (int ch = 0; ch < kWsCh; ++ch) {
        if (ch < nc) {
          typename M::Ops ops;
          M::load(st + ch * kCons * M::GFL, ga, gb, ops);
          M::mac(acc, ops);
        }
      }
      dev::mbar_arrive_warp(&empty[s]);
    }
    if (ok && k < a.n_bins) {
      const bool real_only = (a.k_begin + k == a.real_bin_a) || (a.k_begin + k == a.real_bin_b);
#pragma unroll
      for (int ii = 0; ii < Gm::AT; ++ii) {
#pragma unroll
        for (int jj = 0; jj < Gm::BT; ++jj) {
          const int jl = jblk + (ga * Gm::AT + ii) * Gm::TW + gb * Gm::BT + jj;
          if (jl < a.n_dm) {
            const float2 v = M::get(acc, ii, jj);
            const float re = v.x * a.scale;
            const float im = real_only ? 0.f : v.y * a.scale;
            const int64_t o = static_cast<int64_t>(series) * a.y_series_stride +
                              static_cast<int64_t>(jl) * a.y_dm_stride + k;
            if (a.out_kind == 2)
              static_cast<float*>(a.Y)[o] = re * re + im * im;
            else
              static_cast<float2*>(a.Y)[o] = make_float2(re, im);
          }
        }
      }
    }
  }
  if (!ok) {
    *abort_flag = 1;
    if (a.status) atomicExch(a.status, FDD_ERR_TIMEOUT);
  }
  return ok;
}

// Shared-memory carve-up of the warp-specialised kernels: phase table, then
// the barriers and abort flag, then the stages.
template <class Ly>
struct WsSmem {
  PhaseConst* pcs;
  uint64_t* full;
  uint64_t* empty;
  volatile int* abort_flag;
  float* stages;
  template <int kWsStages>
  __device__ __forceinline__ void init(unsigned char* raw, int n_chan, int n_cons_warps,
                                       int n_prod_warps) {
    pcs = reinterpret_cast<PhaseConst*>(raw);
    unsigned char* tail = raw + sizeof(PhaseConst) * n_chan;  // 16-byte aligned
    full = reinterpret_cast<uint64_t*>(tail);
    empty = full + kWsStages;
    abort_flag = reinterpret_cast<volatile int*>(empty + kWsStages);
    stages = reinterpret_cast<float*>(tail + Ly::kBarBytes);
    if (threadIdx.x == 0) {
      for (int i = 0; i < kWsStages; ++i) {
        dev::mbar_init(&full[i], n_prod_warps);  // one arrive per warp
        dev::mbar_init(&empty[i], n_cons_warps);
      }
      *abort_flag = 0;
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
  }
};

template <class Gm, class M, int kCons, int kProd, int kWsCh, int kWsStages>
__global__ void __launch_bounds__((kCons + kProd) * 32, 1) mac_ws_kernel(const MacArgs a) {
  using Ly = WsLayout<Gm, M, kCons, kProd, kWsCh, kWsStages>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  WsSmem<Ly> sm;
  sm.template init<kWsStages>(smem_raw, a.n_chan, kCons, kProd);
  for (int i = threadIdx.x; i < a.n_chan; i += blockDim.x) sm.pcs[i] = a.pc[i];
  __syncthreads();
  ws_item<Gm, M, kCons, kProd, kWsCh, kWsStages>(
      a, sm.pcs, sm.stages, sm.full, sm.empty, sm.abort_flag, blockIdx.x, blockIdx.y, blockIdx.z,
      0u);
}

// Persistent form of the warp-specialised schedule over a batch of spectra
// sets (the batching form): CTAs pull (set, bin tile, trial block) items from
// a global counter, numbered bin-tile-major from each set's item_begin; the
// stage ring runs on across items; the phase table is reloaded when the set
// changes.
template <class Gm, class M, int kCons, int kProd, int kWsCh, int kWsStages>
__global__ void __launch_bounds__((kCons + kProd) * 32, 1)
    mac_ws_batch_kernel(const BatchSet* sets, int n_sets, int64_t n_items,
                        unsigned long long* counter) {
  using Ly = WsLayout<Gm, M, kCons, kProd, kWsCh, kWsStages>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ long long item_s;
  const int n_chan = sets[0].args.n_chan;  // common to the batch
  WsSmem<Ly> sm;
  sm.template init<kWsStages>(smem_raw, n_chan, kCons, kProd);
  int cur = -1;
  uint32_t it0 = 0;
  const uint32_t n_iter = static_cast<uint32_t>((n_chan + kWsCh - 1) / kWsCh);
  while (true) {
    if (threadIdx.x == 0) item_s = static_cast<long long>(atomicAdd(counter, 1ull));
    __syncthreads();  // also: every stage of the previous item has been read
    const long long item = item_s;
    if (item >= n_items || *sm.abort_flag) break;
    int lo = 0, hi = n_sets - 1;  // last set with item_begin <= item
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (sets[mid].item_begin <= item) lo = mid; else hi = mid - 1;
    }
    const BatchSet& bs = sets[lo];
    if (lo != cur) {
      for (int i = threadIdx.x; i < n_chan; i += blockDim.x) sm.pcs[i] = bs.args.pc[i];
      cur = lo;
    }
    __syncthreads();  // phase table ready; item_s read by every thread
    const long long local = item - bs.item_begin;
    ws_item<Gm, M, kCons, kProd, kWsCh, kWsStages>(
        bs.args, sm.pcs, sm.stages, sm.full, sm.empty, sm.abort_flag,
        static_cast<int>(local / bs.n_dm_blocks), static_cast<int>(local % bs.n_dm_blocks), 0,
        it0);
    it0 += n_iter;
  }
}

// Persistent form over a batch of spectra sets of uneven sizes (the batching
// form): CTAs pull work items (set, bin tile, trial block) from a global
// counter; a set's phase table is loaded into shared memory when the set
// changes.  Items of a set are numbered bin-tile-major from item_begin.
template <class Gm, class M, int W = kWarps>
__global__ void __launch_bounds__(W * 32, 1) mac_batch_kernel(const BatchSet* sets, int n_sets,
                                                              int64_t n_items,
                                                              unsigned long long* counter) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ long long item_s;
  const int n_chan = sets[0].args.n_chan;  // common to the batch
  PhaseConst* pcs = reinterpret_cast<PhaseConst*>(smem_raw);
  float* swap_all = reinterpret_cast<float*>(smem_raw + sizeof(PhaseConst) * n_chan);
  int cur = -1;
  while (true) {
    if (threadIdx.x == 0) item_s = static_cast<long long>(atomicAdd(counter, 1ull));
    __syncthreads();
    const long long item = item_s;
    __syncthreads();
    if (item >= n_items) break;
    int lo = 0, hi = n_sets - 1;  // last set with item_begin <= item
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (sets[mid].item_begin <= item) lo = mid; else hi = mid - 1;
    }
    const BatchSet& bs = sets[lo];
    if (lo != cur) {
      for (int i = threadIdx.x; i < n_chan; i += W * 32) pcs[i] = bs.args.pc[i];
      __syncthreads();
      cur = lo;
    }
    const long long local = item - bs.item_begin;
    mac_block<Gm, M, W>(bs.args, pcs, swap_all, static_cast<int>(local / bs.n_dm_blocks),
                               static_cast<int>(local % bs.n_dm_blocks), 0);
    __syncthreads();
  }
}

// --------------------------------------- three-multiplication warp-specialised tile
// The complex multiply-accumulate y += z p needs four real products; with
//   A += zr pr,  B += zi pi,  C += (zr + zi)(pr + pi)
// accumulated instead, Re y = A - B and Im y = C - A - B at the end: three
// real products per complex MAC (Gauss's three-multiplication form).  Its
// FP32 rounding is that of the four-product form to within a few percent
// (every term is of the size of a product of the four-product form).  The
// tile: producer warp q evaluates, for bin q of the CTA's four and each
// channel, the 64 Z_a = X Q_a and 32 P_b of a 2048-trial block (T = 32), as
// planes zr, zi and pr, pi; consumer warps 2q and 2q + 1 own the a's 0..31
// and 32..63 of that bin, each lane a 4 x 8 tile of (a, b) with the three
// accumulators as pairs along b, the sums zr + zi and pr + pi formed in
// registers after the loads (shared-memory traffic per lane as the
// four-product form's, two floats per operand): 48 paired FMAs and 6 paired
// adds per lane and channel for 32 complex MACs.  A stage carries kCh
// channels of full items (16 in use: against 4, a quarter of the barrier
// round trips per channel and longer independent runs of loads and FMAs;
// 0.661, 0.726 and 0.752 of the FP32 peak with 4, 8 and 16 channels on the
// same launch) and kChWide = 8 of wide items, whose per-channel operands
// are up to twice as large.
template <int kCh, int kStages>
struct G3 {
  static constexpr int kA = 64;                // a's per bin (Z_a)
  static constexpr int kT = 32;                // b's per bin (P_b): T
  static constexpr int kDms = kA * kT;         // 2048 trials per bin
  static constexpr int kBins = 4;              // bins per CTA (one producer warp each)
  static constexpr int kCons = 2 * kBins;      // consumer warps
  static constexpr int kProd = kBins;          // producer warps
  static constexpr int kThreads = 32 * (kCons + kProd);
  static constexpr int kGFL = 2 * kA + 2 * kT;  // floats per (bin, channel): zr zi pr pi
  // wide items (a ragged remainder of at most 1024 or 512 trials): the a's
  // 0 .. kAw - 1 (kAw 32 or 16) of 8 x 32 / kAw bins, zr zi (kAw each) and
  // pr pi (32 each) per (bin, channel)
  __host__ __device__ static constexpr int wide_bins(int aw) { return 8 * 32 / aw; }
  __host__ __device__ static constexpr int wide_floats(int aw) { return 2 * aw + 2 * kT; }
  static constexpr int kWideMax = wide_bins(16) * wide_floats(16) > wide_bins(32) * wide_floats(32)
                                      ? wide_bins(16) * wide_floats(16)
                                      : wide_bins(32) * wide_floats(32);
  // channels per stage of the wide items (their per-channel operands are up
  // to twice the full item's, so they fill a stage with fewer channels)
  static constexpr int kChWide = kCh < 8 ? kCh : 8;
  static constexpr int kStageFloats = kCh * kBins * kGFL > kChWide * kWideMax
                                          ? kCh * kBins * kGFL
                                          : kChWide * kWideMax;
  static constexpr size_t kBarBytes = (2 * kStages * 8 + 4 + 15) / 16 * 16;
  static constexpr size_t kSwapBytes = kBarBytes + sizeof(float) * size_t(kStages) * kStageFloats;
};

// One work item of the three-multiplication tile: the CTA's four bins from
// local bin bin_tile * 4 and trials dm_block * 2048 + .. of one set of
// spectra; ring stages and barrier phases continue from iteration it0.
// Returns false after a timeout.
template <int kCh, int kStages>
__device__ __forceinline__ bool g3_body(const MacArgs& a, const PhaseConst* pcs, float* stages,
                                        uint64_t* full, uint64_t* empty,
                                        volatile int* abort_flag, int bin_tile, int dm_block,
                                        int series, uint32_t it0) {
  using Ly = G3<kCh, kStages>;
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int n_iter = (a.n_chan + kCh - 1) / kCh;
  const int jblk = dm_block * Ly::kDms;
  bool ok = true;

  if (warp >= Ly::kCons) {
    // ------------------------------------------------------------ producers
    const int q = warp - Ly::kCons;               // the CTA's bin q
    const int k = bin_tile * Ly::kBins + q;
    const int kl = k < a.n_bins ? k : 0;          // idle bins evaluate local bin 0, unused
    const uint32_t ku = static_cast<uint32_t>(a.k_begin + kl);
    // Phases (units of 2^-32 cycle) of trial j0 + a T + b, j0 the block's
    // first trial: Z_a takes k u + k j0 v + a (T k v) and P_b takes b k v.
    // The lane-independent parts k u + k j0 v and 32 T k v of a channel are
    // evaluated by one lane per channel and broadcast; a lane's own P phase
    // (b = lane) gives its Z phases by a shift and an add (a T k v = T (a k
    // v)), within 33 units of the exact phase.
    const uint32_t m_j0 = ku * static_cast<uint32_t>(a.j_begin + jblk);
    const uint32_t m_d = ku * static_cast<uint32_t>(32 * Ly::kT);
    const uint32_t m_p = ku * static_cast<uint32_t>(lane);
    static_assert(Ly::kT == 32 && kCh <= 32 && (kCh & (kCh - 1)) == 0, "phase layout");
    const float2* xp = a.X + static_cast<int64_t>(series) * a.x_series_stride + kl;
    const int64_t xs = a.x_chan_stride;
    float2 xn[kCh];
#pragma unroll
    for (int ch = 0; ch < kCh; ++ch)
      xn[ch] = ch < a.n_chan ? __ldg(xp + ch * xs) : make_float2(0.f, 0.f);
    for (int it = 0; it < n_iter; ++it) {
      const uint32_t g = it0 + it;
      const int s = g % kStages;
      float2 x[kCh];
#pragma unroll
      for (int ch = 0; ch < kCh; ++ch) {
        x[ch] = xn[ch];
        const int c = (it + 1) * kCh + ch;  // prefetch the next stage's X
        xn[ch] = c < a.n_chan ? __ldg(xp + c * xs) : make_float2(0.f, 0.f);
      }
      ok = __all_sync(0xffffffffu,
                      dev::mbar_wait(&empty[s], ((g / kStages) & 1) ^ 1, abort_flag));
      if (!ok) break;
      float* st = stages + s * Ly::kStageFloats + q * Ly::kGFL;
      // lane l < kCh: the lane-independent phases of channel it kCh + l
      uint32_t ph_a = 0, ph_d = 0;
      {
        const int c = it * kCh + (lane & (kCh - 1));
        if (c < a.n_chan) {
          const PhaseConst p = pcs[c];
          ph_a = top32_mul(ku, p.u_lo, p.u_hi) + top32_mul(m_j0, p.v_lo, p.v_hi);
          ph_d = top32_mul(m_d, p.v_lo, p.v_hi);
        }
      }
#pragma unroll
      for (int ch = 0; ch < kCh; ++ch) {
        const int c = it * kCh + ch;
        const uint32_t pa = __shfl_sync(0xffffffffu, ph_a, ch);
        const uint32_t pd = __shfl_sync(0xffffffffu, ph_d, ch);
        if (c < a.n_chan) {
          const PhaseConst p = pcs[c];
          const uint32_t pp = top32_mul(m_p, p.v_lo, p.v_hi);
          const uint32_t pz0 = pa + (pp << 5);
          const float2 w0 = unit_phasor(pz0);
          const float2 w1 = unit_phasor(pz0 + pd);
          const float2 wp = unit_phasor(pp);
          // Z_lane and Z_lane+32 = X W as pairs
          const float2 xv = x[ch];
          const float2 cw = make_float2(w0.x, w1.x), sw = make_float2(w0.y, w1.y);
          const float2 xr = make_float2(xv.x, xv.x);
          const float2 zr = __ffma2_rn(xr, cw, __fmul2_rn(make_float2(-xv.y, -xv.y), sw));
          const float2 zi = __ffma2_rn(xr, sw, __fmul2_rn(make_float2(xv.y, xv.y), cw));
          float* grp = st + ch * Ly::kBins * Ly::kGFL;
          grp[lane] = zr.x;
          grp[Ly::kA + lane] = zi.x;
          grp[32 + lane] = zr.y;
          grp[Ly::kA + 32 + lane] = zi.y;
          grp[2 * Ly::kA + lane] = wp.x;
          grp[2 * Ly::kA + Ly::kT + lane] = wp.y;
        }
      }
      if (!a.test_withhold) dev::mbar_arrive_warp(&full[s]);
    }
  } else {
    // ------------------------------------------------------------ consumers
    const int q = warp >> 1;                      // the CTA's bin
    const int h = warp & 1;                       // a's 32 h .. 32 h + 31
    const int k = bin_tile * Ly::kBins + q;       // local bin
    const int ga = lane >> 2;                     // a = 32 h + 4 ga + i
    const int gb = lane & 3;                      // b = 8 gb + j
    float2 A[4][4], B[4][4], C[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int m = 0; m < 4; ++m) A[i][m] = B[i][m] = C[i][m] = make_float2(0.f, 0.f);
    for (int it = 0; it < n_iter; ++it) {
      const uint32_t g = it0 + it;
      const int s = g % kStages;
      ok = __all_sync(0xffffffffu, dev::mbar_wait(&full[s], (g / kStages) & 1, abort_flag));
      if (!ok) break;
      const float* st = stages + s * Ly::kStageFloats + q * Ly::kGFL;
      const int nc = a.n_chan - it * kCh;
#pragma unroll
      for (int ch = 0; ch < kCh; ++ch) {
        if (ch < nc) {
          const float* grp = st + ch * Ly::kBins * Ly::kGFL;
          const float4 zr = *reinterpret_cast<const float4*>(grp + 32 * h + 4 * ga);
          const float4 zi = *reinterpret_cast<const float4*>(grp + Ly::kA + 32 * h + 4 * ga);
          const float* pp = grp + 2 * Ly::kA + 8 * gb;
          const float4 pr0 = *reinterpret_cast<const float4*>(pp);
          const float4 pr1 = *reinterpret_cast<const float4*>(pp + 4);
          const float4 pi0 = *reinterpret_cast<const float4*>(pp + Ly::kT);
          const float4 pi1 = *reinterpret_cast<const float4*>(pp + Ly::kT + 4);
          const float2 pr[4] = {make_float2(pr0.x, pr0.y), make_float2(pr0.z, pr0.w),
                                make_float2(pr1.x, pr1.y), make_float2(pr1.z, pr1.w)};
          const float2 pi[4] = {make_float2(pi0.x, pi0.y), make_float2(pi0.z, pi0.w),
                                make_float2(pi1.x, pi1.y), make_float2(pi1.z, pi1.w)};
          float2 ps[4];
#pragma unroll
          for (int m = 0; m < 4; ++m) ps[m] = __fadd2_rn(pr[m], pi[m]);
          const float2 zs01 = __fadd2_rn(make_float2(zr.x, zr.y), make_float2(zi.x, zi.y));
          const float2 zs23 = __fadd2_rn(make_float2(zr.z, zr.w), make_float2(zi.z, zi.w));
          const float zrv[4] = {zr.x, zr.y, zr.z, zr.w};
          const float ziv[4] = {zi.x, zi.y, zi.z, zi.w};
          const float zsv[4] = {zs01.x, zs01.y, zs23.x, zs23.y};
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const float2 r2 = make_float2(zrv[i], zrv[i]);
            const float2 i2 = make_float2(ziv[i], ziv[i]);
            const float2 s2 = make_float2(zsv[i], zsv[i]);
#pragma unroll
            for (int m = 0; m < 4; ++m) {
              A[i][m] = __ffma2_rn(r2, pr[m], A[i][m]);
              B[i][m] = __ffma2_rn(i2, pi[m], B[i][m]);
              C[i][m] = __ffma2_rn(s2, ps[m], C[i][m]);
            }
          }
        }
      }
      dev::mbar_arrive_warp(&empty[s]);
    }
    if (ok && k < a.n_bins) {
      const bool real_only = (a.k_begin + k == a.real_bin_a) || (a.k_begin + k == a.real_bin_b);
#pragma unroll
      for (int i = 0; i < 4; ++i) {
#pragma unroll
        for (int m = 0; m < 4; ++m) {
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            const float av = e ? A[i][m].y : A[i][m].x;
            const float bv = e ? B[i][m].y : B[i][m].x;
            const float cv = e ? C[i][m].y : C[i][m].x;
            const int jl = jblk + (32 * h + 4 * ga + i) * Ly::kT + 8 * gb + 2 * m + e;
            if (jl < a.n_dm) {
              const float re = (av - bv) * a.scale;
              const float im = real_only ? 0.f : (cv - av - bv) * a.scale;
              const int64_t o = static_cast<int64_t>(series) * a.y_series_stride +
                                static_cast<int64_t>(jl) * a.y_dm_stride + k;
              if (a.out_kind == 2)
                static_cast<float*>(a.Y)[o] = re * re + im * im;
              else
                static_cast<float2*>(a.Y)[o] = make_float2(re, im);
            }
          }
        }
      }
    }
  }
  if (!ok) {
    *abort_flag = 1;
    if (a.status) atomicExch(a.status, FDD_ERR_TIMEOUT);
  }
  return ok;
}

// Wide item of the three-multiplication tile: a ragged remainder of at most
// kAw x 32 trials (kAw = 32: 1024, kAw = 16: 512) from trial jw over the
// CTA's 8 x 32 / kAw bins from bin_tile times that: consumer warp w owns
// 32 / kAw of them (kAw / 4 x 4 lanes each, every lane busy), each lane a
// 4 x 8 tile of (a, b) as in the full item; producer warp q evaluates, for its
// quarter of the bins, P_b (b = lane) of each and the kAw Z_a of each (two per
// lane).  Same stage ring and handshake as the full item.
template <int kCh, int kStages, int kAw>
__device__ __forceinline__ bool g3_wide_body(const MacArgs& a, const PhaseConst* pcs,
                                             float* stages, uint64_t* full, uint64_t* empty,
                                             volatile int* abort_flag, int bin_tile, int jw,
                                             int series, uint32_t it0) {
  using Ly = G3<kCh, kStages>;
  constexpr int kC = Ly::kChWide;  // channels per stage
  constexpr int kNB = Ly::wide_bins(kAw);   // bins per CTA
  constexpr int kW = Ly::wide_floats(kAw);  // floats per (bin, channel)
  constexpr int kPB = kNB / Ly::kProd;      // bins per producer warp
  constexpr int kLPB = kAw;                 // lanes per bin in a consumer warp (kAw/4 x 4)
  static_assert(kAw == 32 || kAw == 16, "wide items of 1024 or 512 trials");
  static_assert(kNB == Ly::kCons * 32 / kLPB && 2 * 32 == kPB * kAw, "wide layout");
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int n_iter = (a.n_chan + kC - 1) / kC;
  const int bin0 = bin_tile * kNB;
  bool ok = true;

  if (warp >= Ly::kCons) {
    // ------------------------------------------------------------ producers
    const int q = warp - Ly::kCons;
    uint32_t ku[kPB], m_p[kPB];
    const float2* xp[kPB];
#pragma unroll
    for (int r = 0; r < kPB; ++r) {
      const int k = bin0 + q * kPB + r;
      const int kl = k < a.n_bins ? k : 0;  // idle bins evaluate local bin 0, unused
      ku[r] = static_cast<uint32_t>(a.k_begin + kl);
      m_p[r] = ku[r] * static_cast<uint32_t>(lane);
      xp[r] = a.X + static_cast<int64_t>(series) * a.x_series_stride + kl;
    }
    // the lane's two Z_a: a = lane mod kAw of the warp's bins 32 t / kAw + lane / kAw
    // (bin t for kAw 32; bin 2 t + lane / 16 for kAw 16: chosen by selects)
    const bool hi = kAw == 16 && lane >= 16;
    uint32_t m_z[2], k_z[2];
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      const int r0 = t * (32 / kAw);
      k_z[t] = (kAw == 16 && hi) ? ku[(r0 + 1) % kPB] : ku[r0];
      m_z[t] = k_z[t] * static_cast<uint32_t>(a.j_begin + jw + (lane % kAw) * Ly::kT);
    }
    const int64_t xs = a.x_chan_stride;
    float2 xn[kPB][kC];
#pragma unroll
    for (int r = 0; r < kPB; ++r)
#pragma unroll
      for (int ch = 0; ch < kC; ++ch)
        xn[r][ch] = ch < a.n_chan ? __ldg(xp[r] + ch * xs) : make_float2(0.f, 0.f);
    for (int it = 0; it < n_iter; ++it) {
      const uint32_t g = it0 + it;
      const int s = g % kStages;
      float2 x[kPB][kC];
#pragma unroll
      for (int r = 0; r < kPB; ++r)
#pragma unroll
        for (int ch = 0; ch < kC; ++ch) {
          x[r][ch] = xn[r][ch];
          const int c = (it + 1) * kC + ch;  // prefetch the next stage's X
          xn[r][ch] = c < a.n_chan ? __ldg(xp[r] + c * xs) : make_float2(0.f, 0.f);
        }
      ok = __all_sync(0xffffffffu,
                      dev::mbar_wait(&empty[s], ((g / kStages) & 1) ^ 1, abort_flag));
      if (!ok) break;
      float* st = stages + s * Ly::kStageFloats;
#pragma unroll
      for (int ch = 0; ch < kC; ++ch) {
        const int c = it * kC + ch;
        if (c < a.n_chan) {
          const PhaseConst p = pcs[c];
#pragma unroll
          for (int r = 0; r < kPB; ++r) {
            const float2 wp = unit_phasor(top32_mul(m_p[r], p.v_lo, p.v_hi));
            float* grp = st + (ch * kNB + q * kPB + r) * kW;
            grp[2 * kAw + lane] = wp.x;
            grp[2 * kAw + 32 + lane] = wp.y;
          }
#pragma unroll
          for (int t = 0; t < 2; ++t) {
            const int r0 = t * (32 / kAw);
            const int r = hi ? r0 + 1 : r0;
            const float2 xv = (kAw == 16 && hi) ? x[(r0 + 1) % kPB][ch] : x[r0][ch];
            const float2 w = unit_phasor(top32_mul(k_z[t], p.u_lo, p.u_hi) +
                                         top32_mul(m_z[t], p.v_lo, p.v_hi));
            float* grp = st + (ch * kNB + q * kPB + r) * kW;
            const int ai = lane % kAw;
            grp[ai] = xv.x * w.x - xv.y * w.y;
            grp[kAw + ai] = xv.x * w.y + xv.y * w.x;
          }
        }
      }
      if (!a.test_withhold) dev::mbar_arrive_warp(&full[s]);
    }
  } else {
    // ------------------------------------------------------------ consumers
    const int wb = warp * (32 / kLPB) + lane / kLPB;  // the lane's bin in the CTA
    const int k = bin0 + wb;                          // local bin
    const int ll = lane % kLPB;
    const int ga = ll >> 2;  // a = 4 ga + i
    const int gb = ll & 3;   // b = 8 gb + j
    float2 A[4][4], B[4][4], C[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int m = 0; m < 4; ++m) A[i][m] = B[i][m] = C[i][m] = make_float2(0.f, 0.f);
    for (int it = 0; it < n_iter; ++it) {
      const uint32_t g = it0 + it;
      const int s = g % kStages;
      ok = __all_sync(0xffffffffu, dev::mbar_wait(&full[s], (g / kStages) & 1, abort_flag));
      if (!ok) break;
      const int nc = a.n_chan - it * kC;
#pragma unroll
      for (int ch = 0; ch < kC; ++ch) {
        if (ch < nc) {
          const float* grp = stages + s * Ly::kStageFloats + (ch * kNB + wb) * kW;
          const float4 zr = *reinterpret_cast<const float4*>(grp + 4 * ga);
          const float4 zi = *reinterpret_cast<const float4*>(grp + kAw + 4 * ga);
          const float4 pr0 = *reinterpret_cast<const float4*>(grp + 2 * kAw + 8 * gb);
          const float4 pr1 = *reinterpret_cast<const float4*>(grp + 2 * kAw + 8 * gb + 4);
          const float4 pi0 = *reinterpret_cast<const float4*>(grp + 2 * kAw + 32 + 8 * gb);
          const float4 pi1 = *reinterpret_cast<const float4*>(grp + 2 * kAw + 32 + 8 * gb + 4);
          const float2 pr[4] = {make_float2(pr0.x, pr0.y), make_float2(pr0.z, pr0.w),
                                make_float2(pr1.x, pr1.y), make_float2(pr1.z, pr1.w)};
          const float2 pi[4] = {make_float2(pi0.x, pi0.y), make_float2(pi0.z, pi0.w),
                                make_float2(pi1.x, pi1.y), make_float2(pi1.z, pi1.w)};
          float2 ps[4];
#pragma unroll
          for (int m = 0; m < 4; ++m) ps[m] = __fadd2_rn(pr[m], pi[m]);
          const float2 zs01 = __fadd2_rn(make_float2(zr.x, zr.y), make_float2(zi.x, zi.y));
          const float2 zs23 = __fadd2_rn(make_float2(zr.z, zr.w), make_float2(zi.z, zi.w));
          const float zrv[4] = {zr.x, zr.y, zr.z, zr.w};
          const float ziv[4] = {zi.x, zi.y, zi.z, zi.w};
          const float zsv[4] = {zs01.x, zs01.y, zs23.x, zs23.y};
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const float2 r2 = make_float2(zrv[i], zrv[i]);
            const float2 i2 = make_float2(ziv[i], ziv[i]);
            const float2 s2 = make_float2(zsv[i], zsv[i]);
#pragma unroll
            for (int m = 0; m < 4; ++m) {
              A[i][m] = __ffma2_rn(r2, pr[m], A[i][m]);
              B[i][m] = __ffma2_rn(i2, pi[m], B[i][m]);
              C[i][m] = __ffma2_rn(s2, ps[m], C[i][m]);
            }
          }
        }
      }
      dev::mbar_arrive_warp(&empty[s]);
    }
    if (ok && k < a.n_bins) {
      const bool real_only = (a.k_begin + k == a.real_bin_a) || (a.k_begin + k == a.real_bin_b);
#pragma unroll
      for (int i = 0; i < 4; ++i) {
#pragma unroll
        for (int m = 0; m < 4; ++m) {
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            const float av = e ? A[i][m].y : A[i][m].x;
            const float bv = e ? B[i][m].y : B[i][m].x;
            const float cv = e ? C[i][m].y : C[i][m].x;
            const int jl = jw + (4 * ga + i) * Ly::kT + 8 * gb + 2 * m + e;
            if (jl < a.n_dm) {
              const float re = (av - bv) * a.scale;
              const float im = real_only ? 0.f : (cv - av - bv) * a.scale;
              const int64_t o = static_cast<int64_t>(series) * a.y_series_stride +
                                static_cast<int64_t>(jl) * a.y_dm_stride + k;
              if (a.out_kind == 2)
                static_cast<float*>(a.Y)[o] = re * re + im * im;
              else
                static_cast<float2*>(a.Y)[o] = make_float2(re, im);
            }
          }
        }
      }
    }
  }
  if (!ok) {
    *abort_flag = 1;
    if (a.status) atomicExch(a.status, FDD_ERR_TIMEOUT);
  }
  return ok;
}

// A grid item of the three-multiplication tile: a full item, or for a last
// block of at most 1024 (512) trials a wide item over twice (four times) the
// bins (the grid's bin tiles beyond the wide ones have nothing to do and
// leave at once).
template <int kCh, int kStages>
__device__ __forceinline__ bool g3_item(const MacArgs& a, const PhaseConst* pcs, float* stages,
                                        uint64_t* full, uint64_t* empty,
                                        volatile int* abort_flag, int bin_tile, int dm_block,
                                        int series, uint32_t it0) {
  using Ly = G3<kCh, kStages>;
  const int jblk = dm_block * Ly::kDms;
  const int rem = a.n_dm - jblk;
  if (rem <= Ly::kDms / 4) {
    if (bin_tile * Ly::wide_bins(16) >= a.n_bins) return true;
    return g3_wide_body<kCh, kStages, 16>(a, pcs, stages, full, empty, abort_flag, bin_tile,
                                          jblk, series, it0);
  }
  if (rem <= Ly::kDms / 2) {
    if (bin_tile * Ly::wide_bins(32) >= a.n_bins) return true;
    return g3_wide_body<kCh, kStages, 32>(a, pcs, stages, full, empty, abort_flag, bin_tile,
                                          jblk, series, it0);
  }
  return g3_body<kCh, kStages>(a, pcs, stages, full, empty, abort_flag, bin_tile, dm_block,
                               series, it0);
}

template <int kCh, int kStages>
__global__ void __launch_bounds__(G3<kCh, kStages>::kThreads, 1) mac_g3_kernel(const MacArgs a) {
  using Ly = G3<kCh, kStages>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  WsSmem<Ly> sm;
  sm.template init<kStages>(smem_raw, a.n_chan, Ly::kCons, Ly::kProd);
  for (int i = threadIdx.x; i < a.n_chan; i += blockDim.x) sm.pcs[i] = a.pc[i];
  __syncthreads();
  g3_item<kCh, kStages>(a, sm.pcs, sm.stages, sm.full, sm.empty, sm.abort_flag, blockIdx.x,
                        blockIdx.y, blockIdx.z, 0u);
}

// Persistent form of the three-multiplication tile over a batch of spectra
// sets (the batching form), as mac_ws_batch_kernel.
template <int kCh, int kStages>
__global__ void __launch_bounds__(G3<kCh, kStages>::kThreads, 1)
    mac_g3_batch_kernel(const BatchSet* sets, int n_sets, int64_t n_items,
                        unsigned long long* counter) {
  using Ly = G3<kCh, kStages>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ long long item_s;
  const int n_chan = sets[0].args.n_chan;  // common to the batch
  WsSmem<Ly> sm;
  sm.template init<kStages>(smem_raw, n_chan, Ly::kCons, Ly::kProd);
  int cur = -1;
  uint32_t it0 = 0;
  const uint32_t n_iter = static_cast<uint32_t>((n_chan + kCh - 1) / kCh);
  const uint32_t n_iter_wide =
      static_cast<uint32_t>((n_chan + Ly::kChWide - 1) / Ly::kChWide);
  while (true) {
    if (threadIdx.x == 0) item_s = static_cast<long long>(atomicAdd(counter, 1ull));
    __syncthreads();  // also: every stage of the previous item has been read
    const long long item = item_s;
    if (item >= n_items || *sm.abort_flag) break;
    int lo = 0, hi = n_sets - 1;  // last set with item_begin <= item
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (sets[mid].item_begin <= item) lo = mid; else hi = mid - 1;
    }
    const BatchSet& bs = sets[lo];
    if (lo != cur) {
      for (int i = threadIdx.x; i < n_chan; i += blockDim.x) sm.pcs[i] = bs.args.pc[i];
      cur = lo;
    }
    __syncthreads();  // phase table ready; item_s read by every thread
    const long long local = item - bs.item_begin;
    const long long n_full = static_cast<long long>(bs.n_bin_tiles) * bs.n_dm_blocks;
    // the set's arguments as a local copy: the item's loops then keep what
    // they use in registers instead of re-reading the set after each store
    const MacArgs args = bs.args;
    const bool full_item = local < n_full;
    if (full_item)
      g3_body<kCh, kStages>(args, sm.pcs, sm.stages, sm.full, sm.empty, sm.abort_flag,
                            static_cast<int>(local / bs.n_dm_blocks),
                            static_cast<int>(local % bs.n_dm_blocks), 0, it0);
    else if (local < n_full + bs.n_wide_tiles)
      g3_wide_body<kCh, kStages, 32>(args, sm.pcs, sm.stages, sm.full, sm.empty,
                                     sm.abort_flag, static_cast<int>(local - n_full), bs.j_wide,
                                     0, it0);
    else
      g3_wide_body<kCh, kStages, 16>(args, sm.pcs, sm.stages, sm.full, sm.empty,
                                     sm.abort_flag,
                                     static_cast<int>(local - n_full - bs.n_wide_tiles),
                                     bs.j_narrow, 0, it0);
    it0 += full_item ? n_iter : n_iter_wide;  // stages this item used
  }
}

// ----------------------------------------------------------------- variants
struct VariantInfo {
  const void* fn;
  int dms;
  int ng;
  size_t swap_bytes;  // per CTA, excluding the phase-constant table
  int warps = kWarps;
  const void* batch_fn = nullptr;  // persistent batch kernel of the same tile
  int bin_warps = 0;  // warps that own bins (0: all of them)
  int bins() const { return (bin_warps ? bin_warps : warps) * ng; }
};

template <class Gm, class M, int W = kWarps>
VariantInfo info() {
  return {reinterpret_cast<const void*>(&mac_kernel<Gm, M, W>), Gm::DMS, Gm::NG,
          sizeof(float) * static_cast<size_t>(W) * 2 * Gm::NG * M::GFL, W,
          reinterpret_cast<const void*>(&mac_batch_kernel<Gm, M, W>)};
}

template <class Gm, class M, int kCons, int kProd, int kCh = 4, int kSt = 3>
VariantInfo info_ws() {
  using Ly = WsLayout<Gm, M, kCons, kProd, kCh, kSt>;
  VariantInfo vi{reinterpret_cast<const void*>(&mac_ws_kernel<Gm, M, kCons, kProd, kCh, kSt>),
                 Gm::DMS, Gm::NG, Ly::kSwapBytes, kCons + kProd,
                 reinterpret_cast<const void*>(&mac_ws_batch_kernel<Gm, M, kCons, kProd, kCh, kSt>)};
  vi.bin_warps = kCons;
  return vi;
}

template <int kCh, int kSt>
VariantInfo info_g3() {
  using Ly = G3<kCh, kSt>;
  VariantInfo vi{reinterpret_cast<const void*>(&mac_g3_kernel<kCh, kSt>), Ly::kDms, 1,
                 Ly::kSwapBytes, Ly::kCons + Ly::kProd,
                 reinterpret_cast<const void*>(&mac_g3_batch_kernel<kCh, kSt>)};
  vi.bin_warps = Ly::kBins;
  return vi;
}

// The G12 tile keeps three ring stages while the channels' phase table leaves
// room for them in a CTA's 227 KB and drops to two beyond that (up to 8381
// channels).  One plain launch runs as fast with two as with three; the
// persistent batch kernel, whose items follow one another in the same ring,
// lost 5 % with two.
constexpr size_t kMaxSmem = 227 * 1024;

VariantInfo variant_info(int v, int n_chan) {
  switch (v) {
    case MAC_G12_4x8:
      return sizeof(PhaseConst) * static_cast<size_t>(n_chan) + G3<16, 3>::kSwapBytes <= kMaxSmem
                 ? info_g3<16, 3>()
                 : info_g3<16, 2>();
    case MAC_Q12_8x8: return info<G8x8, PackedCompact<G8x8>, 12>();
    case MAC_Q_4x8: return info<G4x8, PackedCompact<G4x8>>();
    case MAC_Q_8x8_512: return info<G8x8q, PackedCompact<G8x8q>>();
    case MAC_Q_4x4: return info<G4x4, PackedCompact<G4x4>>();
    default: return info_ws<G8x8, PackedCompact<G8x8>, 8, 4>();  // MAC_W12_8x8
  }
}

}  // namespace

// Default tile for a trial count: the one with the least time for the padded
// trial blocks, ceil(n_dm / block) * block / rate, with each tile's rate
// measured kernel-only on GB300 (fraction of the FP32 peak, 1024 channels,
// 131073 bins): G12_4x8 0.752 on full 2048-trial blocks, whose last block
// runs as 1024-trial wide items at 0.616 (at most 1024 trials) or 512-trial
// ones at 0.510 (at most 512); Q_4x8 0.493 (1024-trial blocks), Q_8x8_512
// 0.415 (512), Q_4x4 0.347 (128).  (The four-product warp-specialised tile
// W12_8x8 measured 0.621 on the same launch, Q12_8x8, the 2048-trial tile on
// the plain schedule, 0.553.)
int mac_variant_for(int n_dm, int n_chan) {
  struct Tile {
    int variant, block;
    double rate, wide_rate, narrow_rate;  // > 0: a last block of <= block / 2, / 4
  };
  static const Tile tiles[] = {{MAC_G12_4x8, 2048, 0.752, 0.616, 0.510},
                               {MAC_Q_4x8, 1024, 0.493, 0.0, 0.0},
                               {MAC_Q_8x8_512, 512, 0.415, 0.0, 0.0},
                               {MAC_Q_4x4, 128, 0.347, 0.0, 0.0}};
  int best = MAC_W12_8x8;  // (the smallest shared-memory need of the 2048-trial tiles)
  double best_cost = 0.0;
  for (const Tile& t : tiles) {
    if (mac_smem_bytes(t.variant, n_chan) > kMaxSmem) continue;
    const int full = n_dm / t.block, rem = n_dm % t.block;
    double cost = full * t.block / t.rate;
    if (rem > 0 && t.narrow_rate > 0.0 && rem <= t.block / 4)
      cost += (t.block / 4) / t.narrow_rate;
    else if (rem > 0 && t.wide_rate > 0.0 && rem <= t.block / 2)
      cost += (t.block / 2) / t.wide_rate;
    else if (rem > 0)
      cost += t.block / t.rate;
    if (best_cost == 0.0 || cost < best_cost) {
      best = t.variant;
      best_cost = cost;
    }
  }
  return best;
}

int mac_variant_trials_per_block(int variant) { return variant_info(variant, 1).dms; }

size_t mac_smem_bytes(int variant, int n_chan) {
  return sizeof(PhaseConst) * static_cast<size_t>(n_chan) + variant_info(variant, n_chan).swap_bytes;
}

cudaError_t mac_prepare(int variant, int n_chan) {
  const VariantInfo vi = variant_info(variant, n_chan);
  const int bytes = static_cast<int>(mac_smem_bytes(variant, n_chan));
  cudaError_t e = cudaFuncSetAttribute(vi.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess || !vi.batch_fn) return e;
  return cudaFuncSetAttribute(vi.batch_fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

int mac_variant_bins_per_cta(int variant) { return variant_info(variant, 1).bins(); }

bool mac_variant_batchable(int variant) { return variant_info(variant, 1).batch_fn != nullptr; }

int mac_batch_ctas_per_sm(int variant, int n_chan) {
  const VariantInfo vi = variant_info(variant, n_chan);
  if (!vi.batch_fn) return 0;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, vi.batch_fn, vi.warps * 32,
                                                    mac_smem_bytes(variant, n_chan)) !=
      cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

cudaError_t launch_mac_batch(const BatchSet* d_sets, int n_sets, long long n_items,
                             unsigned long long* d_counter, int variant, int n_ctas, int n_chan,
                             cudaStream_t s) {
  const VariantInfo vi = variant_info(variant, n_chan);
  if (!vi.batch_fn) return cudaErrorInvalidValue;
  if (n_items <= 0) return cudaSuccess;
  void* params[] = {&d_sets, &n_sets, &n_items, &d_counter};
  note_launches(1);
  return cudaLaunchKernel(vi.batch_fn, dim3(n_ctas), dim3(vi.warps * 32), params,
                          mac_smem_bytes(variant, n_chan), s);
}

cudaError_t launch_mac_fp32(const MacArgs& a, int variant, cudaStream_t s) {
  if (a.n_dm <= 0 || a.n_series <= 0 || a.n_bins <= 0) return cudaSuccess;
  const VariantInfo vi = variant_info(variant, a.n_chan);
  const int bins_per_cta = vi.bins();
  dim3 grid((a.n_bins + bins_per_cta - 1) / bins_per_cta, (a.n_dm + vi.dms - 1) / vi.dms,
            a.n_series);
  if (grid.y > 65535u || grid.z > 65535u) return cudaErrorInvalidConfiguration;
  MacArgs args = a;
  void* params[] = {&args};
  note_launches(1);
  return cudaLaunchKernel(vi.fn, grid, dim3(vi.warps * 32), params,
                          mac_smem_bytes(variant, a.n_chan), s);
}

}  // namespace fdd

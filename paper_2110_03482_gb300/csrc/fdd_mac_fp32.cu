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
// every channel, each lane evaluates a few Q_a, P_b directly from the exact
// phase (MUFU sin/cos, no recurrence), the warp swaps them through shared
// memory, and each lane accumulates an AT x BT register tile with four FFMA
// per complex multiply-accumulate, the FP32-pipe minimum for 8 flops.
#include "fdd_internal.h"

namespace fdd {
namespace {

constexpr int kWarps = 8;
constexpr int kThreads = kWarps * 32;
constexpr int kPrefetch = 4;  // channels of X kept in flight per lane

template <int AT_, int BT_, int GA_, int GB_>
struct Tile {
  static constexpr int AT = AT_;            // Q_a values per lane
  static constexpr int BT = BT_;            // P_b values per lane
  static constexpr int GA = GA_;            // lanes along a in a bin group
  static constexpr int GB = GB_;            // lanes along b in a bin group
  static constexpr int G = GA * GB;         // lanes per bin group
  static constexpr int NG = 32 / G;         // bin groups per warp
  static constexpr int AW = GA * AT;        // A: super-steps of the trial block
  static constexpr int TW = GB * BT;        // T: sub-steps of the trial block
  static constexpr int DMS = AW * TW;       // trials per block
  static constexpr int ZROW = AT + 2;       // padded rows (float2) of the swap area
  static constexpr int PROW = BT + 2;
  static constexpr int ZSZ = GA * ZROW;     // float2 per group per stage
  static constexpr int PSZ = GB * PROW;
  static constexpr int GSZ = ZSZ + PSZ;
  static constexpr int XCH = NG * GSZ;      // float2 per warp per stage
  static constexpr int ZGEN = (AW + G - 1) / G;  // Q_a evaluated per lane
  static constexpr int PGEN = (TW + G - 1) / G;  // P_b evaluated per lane
  static_assert(32 % G == 0, "bin group must divide a warp");
  static_assert(AT % 2 == 0 && BT % 2 == 0, "tiles are read as float4 pairs");
};

using TileV8x8 = Tile<8, 8, 4, 8>;  // 32 x 64 = 2048 trials per bin and warp
using TileV4x8 = Tile<4, 8, 4, 8>;  // 16 x 64 = 1024
using TileV4x4 = Tile<4, 4, 2, 4>;  //  8 x 16 =  128, four bins per warp

// Top 32 bits of (m * (hi:lo)) mod 2^64, without the carry of the low word
// (an error of at most 2^-32 cycle).
__device__ __forceinline__ uint32_t top32_mul(uint32_t m, uint32_t lo, uint32_t hi) {
  return __umulhi(m, lo) + m * hi;
}

// Unit phasor of a phase given in units of 2^-32 cycle.  Read as a signed
// integer the phase lies in [-1/2, 1/2) cycle, i.e. [-pi, pi) radians, the
// range in which the hardware sine/cosine are accurate to about 2^-21.
__device__ __forceinline__ float2 unit_phasor(uint32_t phase) {
  const float x = __int2float_rn(static_cast<int>(phase)) * 1.46291807926715968e-9f;  // 2pi/2^32
  float s, c;
  __sincosf(x, &s, &c);
  return make_float2(c, s);
}

template <class T>
__global__ void __launch_bounds__(kThreads, 1) mac_fp32_kernel(const MacArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  PhaseConst* pcs = reinterpret_cast<PhaseConst*>(smem_raw);
  float2* swap_all = reinterpret_cast<float2*>(smem_raw + sizeof(PhaseConst) * a.n_chan);

  for (int i = threadIdx.x; i < a.n_chan; i += kThreads) pcs[i] = a.pc[i];
  __syncthreads();

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int g = lane / T::G;
  const int lg = lane % T::G;
  const int ga = lg / T::GB;
  const int gb = lg % T::GB;
  const int k = (blockIdx.x * kWarps + warp) * T::NG + g;
  const bool k_ok = k < a.n_bins;
  const uint32_t ku = k_ok ? static_cast<uint32_t>(k) : 0u;  // idle groups compute bin 0, store nothing
  const int jblk = blockIdx.y * T::DMS;
  const int series = blockIdx.z;

  float2* swap0 = swap_all + warp * 2 * T::XCH + g * T::GSZ;

  // Generation duties of this lane: Q_a for a = lg + q G, P_b for b = lg + q G.
  uint32_t mz[T::ZGEN];
  int zoff[T::ZGEN];
  bool zon[T::ZGEN];
#pragma unroll
  for (int q = 0; q < T::ZGEN; ++q) {
    const int ai = lg + q * T::G;
    zon[q] = ai < T::AW;
    mz[q] = ku * static_cast<uint32_t>(a.j_begin + jblk + ai * T::TW);
    zoff[q] = (ai / T::AT) * T::ZROW + (ai % T::AT);
  }
  uint32_t mp[T::PGEN];
  int poff[T::PGEN];
  bool pon[T::PGEN];
#pragma unroll
  for (int q = 0; q < T::PGEN; ++q) {
    const int bi = lg + q * T::G;
    pon[q] = bi < T::TW;
    mp[q] = ku * static_cast<uint32_t>(bi);
    poff[q] = T::ZSZ + (bi / T::BT) * T::PROW + (bi % T::BT);
  }

  const float2* xp = a.X + static_cast<int64_t>(series) * a.x_series_stride + ku;
  const int64_t xs = a.x_chan_stride;

  float acc_re[T::AT][T::BT];
  float acc_im[T::AT][T::BT];
#pragma unroll
  for (int i = 0; i < T::AT; ++i)
#pragma unroll
    for (int j = 0; j < T::BT; ++j) {
      acc_re[i][j] = 0.f;
      acc_im[i][j] = 0.f;
    }

  float2 xnext[kPrefetch];
#pragma unroll
  for (int i = 0; i < kPrefetch; ++i)
    xnext[i] = (i < a.n_chan) ? __ldg(xp + i * xs) : make_float2(0.f, 0.f);

  int stage = 0;
  for (int c0 = 0; c0 < a.n_chan; c0 += kPrefetch) {
    float2 xcur[kPrefetch];
#pragma unroll
    for (int i = 0; i < kPrefetch; ++i) {
      xcur[i] = xnext[i];
      const int cn = c0 + kPrefetch + i;
      xnext[i] = (cn < a.n_chan) ? __ldg(xp + cn * xs) : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int i = 0; i < kPrefetch; ++i) {
      const int c = c0 + i;
      if (c < a.n_chan) {
        const PhaseConst p = pcs[c];
        const uint32_t base = top32_mul(ku, p.u_lo, p.u_hi);
        float2* buf = swap0 + stage * T::XCH;
#pragma unroll
        for (int q = 0; q < T::ZGEN; ++q) {
          if (zon[q]) {
            const float2 w = unit_phasor(base + top32_mul(mz[q], p.v_lo, p.v_hi));
            const float2 x = xcur[i];
            buf[zoff[q]] = make_float2(x.x * w.x - x.y * w.y, x.x * w.y + x.y * w.x);
          }
        }
#pragma unroll
        for (int q = 0; q < T::PGEN; ++q)
          if (pon[q]) buf[poff[q]] = unit_phasor(top32_mul(mp[q], p.v_lo, p.v_hi));
        __syncwarp();

        float zr[T::AT], zi[T::AT], pr[T::BT], pi[T::BT];
        const float4* zrow = reinterpret_cast<const float4*>(buf + ga * T::ZROW);
        const float4* prow = reinterpret_cast<const float4*>(buf + T::ZSZ + gb * T::PROW);
#pragma unroll
        for (int h = 0; h < T::AT / 2; ++h) {
          const float4 v = zrow[h];
          zr[2 * h] = v.x;
          zi[2 * h] = v.y;
          zr[2 * h + 1] = v.z;
          zi[2 * h + 1] = v.w;
        }
#pragma unroll
        for (int h = 0; h < T::BT / 2; ++h) {
          const float4 v = prow[h];
          pr[2 * h] = v.x;
          pi[2 * h] = v.y;
          pr[2 * h + 1] = v.z;
          pi[2 * h + 1] = v.w;
        }
#pragma unroll
        for (int ii = 0; ii < T::AT; ++ii)
#pragma unroll
          for (int jj = 0; jj < T::BT; ++jj) {
            acc_re[ii][jj] = fmaf(zr[ii], pr[jj], acc_re[ii][jj]);
            acc_re[ii][jj] = fmaf(-zi[ii], pi[jj], acc_re[ii][jj]);
            acc_im[ii][jj] = fmaf(zr[ii], pi[jj], acc_im[ii][jj]);
            acc_im[ii][jj] = fmaf(zi[ii], pr[jj], acc_im[ii][jj]);
          }
        stage ^= 1;
      }
    }
  }

  if (!k_ok) return;
  const bool real_only = (k == a.real_bin_a) || (k == a.real_bin_b);
#pragma unroll
  for (int ii = 0; ii < T::AT; ++ii) {
#pragma unroll
    for (int jj = 0; jj < T::BT; ++jj) {
      const int jl = jblk + (ga * T::AT + ii) * T::TW + gb * T::BT + jj;
      if (jl < a.n_dm) {
        const float re = acc_re[ii][jj] * a.scale;
        const float im = real_only ? 0.f : acc_im[ii][jj] * a.scale;
        const int64_t off = static_cast<int64_t>(series) * a.y_series_stride +
                            static_cast<int64_t>(jl) * a.y_dm_stride + k;
        if (a.out_kind == 2)
          static_cast<float*>(a.Y)[off] = re * re + im * im;
        else
          static_cast<float2*>(a.Y)[off] = make_float2(re, im);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Packed form.  The same factorised product, with the MAC issued as Blackwell's
// paired FP32 FMA (fma.rn.f32x2): two FMAs per issued instruction at the
// FMA-pipe rate of single FFMAs, so the phasor evaluation, the shared-memory
// swap and the loads issue in the slots the MAC leaves free.  Pairs run along
// b: acc_re[a][b:b+2] += (zr, zr)(pr_b, pr_b+1) + (zi, zi)(-pi_b, -pi_b+1) and
// acc_im[a][b:b+2] += (zr, zr)(pi_b, pi_b+1) + (zi, zi)(pr_b, pr_b+1), so the
// swap area holds Z as (zr, zr, zi, zi) quads and P as three planes
// (pr, pi, -pi).  Rows are padded so that the writes of a quarter warp and
// the reads of the eight b-groups fall in distinct banks.
typedef unsigned long long u64;

// Two spellings of the paired FMA: inline PTX on 64-bit registers, and the
// compiler builtin on float2.
struct PairAsm {
  typedef u64 pair;
  typedef ulonglong2 quad;
  static __device__ __forceinline__ pair zero() { return 0ull; }
  static __device__ __forceinline__ pair fma(pair a, pair b, pair c) {
    pair d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
  }
  static __device__ __forceinline__ pair lo(quad q) { return q.x; }
  static __device__ __forceinline__ pair hi(quad q) { return q.y; }
  static __device__ __forceinline__ float2 split(pair v) {
    float2 r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
    return r;
  }
};

struct PairBuiltin {
  typedef float2 pair;
  typedef float4 quad;
  static __device__ __forceinline__ pair zero() { return make_float2(0.f, 0.f); }
  static __device__ __forceinline__ pair fma(pair a, pair b, pair c) { return __ffma2_rn(a, b, c); }
  static __device__ __forceinline__ pair lo(quad q) { return make_float2(q.x, q.y); }
  static __device__ __forceinline__ pair hi(quad q) { return make_float2(q.z, q.w); }
  static __device__ __forceinline__ float2 split(pair v) { return v; }
};

template <int AT_, int BT_, int GA_, int GB_>
struct Tile2 {
  static constexpr int AT = AT_, BT = BT_, GA = GA_, GB = GB_;
  static constexpr int G = GA * GB;
  static constexpr int NG = 32 / G;
  static constexpr int AW = GA * AT;
  static constexpr int TW = GB * BT;
  static constexpr int DMS = AW * TW;
  static constexpr int ZG = AT + 1;           // Z quads per a-group row (one quad of padding)
  static constexpr int ZFL = GA * ZG * 4;     // floats of the Z area
  static constexpr int PSTR = BT + 4;         // floats per b-group row of a P plane
  static constexpr int PFL = GB * PSTR;       // floats per P plane
  static constexpr int GFL = ZFL + 3 * PFL;   // floats per group per stage
  static constexpr int XFL = NG * GFL;        // floats per warp per stage
  static constexpr int ZGEN = (AW + G - 1) / G;
  static constexpr int PGEN = (TW + G - 1) / G;
  static_assert(32 % G == 0, "bin group must divide a warp");
  static_assert(BT % 4 == 0, "P rows are read as float4");
};

using Tile2V8x8 = Tile2<8, 8, 4, 8>;  // 32 x 64 = 2048 trials per bin and warp
using Tile2V4x8 = Tile2<4, 8, 4, 8>;  // 16 x 64 = 1024
using Tile2V4x4 = Tile2<4, 4, 2, 4>;  //  8 x 16 =  128, four bins per warp

template <class T, class Op>
__global__ void __launch_bounds__(kThreads, 1) mac_fp32x2_kernel(const MacArgs a) {
  typedef typename Op::pair pair;
  typedef typename Op::quad quad;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  PhaseConst* pcs = reinterpret_cast<PhaseConst*>(smem_raw);
  float* swap_all = reinterpret_cast<float*>(smem_raw + sizeof(PhaseConst) * a.n_chan);

  for (int i = threadIdx.x; i < a.n_chan; i += kThreads) pcs[i] = a.pc[i];
  __syncthreads();

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int g = lane / T::G;
  const int lg = lane % T::G;
  const int ga = lg / T::GB;
  const int gb = lg % T::GB;
  const int k = (blockIdx.x * kWarps + warp) * T::NG + g;
  const bool k_ok = k < a.n_bins;
  const uint32_t ku = k_ok ? static_cast<uint32_t>(k) : 0u;
  const int jblk = blockIdx.y * T::DMS;
  const int series = blockIdx.z;

  float* grp0 = swap_all + warp * 2 * T::XFL + g * T::GFL;

  uint32_t mz[T::ZGEN];
  int zoff[T::ZGEN];
  bool zon[T::ZGEN];
#pragma unroll
  for (int q = 0; q < T::ZGEN; ++q) {
    const int ai = lg + q * T::G;
    zon[q] = ai < T::AW;
    mz[q] = ku * static_cast<uint32_t>(a.j_begin + jblk + ai * T::TW);
    zoff[q] = ((ai / T::AT) * T::ZG + (ai % T::AT)) * 4;
  }
  uint32_t mp[T::PGEN];
  int poff[T::PGEN];
  bool pon[T::PGEN];
#pragma unroll
  for (int q = 0; q < T::PGEN; ++q) {
    const int bi = lg + q * T::G;
    pon[q] = bi < T::TW;
    mp[q] = ku * static_cast<uint32_t>(bi);
    poff[q] = T::ZFL + (bi / T::BT) * T::PSTR + (bi % T::BT);
  }

  const float2* xp = a.X + static_cast<int64_t>(series) * a.x_series_stride + ku;
  const int64_t xs = a.x_chan_stride;

  pair accr[T::AT][T::BT / 2];
  pair acci[T::AT][T::BT / 2];
#pragma unroll
  for (int i = 0; i < T::AT; ++i)
#pragma unroll
    for (int j = 0; j < T::BT / 2; ++j) {
      accr[i][j] = Op::zero();
      acci[i][j] = Op::zero();
    }

  float2 xnext[kPrefetch];
#pragma unroll
  for (int i = 0; i < kPrefetch; ++i)
    xnext[i] = (i < a.n_chan) ? __ldg(xp + i * xs) : make_float2(0.f, 0.f);

  int stage = 0;
  for (int c0 = 0; c0 < a.n_chan; c0 += kPrefetch) {
    float2 xcur[kPrefetch];
#pragma unroll
    for (int i = 0; i < kPrefetch; ++i) {
      xcur[i] = xnext[i];
      const int cn = c0 + kPrefetch + i;
      xnext[i] = (cn < a.n_chan) ? __ldg(xp + cn * xs) : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int i = 0; i < kPrefetch; ++i) {
      const int c = c0 + i;
      if (c < a.n_chan) {
        const PhaseConst p = pcs[c];
        const uint32_t base = top32_mul(ku, p.u_lo, p.u_hi);
        float* buf = grp0 + stage * T::XFL;
#pragma unroll
        for (int q = 0; q < T::ZGEN; ++q) {
          if (zon[q]) {
            const float2 w = unit_phasor(base + top32_mul(mz[q], p.v_lo, p.v_hi));
            const float2 x = xcur[i];
            const float zr = x.x * w.x - x.y * w.y;
            const float zi = x.x * w.y + x.y * w.x;
            *reinterpret_cast<float4*>(buf + zoff[q]) = make_float4(zr, zr, zi, zi);
          }
        }
#pragma unroll
        for (int q = 0; q < T::PGEN; ++q) {
          if (pon[q]) {
            const float2 w = unit_phasor(top32_mul(mp[q], p.v_lo, p.v_hi));
            buf[poff[q]] = w.x;
            buf[poff[q] + T::PFL] = w.y;
            buf[poff[q] + 2 * T::PFL] = -w.y;
          }
        }
        __syncwarp();

        const float* prow = buf + T::ZFL + gb * T::PSTR;
        pair pr2[T::BT / 2], pi2[T::BT / 2], pn2[T::BT / 2];
#pragma unroll
        for (int h = 0; h < T::BT / 4; ++h) {
          const quad vr = *reinterpret_cast<const quad*>(prow + 4 * h);
          const quad vi = *reinterpret_cast<const quad*>(prow + T::PFL + 4 * h);
          const quad vn = *reinterpret_cast<const quad*>(prow + 2 * T::PFL + 4 * h);
          pr2[2 * h] = Op::lo(vr);
          pr2[2 * h + 1] = Op::hi(vr);
          pi2[2 * h] = Op::lo(vi);
          pi2[2 * h + 1] = Op::hi(vi);
          pn2[2 * h] = Op::lo(vn);
          pn2[2 * h + 1] = Op::hi(vn);
        }
        const quad* zq = reinterpret_cast<const quad*>(buf + ga * T::ZG * 4);
#pragma unroll
        for (int ii = 0; ii < T::AT; ++ii) {
          const quad z = zq[ii];  // (zr, zr), (zi, zi)
          const pair zrr = Op::lo(z), zii = Op::hi(z);
#pragma unroll
          for (int jp = 0; jp < T::BT / 2; ++jp) {
            accr[ii][jp] = Op::fma(zrr, pr2[jp], accr[ii][jp]);
            acci[ii][jp] = Op::fma(zrr, pi2[jp], acci[ii][jp]);
          }
#pragma unroll
          for (int jp = 0; jp < T::BT / 2; ++jp) {
            accr[ii][jp] = Op::fma(zii, pn2[jp], accr[ii][jp]);
            acci[ii][jp] = Op::fma(zii, pr2[jp], acci[ii][jp]);
          }
        }
        stage ^= 1;
      }
    }
  }

  if (!k_ok) return;
  const bool real_only = (k == a.real_bin_a) || (k == a.real_bin_b);
#pragma unroll
  for (int ii = 0; ii < T::AT; ++ii) {
#pragma unroll
    for (int jp = 0; jp < T::BT / 2; ++jp) {
      const float2 re2 = Op::split(accr[ii][jp]);
      const float2 im2 = Op::split(acci[ii][jp]);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int jl = jblk + (ga * T::AT + ii) * T::TW + gb * T::BT + 2 * jp + h;
        if (jl < a.n_dm) {
          const float re = (h ? re2.y : re2.x) * a.scale;
          const float im = real_only ? 0.f : (h ? im2.y : im2.x) * a.scale;
          const int64_t off = static_cast<int64_t>(series) * a.y_series_stride +
                              static_cast<int64_t>(jl) * a.y_dm_stride + k;
          if (a.out_kind == 2)
            static_cast<float*>(a.Y)[off] = re * re + im * im;
          else
            static_cast<float2*>(a.Y)[off] = make_float2(re, im);
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Variant table: kernel, trials per block, bin groups per warp, swap bytes.
struct VariantInfo {
  const void* fn;
  int dms;
  int ng;
  size_t swap_bytes;  // per CTA, excluding the phase-constant table
};

template <class T>
VariantInfo info_f1() {
  return {reinterpret_cast<const void*>(&mac_fp32_kernel<T>), T::DMS, T::NG,
          sizeof(float2) * static_cast<size_t>(kWarps) * 2 * T::XCH};
}

template <class T, class Op>
VariantInfo info_f2() {
  return {reinterpret_cast<const void*>(&mac_fp32x2_kernel<T, Op>), T::DMS, T::NG,
          sizeof(float) * static_cast<size_t>(kWarps) * 2 * T::XFL};
}

VariantInfo variant_info(int v) {
  switch (v) {
    case MAC_F1_8x8: return info_f1<TileV8x8>();
    case MAC_F1_4x8: return info_f1<TileV4x8>();
    case MAC_F1_4x4: return info_f1<TileV4x4>();
    case MAC_F2_8x8: return info_f2<Tile2V8x8, PairAsm>();
    case MAC_F2_4x8: return info_f2<Tile2V4x8, PairAsm>();
    case MAC_F2_4x4: return info_f2<Tile2V4x4, PairAsm>();
    case MAC_F3_8x8: return info_f2<Tile2V8x8, PairBuiltin>();
    case MAC_F3_4x8: return info_f2<Tile2V4x8, PairBuiltin>();
    default: return info_f2<Tile2V4x4, PairBuiltin>();
  }
}

}  // namespace

int mac_variant_for(int n_dm) {
  if (n_dm > 1024) return MAC_F1_8x8;
  if (n_dm > 256) return MAC_F1_4x8;
  return MAC_F1_4x4;
}

int mac_variant_trials_per_block(int variant) { return variant_info(variant).dms; }

size_t mac_smem_bytes(int variant, int n_chan) {
  return sizeof(PhaseConst) * static_cast<size_t>(n_chan) + variant_info(variant).swap_bytes;
}

cudaError_t mac_prepare(int variant, int n_chan) {
  const VariantInfo vi = variant_info(variant);
  return cudaFuncSetAttribute(vi.fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              static_cast<int>(mac_smem_bytes(variant, n_chan)));
}

cudaError_t launch_mac_fp32(const MacArgs& a, int variant, cudaStream_t s) {
  if (a.n_dm <= 0 || a.n_series <= 0 || a.n_bins <= 0) return cudaSuccess;
  const VariantInfo vi = variant_info(variant);
  const int bins_per_cta = kWarps * vi.ng;
  dim3 grid((a.n_bins + bins_per_cta - 1) / bins_per_cta, (a.n_dm + vi.dms - 1) / vi.dms,
            a.n_series);
  if (grid.y > 65535u || grid.z > 65535u) return cudaErrorInvalidConfiguration;
  MacArgs args = a;
  void* params[] = {&args};
  return cudaLaunchKernel(vi.fn, grid, dim3(kThreads), params, mac_smem_bytes(variant, a.n_chan),
                          s);
}

}  // namespace fdd

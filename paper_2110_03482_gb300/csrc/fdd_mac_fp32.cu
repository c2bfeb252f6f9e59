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

template <class T>
size_t smem_for(int n_chan) {
  return sizeof(PhaseConst) * static_cast<size_t>(n_chan) +
         sizeof(float2) * static_cast<size_t>(kWarps) * 2 * T::XCH;
}

template <class T>
cudaError_t launch_t(const MacArgs& a, cudaStream_t s) {
  const int bins_per_cta = kWarps * T::NG;
  dim3 grid((a.n_bins + bins_per_cta - 1) / bins_per_cta, (a.n_dm + T::DMS - 1) / T::DMS,
            a.n_series);
  if (grid.y > 65535u || grid.z > 65535u) return cudaErrorInvalidConfiguration;
  mac_fp32_kernel<T><<<grid, kThreads, smem_for<T>(a.n_chan), s>>>(a);
  return cudaGetLastError();
}

template <class T>
cudaError_t prepare_t(int n_chan) {
  const size_t bytes = smem_for<T>(n_chan);
  return cudaFuncSetAttribute(mac_fp32_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              static_cast<int>(bytes));
}

}  // namespace

int mac_variant_for(int n_dm) {
  if (n_dm > 1024) return MAC_V8x8;
  if (n_dm > 256) return MAC_V4x8;
  return MAC_V4x4;
}

int mac_variant_trials_per_block(int variant) {
  switch (variant) {
    case MAC_V8x8: return TileV8x8::DMS;
    case MAC_V4x8: return TileV4x8::DMS;
    default: return TileV4x4::DMS;
  }
}

size_t mac_smem_bytes(int variant, int n_chan) {
  switch (variant) {
    case MAC_V8x8: return smem_for<TileV8x8>(n_chan);
    case MAC_V4x8: return smem_for<TileV4x8>(n_chan);
    default: return smem_for<TileV4x4>(n_chan);
  }
}

cudaError_t mac_prepare(int variant, int n_chan) {
  switch (variant) {
    case MAC_V8x8: return prepare_t<TileV8x8>(n_chan);
    case MAC_V4x8: return prepare_t<TileV4x8>(n_chan);
    default: return prepare_t<TileV4x4>(n_chan);
  }
}

cudaError_t launch_mac_fp32(const MacArgs& a, int variant, cudaStream_t s) {
  if (a.n_dm <= 0 || a.n_series <= 0 || a.n_bins <= 0) return cudaSuccess;
  switch (variant) {
    case MAC_V8x8: return launch_t<TileV8x8>(a, s);
    case MAC_V4x8: return launch_t<TileV4x8>(a, s);
    default: return launch_t<TileV4x4>(a, s);
  }
}

}  // namespace fdd

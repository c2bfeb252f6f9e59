// fdd_tdd.cu -- brute-force time-domain dedispersion (Eq. 2; the method the
// paper measures Fourier-domain dedispersion against, Sect. 4):
//
//   y[j][n] = sum_nu x[nu][n + s[j][nu]],   s = delay of Eq. 1 rounded to the
//                                              nearest sample,
//
// for the valid samples n < n_t - D_max (every channel in range).  One CTA
// computes kTdDms trials x kTdSamp samples: for kTdCh channels at a time it
// stages each channel's input window (the samples the block's trials read:
// from t0 + the block's smallest shift, kTdSamp + the shift span wide) in
// shared memory, then every lane adds, for its 4 trials and 8 samples
// (lane + 32 i), one window value per channel: 32 consecutive lanes read 32
// consecutive floats, so each add costs one conflict-free 4-byte shared load.
// Shared-memory bandwidth (128 B per clock per SM) bounds the kernel at 32
// adds per clock per SM.  Trial blocks run fastest in the grid, so the blocks
// that share a time window run together and read it from L2.
#include "fdd_internal.h"

namespace fdd {
namespace {

constexpr int kTdWarps = 8;
constexpr int kTdDmsWarp = kTdDms / kTdWarps;  // trials per warp (4)
constexpr int kTdPer = kTdSamp / 32;           // samples per lane (8)

__global__ void __launch_bounds__(kTdWarps * 32) tdd_kernel(const TddArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  int* rel = reinterpret_cast<int*>(smem_raw);                         // [kTdCh][kTdDms]
  float* win = reinterpret_cast<float*>(smem_raw + sizeof(int) * kTdCh * kTdDms);  // [kTdCh][a.win]
  const int blk = blockIdx.x;
  const int j0 = blk * kTdDms;
  const int64_t t0 = static_cast<int64_t>(blockIdx.y) * kTdSamp;
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int nthr = kTdWarps * 32;

  float acc[kTdDmsWarp][kTdPer];
#pragma unroll
  for (int d = 0; d < kTdDmsWarp; ++d)
#pragma unroll
    for (int i = 0; i < kTdPer; ++i) acc[d][i] = 0.f;

  for (int c0 = 0; c0 < a.n_chan; c0 += kTdCh) {
    __syncthreads();  // the previous stage is consumed
    for (int idx = threadIdx.x; idx < kTdCh * kTdDms; idx += nthr) {
      const int cc = idx / kTdDms, jj = idx % kTdDms;
      const int c = c0 + cc, j = j0 + jj;
      rel[idx] = (c < a.n_chan && j < a.n_dm)
                     ? a.shift[static_cast<int64_t>(j) * a.n_chan + c] -
                           a.base[static_cast<int64_t>(blk) * a.n_chan + c]
                     : 0;
    }
    for (int idx = threadIdx.x; idx < kTdCh * a.win; idx += nthr) {
      const int cc = idx / a.win, w = idx % a.win;
      const int c = c0 + cc;
      float v = 0.f;
      if (c < a.n_chan) {
        const int64_t t = t0 + a.base[static_cast<int64_t>(blk) * a.n_chan + c] + w;
        if (t < a.n_t) v = a.x[static_cast<int64_t>(c) * a.n_t + t];
      }
      win[idx] = v;
    }
    __syncthreads();
    const int nc = a.n_chan - c0 < kTdCh ? a.n_chan - c0 : kTdCh;
    for (int cc = 0; cc < nc; ++cc) {
      const float* wr = win + cc * a.win + lane;
#pragma unroll
      for (int d = 0; d < kTdDmsWarp; ++d) {
        const int r = rel[cc * kTdDms + warp * kTdDmsWarp + d];
#pragma unroll
        for (int i = 0; i < kTdPer; ++i) acc[d][i] += wr[32 * i + r];
      }
    }
  }

#pragma unroll
  for (int d = 0; d < kTdDmsWarp; ++d) {
    const int j = j0 + warp * kTdDmsWarp + d;
    if (j >= a.n_dm) continue;
#pragma unroll
    for (int i = 0; i < kTdPer; ++i) {
      const int64_t n = t0 + lane + 32 * i;
      if (n < a.out_len) a.y[static_cast<int64_t>(j) * a.out_len + n] = acc[d][i];
    }
  }
}

}  // namespace

size_t tdd_smem_bytes(int win) {
  return sizeof(int) * kTdCh * kTdDms + sizeof(float) * static_cast<size_t>(kTdCh) * win;
}

cudaError_t tdd_prepare(int win) {
  return cudaFuncSetAttribute(tdd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              static_cast<int>(tdd_smem_bytes(win)));
}

cudaError_t launch_tdd(const TddArgs& a, cudaStream_t s) {
  if (a.n_dm <= 0 || a.out_len <= 0) return cudaSuccess;
  const int64_t t_blocks = (a.out_len + kTdSamp - 1) / kTdSamp;
  if (t_blocks > 65535) return cudaErrorInvalidConfiguration;
  dim3 grid((a.n_dm + kTdDms - 1) / kTdDms, static_cast<unsigned>(t_blocks));
  tdd_kernel<<<grid, kTdWarps * 32, tdd_smem_bytes(a.win), s>>>(a);
  return cudaGetLastError();
}

}  // namespace fdd

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
// adds per clock per SM.  The stages are double-buffered: the next stage's
// windows and relative shifts stream in with cp.async while the current one
// is summed.  Trial blocks run fastest in the grid, so the blocks that share
// a time window run together and read it from L2.
#include "fdd_internal.h"

namespace fdd {
namespace {

constexpr int kTdWarps = 8;
constexpr int kTdThreads = kTdWarps * 32;
constexpr int kTdDmsWarp = kTdDms / kTdWarps;  // trials per warp (4)
constexpr int kTdPer = kTdSamp / 32;           // samples per lane (8)

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// 4 bytes global -> shared, asynchronously; zeros when !valid (no read).
__device__ __forceinline__ void cp_async4(void* dst, const void* src, bool valid) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(smem_addr(dst)), "l"(src),
               "r"(valid ? 4 : 0)
               : "memory");
}

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src)
               : "memory");
}

// Stage (channels c0 .. c0 + kTdCh - 1) into buffer (rel, win).
__device__ __forceinline__ void tdd_fill(const TddArgs& a, int blk, int64_t t0, int c0, int* rel,
                                         float* win) {
  // relative shifts: kTdCh x kTdDms ints, contiguous in the table, 16 bytes a thread
  const int nc = a.n_chan - c0 < kTdCh ? a.n_chan - c0 : kTdCh;
  const int* src_rel = a.rel + (static_cast<int64_t>(blk) * a.n_chan + c0) * kTdDms;
  for (int q = threadIdx.x; q < nc * kTdDms / 4; q += kTdThreads)
    cp_async16(rel + 4 * q, src_rel + 4 * q);
#pragma unroll 1
  for (int cc = 0; cc < nc; ++cc) {
    const int c = c0 + cc;
    float* row = win + cc * a.win;
    const int64_t t_first = t0 + a.base[static_cast<int64_t>(blk) * a.n_chan + c];
    const float* src = a.x + static_cast<int64_t>(c) * a.n_t + t_first;
    const int64_t n_in = a.n_t - t_first;
    for (int w = threadIdx.x; w < a.win; w += kTdThreads)
      cp_async4(row + w, w < n_in ? src + w : a.x, w < n_in);
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
}

__global__ void __launch_bounds__(kTdThreads) tdd_kernel(const TddArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // two buffers, each [kTdCh][kTdDms] relative shifts then [kTdCh][a.win] window
  const size_t buf_bytes = sizeof(int) * kTdCh * kTdDms + sizeof(float) * size_t(kTdCh) * a.win;
  auto rel_of = [&](int b) { return reinterpret_cast<int*>(smem_raw + b * buf_bytes); };
  auto win_of = [&](int b) {
    return reinterpret_cast<float*>(smem_raw + b * buf_bytes + sizeof(int) * kTdCh * kTdDms);
  };
  const int blk = blockIdx.x;
  const int j0 = blk * kTdDms;
  const int64_t t0 = static_cast<int64_t>(blockIdx.y) * kTdSamp;
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;

  float acc[kTdDmsWarp][kTdPer];
#pragma unroll
  for (int d = 0; d < kTdDmsWarp; ++d)
#pragma unroll
    for (int i = 0; i < kTdPer; ++i) acc[d][i] = 0.f;

  const int n_stages = (a.n_chan + kTdCh - 1) / kTdCh;
  tdd_fill(a, blk, t0, 0, rel_of(0), win_of(0));
  for (int st = 0; st < n_stages; ++st) {
    const int cur = st & 1;
    if (st + 1 < n_stages) {
      tdd_fill(a, blk, t0, (st + 1) * kTdCh, rel_of(cur ^ 1), win_of(cur ^ 1));
      asm volatile("cp.async.wait_group 1;" ::: "memory");  // this stage's copies are done
    } else {
      asm volatile("cp.async.wait_group 0;" ::: "memory");
    }
    __syncthreads();  // ... and every thread's
    const int c0 = st * kTdCh;
    const int nc = a.n_chan - c0 < kTdCh ? a.n_chan - c0 : kTdCh;
    const int* rel = rel_of(cur);
    const float* win = win_of(cur);
#pragma unroll
    for (int cc = 0; cc < kTdCh; ++cc) {
      if (cc < nc) {
        const float* wr = win + cc * a.win + lane;
#pragma unroll
        for (int d = 0; d < kTdDmsWarp; ++d) {
          const int r = rel[cc * kTdDms + warp * kTdDmsWarp + d];
#pragma unroll
          for (int i = 0; i < kTdPer; ++i) acc[d][i] += wr[32 * i + r];
        }
      }
    }
    __syncthreads();  // this buffer is refilled by the next iteration's prefetch
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
  return 2 * (sizeof(int) * kTdCh * kTdDms + sizeof(float) * static_cast<size_t>(kTdCh) * win);
}

cudaError_t tdd_prepare(int win) {
  return cudaFuncSetAttribute(tdd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              static_cast<int>(tdd_smem_bytes(win)));
}

cudaError_t launch_tdd(const TddArgs& a, cudaStream_t s) {
  if (a.n_dm <= 0 || a.out_len <= 0) return cudaSuccess;
  if (a.win % 4 != 0) return cudaErrorInvalidValue;  // keeps the buffers 16-byte aligned
  const int64_t t_blocks = (a.out_len + kTdSamp - 1) / kTdSamp;
  if (t_blocks > 65535) return cudaErrorInvalidConfiguration;
  dim3 grid((a.n_dm + kTdDms - 1) / kTdDms, static_cast<unsigned>(t_blocks));
  tdd_kernel<<<grid, kTdThreads, tdd_smem_bytes(a.win), s>>>(a);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace fdd

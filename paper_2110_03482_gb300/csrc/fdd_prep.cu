// fdd_prep.cu -- the HBM-bound steps around the phasor-MAC:
//  * unpack: transpose_and_unpack + zero_pad of Algorithm 1 (Sect. 3), here
//    also cutting one overlap-save chunk: a time-major [n_t][n_chan] u8/f32
//    beam becomes channel-major float series of L samples, zero beyond n_t;
//  * scatter: apply_scaling of Algorithm 1 (1/L) and keep the first n_keep
//    samples of each inverse-transformed DM series (discard rule, Sect. 2.2);
//  * bin transpose: spectra [row][bin] -> [bin][row] for the tensor-core
//    form, and its output back, [bin][series][trial] -> [series][trial][bin].
#include "fdd_internal.h"
#include "fdd.h"

namespace fdd {
namespace {

constexpr int kTile = 32;

// 32 samples x 128 channels through shared memory: coalesced reads along
// channels (each thread four consecutive channels, one 4-byte (u8) or
// 16-byte (f32) load when kVec), coalesced 128-byte writes along time.  The
// tile is [channel][sample] with the sample column rotated by channel / 4,
// so both the scattered writes of the read phase (four channels per thread)
// and the row reads of the write phase hit 32 different banks.
constexpr int kUnpC = 128;  // channels per tile
template <typename Tin>
struct Vec4;
template <>
struct Vec4<uint8_t> {
  __device__ static void load(const uint8_t* p, float (&v)[4]) {
    const uint32_t w = *reinterpret_cast<const uint32_t*>(p);
#pragma unroll
    for (int e = 0; e < 4; ++e) v[e] = static_cast<float>((w >> (8 * e)) & 0xFFu);
  }
};
template <>
struct Vec4<float> {
  __device__ static void load(const float* p, float (&v)[4]) {
    const float4 w = *reinterpret_cast<const float4*>(p);
    v[0] = w.x;
    v[1] = w.y;
    v[2] = w.z;
    v[3] = w.w;
  }
};

template <typename Tin, bool kVec>
__global__ void __launch_bounds__(256) unpack_time_major_kernel(const Tin* __restrict__ in,
                                                                int n_chan, int64_t n_t,
                                                                int64_t t_begin, int64_t L,
                                                                float* __restrict__ out,
                                                                int64_t out_stride) {
  __shared__ float tile[kUnpC][kTile + 1];
  const int64_t n0 = static_cast<int64_t>(blockIdx.x) * kTile;
  const int c0 = blockIdx.y * kUnpC;
  const int cq = c0 + 4 * threadIdx.x;  // this thread's four channels
#pragma unroll
  for (int r = threadIdx.y; r < kTile; r += 8) {
    const int64_t n = n0 + r;
    const int64_t t = t_begin + n;
    float v[4] = {0.f, 0.f, 0.f, 0.f};
    if (n < L && t < n_t) {
      const Tin* row = in + t * n_chan;
      if (kVec && cq + 3 < n_chan) {
        Vec4<Tin>::load(row + cq, v);
      } else {
#pragma unroll
        for (int e = 0; e < 4; ++e)
          if (cq + e < n_chan) v[e] = static_cast<float>(row[cq + e]);
      }
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) tile[4 * threadIdx.x + e][(r + threadIdx.x) & (kTile - 1)] = v[e];
  }
  __syncthreads();
#pragma unroll
  for (int cl = threadIdx.y; cl < kUnpC; cl += 8) {
    const int c = c0 + cl;
    const int64_t n = n0 + threadIdx.x;
    if (c < n_chan && n < L)
      out[static_cast<int64_t>(c) * out_stride + n] = tile[cl][(threadIdx.x + (cl >> 2)) & (kTile - 1)];
  }
}

template <typename Tin>
__global__ void __launch_bounds__(256) unpack_chan_major_kernel(const Tin* __restrict__ in,
                                                                int n_chan, int64_t n_t,
                                                                int64_t t_begin, int64_t L,
                                                                float* __restrict__ out,
                                                                int64_t out_stride) {
  const int c = blockIdx.y;
  for (int64_t n = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; n < L;
       n += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t t = t_begin + n;
    out[static_cast<int64_t>(c) * out_stride + n] =
        (t < n_t) ? static_cast<float>(in[static_cast<int64_t>(c) * n_t + t]) : 0.f;
  }
}

// One row per blockIdx.y.  The destination rows start at arbitrary offsets,
// so each thread writes 16-byte aligned float4 groups of the row (a scalar
// head and tail around them) and reads its four source values with plain
// loads; a warp's loads cover 512 contiguous bytes of the row.
__global__ void __launch_bounds__(256) scatter_kernel(const float* __restrict__ src,
                                                      int64_t src_stride, float* __restrict__ dst,
                                                      int64_t dst_stride, int64_t n_keep,
                                                      float scale) {
  const int r = blockIdx.y;
  const float* s = src + static_cast<int64_t>(r) * src_stride;
  float* d = dst + static_cast<int64_t>(r) * dst_stride;
  // elements before the first 16-byte boundary of the destination row
  int64_t head = static_cast<int64_t>((16 - (reinterpret_cast<uintptr_t>(d) & 15)) & 15) / 4;
  if (head > n_keep) head = n_keep;
  const int64_t tid = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t nth = static_cast<int64_t>(gridDim.x) * blockDim.x;
  if (tid < head) d[tid] = s[tid] * scale;
  const int64_t n_vec = (n_keep - head) / 4;
  float4* dv = reinterpret_cast<float4*>(d + head);
  const float* sv = s + head;
  for (int64_t q = tid; q < n_vec; q += nth) {
    const float* p = sv + 4 * q;
    dv[q] = make_float4(p[0] * scale, p[1] * scale, p[2] * scale, p[3] * scale);
  }
  const int64_t t0 = head + 4 * n_vec;
  if (t0 + tid < n_keep) d[t0 + tid] = s[t0 + tid] * scale;
}

// 32 bins x 32 rows through shared memory: coalesced reads along bins,
// coalesced writes along rows.  Rows beyond gridDim.y tiles are covered by a
// grid-stride loop.  With absmax, each bin's largest |re| or |im| over the
// rows this block read goes to absmax[bin] by one atomic max per bin.
__global__ void __launch_bounds__(256) bin_transpose_kernel(const float2* __restrict__ in,
                                                            int64_t in_stride, int64_t rows,
                                                            int64_t k0, int n_bins,
                                                            float2* __restrict__ out,
                                                            int64_t out_bin_stride,
                                                            unsigned int* __restrict__ absmax) {
  __shared__ float2 tile[kTile][kTile + 1];
  __shared__ float red[8][kTile];
  const int kb0 = blockIdx.x * kTile;
  float m = 0.f;  // bin kb0 + threadIdx.x, the rows this thread read
  for (int64_t r0 = static_cast<int64_t>(blockIdx.y) * kTile; r0 < rows;
       r0 += static_cast<int64_t>(gridDim.y) * kTile) {
#pragma unroll
    for (int i = threadIdx.y; i < kTile; i += 8) {
      const int64_t r = r0 + i;
      const int kb = kb0 + threadIdx.x;
      if (r < rows && kb < n_bins) {
        const float2 v = in[r * in_stride + k0 + kb];
        tile[i][threadIdx.x] = v;
        m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y)));
      }
    }
    __syncthreads();
#pragma unroll
    for (int i = threadIdx.y; i < kTile; i += 8) {
      const int kb = kb0 + i;
      const int64_t r = r0 + threadIdx.x;
      if (r < rows && kb < n_bins) out[static_cast<int64_t>(kb) * out_bin_stride + r] = tile[threadIdx.x][i];
    }
    __syncthreads();
  }
  if (absmax) {
    red[threadIdx.y][threadIdx.x] = m;
    __syncthreads();
    if (threadIdx.y == 0) {
#pragma unroll
      for (int j = 1; j < 8; ++j) m = fmaxf(m, red[j][threadIdx.x]);
      const int kb = kb0 + threadIdx.x;
      if (kb < n_bins && m > 0.f) atomicMax(absmax + kb, __float_as_uint(m));
    }
  }
}


// Per bin k, the largest |re| or |im| of its bin-major spectra
// in[k * bin_stride + r], r < rows (the FP16 tensor-core form scales each
// bin's data by a power of two chosen from it): one block per bin, a
// coalesced sweep of the bin's rows and a block reduction; absmax[k] gets
// the float's bits (non-negative floats order as their bits).
__global__ void __launch_bounds__(256) bin_absmax_kernel(const float2* __restrict__ in,
                                                         int64_t bin_stride, int rows,
                                                         unsigned int* __restrict__ absmax) {
  __shared__ float red[8];
  const float2* p = in + static_cast<int64_t>(blockIdx.x) * bin_stride;
  float m = 0.f;
  for (int r = threadIdx.x; r < rows; r += 256) {
    const float2 v = __ldg(p + r);
    m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y)));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int i = 1; i < 8; ++i) m = fmaxf(m, red[i]);
    absmax[blockIdx.x] = __float_as_uint(m);
  }
}

// Thread rows of the untranspose's 32 x 32 tiles (4: measured 5.7 TB/s on the
// 32-beam slice, against 5.5 TB/s with 8 rows and less with wider tiles).
constexpr int kUntrRows = 4;

template <typename T>
__global__ void __launch_bounds__(32 * kUntrRows) bin_untranspose_kernel(const T* __restrict__ in,
                                                              int n_series, int n_dm, int n_bins,
                                                              int64_t rows, T* __restrict__ out,
                                                              int64_t out_series_stride,
                                                              int64_t out_dm_stride) {
  __shared__ T tile[kTile][kTile + 1];
  const int kb0 = blockIdx.x * kTile;
  const int d_tiles = (n_dm + kTile - 1) / kTile;
  // (rows: elements between bins of the input)
  const int64_t n_tiles = static_cast<int64_t>(n_series) * d_tiles;
  for (int64_t q = blockIdx.y; q < n_tiles; q += gridDim.y) {
    const int sr = static_cast<int>(q / d_tiles);
    const int d0 = static_cast<int>(q - static_cast<int64_t>(sr) * d_tiles) * kTile;
    const T* src = in + static_cast<int64_t>(sr) * n_dm;
#pragma unroll
    for (int i = threadIdx.y; i < kTile; i += kUntrRows) {
      const int kb = kb0 + i;
      const int d = d0 + threadIdx.x;
      if (kb < n_bins && d < n_dm) tile[i][threadIdx.x] = src[static_cast<int64_t>(kb) * rows + d];
    }
    __syncthreads();
    T* dst = out + static_cast<int64_t>(sr) * out_series_stride;
#pragma unroll
    for (int i = threadIdx.y; i < kTile; i += kUntrRows) {
      const int d = d0 + i;
      const int kb = kb0 + threadIdx.x;
      if (kb < n_bins && d < n_dm) dst[static_cast<int64_t>(d) * out_dm_stride + kb] = tile[threadIdx.x][i];
    }
    __syncthreads();
  }
}

}  // namespace

cudaError_t launch_bin_untranspose(const BinUntransposeArgs& a, cudaStream_t s) {
  if (a.n_bins <= 0 || a.n_dm <= 0 || a.n_series <= 0) return cudaSuccess;
  const int64_t tiles = static_cast<int64_t>(a.n_series) * ((a.n_dm + kTile - 1) / kTile);
  dim3 grid((a.n_bins + kTile - 1) / kTile, static_cast<unsigned>(tiles < 65535 ? tiles : 65535));
  note_launches(1);
  const int64_t rows =
      a.in_bin_stride > 0 ? a.in_bin_stride : static_cast<int64_t>(a.n_series) * a.n_dm;
  if (a.elem_bytes == 8)
    bin_untranspose_kernel<float2><<<grid, dim3(kTile, kUntrRows), 0, s>>>(
        static_cast<const float2*>(a.in), a.n_series, a.n_dm, a.n_bins, rows,
        static_cast<float2*>(a.out), a.out_series_stride, a.out_dm_stride);
  else if (a.elem_bytes == 4)
    bin_untranspose_kernel<float><<<grid, dim3(kTile, kUntrRows), 0, s>>>(
        static_cast<const float*>(a.in), a.n_series, a.n_dm, a.n_bins, rows,
        static_cast<float*>(a.out), a.out_series_stride, a.out_dm_stride);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t launch_bin_transpose(const BinTransposeArgs& a, cudaStream_t s) {
  if (a.n_bins <= 0 || a.rows <= 0) return cudaSuccess;
  const int64_t row_tiles = (a.rows + kTile - 1) / kTile;
  dim3 grid((a.n_bins + kTile - 1) / kTile,
            static_cast<unsigned>(row_tiles < 65535 ? row_tiles : 65535));
  note_launches(1);
  bin_transpose_kernel<<<grid, dim3(kTile, 8), 0, s>>>(
      a.in, a.in_stride, a.rows, a.k0, a.n_bins, a.out,
      a.out_bin_stride > 0 ? a.out_bin_stride : a.rows, a.absmax);
  return cudaGetLastError();
}

cudaError_t launch_bin_absmax(const BinAbsmaxArgs& a, cudaStream_t s) {
  if (a.n_bins <= 0 || a.rows <= 0) return cudaSuccess;
  note_launches(1);
  bin_absmax_kernel<<<a.n_bins, 256, 0, s>>>(a.in, a.bin_stride, a.rows, a.absmax);
  return cudaGetLastError();
}

cudaError_t launch_unpack(const UnpackArgs& a, cudaStream_t s) {
  note_launches(1);
  if (a.in_layout == FDD_LAYOUT_TIME_MAJOR) {
    dim3 grid(static_cast<unsigned>((a.L + kTile - 1) / kTile), (a.n_chan + kUnpC - 1) / kUnpC);
    dim3 block(kTile, 8);
    if (grid.y > 65535u) return cudaErrorInvalidConfiguration;
    // vector loads when every row of four channels is aligned for them
    const size_t esz = a.in_dtype == FDD_IN_U8 ? 1 : 4;
    const bool vec = a.n_chan % 4 == 0 && reinterpret_cast<uintptr_t>(a.in) % (4 * esz) == 0;
    if (a.in_dtype == FDD_IN_U8) {
      const uint8_t* in = static_cast<const uint8_t*>(a.in);
      if (vec)
        unpack_time_major_kernel<uint8_t, true><<<grid, block, 0, s>>>(in, a.n_chan, a.n_t,
                                                                       a.t_begin, a.L, a.out,
                                                                       a.out_stride);
      else
        unpack_time_major_kernel<uint8_t, false><<<grid, block, 0, s>>>(in, a.n_chan, a.n_t,
                                                                        a.t_begin, a.L, a.out,
                                                                        a.out_stride);
    } else {
      const float* in = static_cast<const float*>(a.in);
      if (vec)
        unpack_time_major_kernel<float, true><<<grid, block, 0, s>>>(in, a.n_chan, a.n_t,
                                                                     a.t_begin, a.L, a.out,
                                                                     a.out_stride);
      else
        unpack_time_major_kernel<float, false><<<grid, block, 0, s>>>(in, a.n_chan, a.n_t,
                                                                      a.t_begin, a.L, a.out,
                                                                      a.out_stride);
    }
  } else {
    const int64_t blocks = (a.L + 255) / 256;
    dim3 grid(static_cast<unsigned>(blocks < 4096 ? blocks : 4096), a.n_chan);
    if (grid.y > 65535u) return cudaErrorInvalidConfiguration;
    if (a.in_dtype == FDD_IN_U8)
      unpack_chan_major_kernel<uint8_t><<<grid, 256, 0, s>>>(
          static_cast<const uint8_t*>(a.in), a.n_chan, a.n_t, a.t_begin, a.L, a.out, a.out_stride);
    else
      unpack_chan_major_kernel<float><<<grid, 256, 0, s>>>(
          static_cast<const float*>(a.in), a.n_chan, a.n_t, a.t_begin, a.L, a.out, a.out_stride);
  }
  return cudaGetLastError();
}

cudaError_t launch_scatter(const ScatterArgs& a, cudaStream_t s) {
  if (a.n_dm <= 0 || a.n_keep <= 0) return cudaSuccess;
  if (a.n_dm > 65535) return cudaErrorInvalidConfiguration;
  // about 8 float4 groups per thread
  const int64_t blocks = (a.n_keep + 256 * 32 - 1) / (256 * 32);
  dim3 grid(static_cast<unsigned>(blocks < 1024 ? blocks : 1024), a.n_dm);
  note_launches(1);
  scatter_kernel<<<grid, 256, 0, s>>>(a.src, a.src_stride, a.dst, a.dst_stride, a.n_keep,
                                      a.scale);
  return cudaGetLastError();
}

}  // namespace fdd

// philox_filterbank.cu -- the device side of synth/philox.py: seeded
// Gaussian filterbanks with dispersed pulses, generated in place in device
// memory, bit-identical to the host generator.
//
// Sample (t, c) of beam b is the Philox4x32-10 block (Salmon et al., SC 2011)
// of counter (i mod 2^32, i div 2^32, b, 0), i = t * n_chan + c, under the
// key (k0, k1); its eight 16-bit halves are summed (Irwin-Hall(8)), centred
// and scaled to unit variance, then scaled by sigma, offset by mean, the
// pulses added in order and, for 8-bit data, rounded half-to-even and clipped.
// Every float operation is a single correctly rounded one (no contraction).
// This library makes inputs only; it is not part of the dedispersion path.
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

constexpr uint32_t kM0 = 0xD2511F53u, kM1 = 0xCD9E8D57u;
constexpr uint32_t kW0 = 0x9E3779B9u, kW1 = 0xBB67AE85u;
constexpr int kMaxPulses = 8;

struct PulseSet {
  int n;
  int width[kMaxPulses];
  float amp[kMaxPulses];
};

__device__ __forceinline__ void philox4x32_10(uint32_t x[4], uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += kW0;
      k1 += kW1;
    }
    const uint32_t h0 = __umulhi(kM0, x[0]), l0 = kM0 * x[0];
    const uint32_t h1 = __umulhi(kM1, x[2]), l1 = kM1 * x[2];
    const uint32_t y0 = h1 ^ x[1] ^ k0, y2 = h0 ^ x[3] ^ k1;
    x[0] = y0;
    x[1] = l1;
    x[2] = y2;
    x[3] = l0;
  }
}

__global__ void filterbank_kernel(void* out, int u8, int64_t n_rows, int n_chan, int64_t t0,
                                  uint32_t beam, uint32_t k0, uint32_t k1, float mean,
                                  float sigma, float inv_ih_sigma, const int64_t* starts,
                                  PulseSet ps) {
  const int64_t n = n_rows * n_chan;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < n;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t r = e / n_chan;
    const int c = static_cast<int>(e - r * n_chan);
    const int64_t t = t0 + r;
    const uint64_t i = static_cast<uint64_t>(t) * static_cast<uint64_t>(n_chan) + c;
    uint32_t x[4] = {static_cast<uint32_t>(i), static_cast<uint32_t>(i >> 32), beam, 0u};
    philox4x32_10(x, k0, k1);
    int s = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) s += static_cast<int>(x[q] & 0xFFFFu) + static_cast<int>(x[q] >> 16);
    float v = __fmul_rn(__int2float_rn(s - 262140), inv_ih_sigma);
    if (sigma != 1.0f) v = __fmul_rn(v, sigma);
    if (mean != 0.0f) v = __fadd_rn(v, mean);
    for (int p = 0; p < ps.n; ++p) {
      const int64_t st = starts[static_cast<int64_t>(p) * n_chan + c];
      if (t >= st && t < st + ps.width[p]) v = __fadd_rn(v, ps.amp[p]);
    }
    if (u8) {
      v = fminf(fmaxf(rintf(v), 0.0f), 255.0f);
      static_cast<uint8_t*>(out)[e] = static_cast<uint8_t>(v);
    } else {
      static_cast<float*>(out)[e] = v;
    }
  }
}

}  // namespace

// Fills rows [t0, t0 + n_rows) of one beam's [n_t][n_chan] time-major
// filterbank at d_out (uint8 if u8, else float32; contiguous rows).
// d_starts: device int64 [n_pulses][n_chan] first sample of each pulse per
// channel (NULL if n_pulses is 0); widths and amps: host arrays of n_pulses.
// Returns 0, or a CUDA error code (1 for invalid arguments).
extern "C" int synth_philox_filterbank(void* d_out, int u8, int64_t n_rows, int n_chan,
                                       int64_t t0, uint32_t beam, uint64_t seed, float mean,
                                       float sigma, float inv_ih_sigma, const int64_t* d_starts,
                                       const int* widths, const float* amps, int n_pulses,
                                       void* stream) {
  if (!d_out || n_rows < 0 || n_chan < 1 || t0 < 0 || n_pulses < 0 || n_pulses > kMaxPulses ||
      (n_pulses > 0 && (!d_starts || !widths || !amps)))
    return 1;
  if (n_rows == 0) return 0;
  PulseSet ps{};
  ps.n = n_pulses;
  for (int p = 0; p < n_pulses; ++p) {
    ps.width[p] = widths[p];
    ps.amp[p] = amps[p];
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t n = n_rows * n_chan;
  const int64_t want = (n + 255) / 256;
  const int64_t cap = static_cast<int64_t>(sms > 0 ? sms : 1) * 16;
  const int grid = static_cast<int>(want < cap ? want : cap);
  filterbank_kernel<<<grid, 256, 0, static_cast<cudaStream_t>(stream)>>>(
      d_out, u8, n_rows, n_chan, t0, beam, static_cast<uint32_t>(seed),
      static_cast<uint32_t>(seed >> 32), mean, sigma, inv_ih_sigma, d_starts, ps);
  return static_cast<int>(cudaGetLastError());
}

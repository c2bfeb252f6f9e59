// fdd_mac_tc.cu -- phase-rotate-and-sum on the tensor cores (tcgen05 + TMEM)
// for many beams sharing the same Fourier bins (the tensor-core and
// phasor-reuse directions of Sect. 5 of the paper).
//
// With the trial index split j = aT + b (T = 128), the phasor of Eq. 4
// factorises as W(aT + b) = Q_a P_b (see fdd_mac_fp32.cu), so for one bin k
// and beams beta
//
//   Y[aT + b][beta] = sum_nu P_b[nu] Z_a[nu][beta],   Z_a = Q_a X[nu][beta],
//
// i.e. for every group of a's one complex GEMM of (T x N_nu) phasors P by
// (N_nu x beams) data.  It runs on tcgen05 as a real GEMM
//   D[b][(a, beta, re|im)] = sum_{nu, re|im} A[b][(nu, re|im)] B[(a, beta, re|im)][(nu, re|im)]
// with A = [Pr | Pi] (BF16 hi + lo: two MMAs) and B the real embedding
// [[Zr, -Zi], [Zi, Zr]] of Z (BF16), FP32 accumulation in tensor memory.
// M = 128 trials b, N = 256 = 4 a's x 32 beams x (re, im), K = 64 per stage
// (32 channels x (re, im)); two accumulators cover 8 a's = 1024 trials per
// pass over the channels.
//
// Warp 0 allocates tensor memory and one of its threads issues the MMAs; 8
// producer warps evaluate P (exact fixed-point phase, MUFU sin/cos, hi/lo
// split) and Z = Q X for each stage straight into the 128-byte-swizzled
// K-major shared layout the MMA descriptors address, through a 2-stage
// mbarrier ring, and read the accumulators back (tcgen05.ld) for the store.
// Every wait is bounded: on timeout the kernel records FDD_ERR_TIMEOUT in the
// status word, stops, drains its own MMAs (bounded), frees its tensor memory
// and returns.
#include <cuda_bf16.h>

#include "fdd_internal.h"

namespace fdd {
namespace {

constexpr int kM = 128;                  // trials b per a (T)
constexpr int kN = 256;                  // accumulator columns
constexpr int kBeams = 32;               // beams per group
constexpr int kNA = kN / (2 * kBeams);   // a's per accumulator (4)
constexpr int kAcc = 2;                  // accumulators in tensor memory
constexpr int kAPass = kNA * kAcc;       // a's per pass (8)
constexpr int kDmsPass = kAPass * kM;    // trials per pass (1024)
constexpr int kKC = 32;                  // channels per stage
constexpr int kProdWarps = 8;
constexpr int kProd = 32 * kProdWarps;
constexpr int kThreads = 32 + kProd;
constexpr uint32_t kTileA = kM * 64 * 2;  // 16 KB
constexpr uint32_t kTileB = kN * 64 * 2;  // 32 KB
constexpr uint32_t kStageBytes = 2 * kTileA + kAcc * kTileB;  // 96 KB
constexpr int kStages = 2;
constexpr uint32_t kTmemCols = 512;
constexpr long long kWaitCycles = 4000000000LL;  // ~2 s at 2 GHz

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Byte offset of element (row, kk) in a K-major tile of 64 BF16 per row with
// the 128-byte swizzle: 16-byte chunks of a row are permuted by (row mod 8).
__device__ __forceinline__ uint32_t sw128(int row, int kk) {
  return (row >> 3) * 1024 + (row & 7) * 128 + (((kk >> 3) ^ (row & 7)) << 4) + ((kk & 7) << 1);
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  return static_cast<uint64_t>((addr & 0x3FFFF) >> 4) | (static_cast<uint64_t>(1) << 16) |
         (static_cast<uint64_t>(1024 >> 4) << 32) | (static_cast<uint64_t>(1) << 46) |
         (static_cast<uint64_t>(2) << 61);
}

// Instruction descriptor: D FP32, A and B BF16, both K-major, N and M.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) |
                            (static_cast<uint32_t>(kN >> 3) << 17) |
                            (static_cast<uint32_t>(kM >> 4) << 24);

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}" ::"r"(
                   smem_u32(bar))
               : "memory");
}

// Bounded wait for the phase of the given parity; false on timeout or abort.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity,
                                          volatile int* abort_flag) {
  const long long t0 = clock64();
  while (true) {
    uint32_t done;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                 " selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(done)
                 : "r"(smem_u32(bar)), "r"(parity)
                 : "memory");
    if (done) return true;
    if (*abort_flag) return false;
    if (clock64() - t0 > kWaitCycles) return false;
  }
}

__device__ __forceinline__ uint32_t top32_mul(uint32_t m, uint32_t lo, uint32_t hi) {
  return __umulhi(m, lo) + m * hi;
}

__device__ __forceinline__ float2 unit_phasor(uint32_t phase) {
  const float x = __int2float_rn(static_cast<int>(phase)) * 1.46291807926715968e-9f;  // 2pi/2^32
  float s, c;
  __sincosf(x, &s, &c);
  return make_float2(c, s);
}

__device__ __forceinline__ uint32_t bf16x2_bits(__nv_bfloat162 v) {
  return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__global__ void __launch_bounds__(kThreads, 1) mac_tc_kernel(const MacArgs a) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(base + kStages * kStageBytes);
  uint64_t* full = bars;              // [kStages], producers -> MMA
  uint64_t* empty = bars + kStages;   // [kStages], MMA commit -> producers
  uint64_t* acc_full = bars + 2 * kStages;
  uint64_t* acc_empty = bars + 2 * kStages + 1;
  uint64_t* drain = bars + 2 * kStages + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * kStages + 3);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], kProd);
      mbar_init(&empty[s], 1);
    }
    mbar_init(acc_full, 1);
    mbar_init(acc_empty, kProd);
    mbar_init(drain, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  const int n_groups = (a.n_series + kBeams - 1) / kBeams;
  const int n_pass = (a.n_dm + kDmsPass - 1) / kDmsPass;
  const int n_tiles = (a.n_chan + kKC - 1) / kKC;
  const int items_per_bin = n_groups * n_pass;

  if (warp == 0) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      uint32_t s = 0, p = 0;
      bool issued = false;
      for (int k = blockIdx.x; k < a.n_bins && !*abort_flag; k += gridDim.x) {
        for (int it = 0; it < items_per_bin && !*abort_flag; ++it) {
          if (!mbar_wait(acc_empty, (p & 1) ^ 1, abort_flag)) {
            *abort_flag = 1;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          bool ok = true;
          for (int t = 0; t < n_tiles; ++t, ++s) {
            const uint32_t st = s % kStages;
            if (!mbar_wait(&full[st], (s / kStages) & 1, abort_flag)) {
              *abort_flag = 1;
              ok = false;
              break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t stage = smem_u32(base + st * kStageBytes);
#pragma unroll
            for (int acc = 0; acc < kAcc; ++acc) {
              const uint32_t d = tmem + acc * kN;
              const uint32_t b_addr = stage + 2 * kTileA + acc * kTileB;
#pragma unroll
              for (int kk = 0; kk < 4; ++kk) {
                const uint64_t bd = smem_desc(b_addr + kk * 32);
                const uint64_t ahi = smem_desc(stage + kk * 32);
                const uint64_t alo = smem_desc(stage + kTileA + kk * 32);
                const uint32_t accum = (t > 0 || kk > 0) ? 1u : 0u;
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d),
                    "l"(ahi), "l"(bd), "r"(kIdesc), "r"(accum));
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d),
                    "l"(alo), "l"(bd), "r"(kIdesc), "r"(1u));
              }
            }
            issued = true;
            asm volatile(
                "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    smem_u32(&empty[st]))
                : "memory");
          }
          if (!ok) break;
          asm volatile(
              "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                  smem_u32(acc_full))
              : "memory");
          ++p;
        }
      }
      if (*abort_flag && a.status) atomicExch(a.status, FDD_ERR_TIMEOUT);
      if (issued) {  // drain this thread's MMAs before tensor memory is freed
        asm volatile(
            "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_u32(drain))
            : "memory");
        volatile int never = 0;
        mbar_wait(drain, 0, &never);
      }
    }
  } else {
    // ------------------------------------------------------------ producers
    const int pw = warp - 1;              // 0..7
    const int quarter = warp & 3;         // tensor-memory lanes this warp may read
    const int my_acc = pw / 4;            // accumulator this warp stores
    uint32_t s = 0, p = 0;
    bool ok = true;
    for (int k = blockIdx.x; k < a.n_bins && ok; k += gridDim.x) {
      const uint32_t ku = static_cast<uint32_t>(k);
      for (int it = 0; it < items_per_bin && ok; ++it) {
        const int group = it / n_pass;
        const int pass = it % n_pass;
        const int j_pass = pass * kDmsPass;  // local trial offset of this pass
        for (int t = 0; t < n_tiles; ++t, ++s) {
          const uint32_t st = s % kStages;
          // warp-uniform outcome, so the warp stays converged
          if (!__all_sync(0xffffffffu, mbar_wait(&empty[st], ((s / kStages) & 1) ^ 1, abort_flag))) {
            ok = false;
            break;
          }
          unsigned char* stage = base + st * kStageBytes;
          const int nu = t * kKC + lane;
          const bool nu_ok = nu < a.n_chan;
          PhaseConst pc = {0u, 0u, 0u, 0u};
          if (nu_ok) pc = a.pc[nu];
          // P_b = exp(2 pi i k b v): rows b = pw*16 .. pw*16+15, column pair 2*lane
#pragma unroll 4
          for (int i = 0; i < kM / kProdWarps; ++i) {
            const int b = pw * (kM / kProdWarps) + i;
            uint32_t hi_bits = 0u, lo_bits = 0u;
            if (nu_ok) {
              const float2 w = unit_phasor(top32_mul(ku * static_cast<uint32_t>(b), pc.v_lo, pc.v_hi));
              const __nv_bfloat162 hi = __floats2bfloat162_rn(w.x, w.y);
              const __nv_bfloat162 lo = __floats2bfloat162_rn(w.x - __low2float(hi),
                                                              w.y - __high2float(hi));
              hi_bits = bf16x2_bits(hi);
              lo_bits = bf16x2_bits(lo);
            }
            const uint32_t off = sw128(b, 2 * lane);
            *reinterpret_cast<uint32_t*>(stage + off) = hi_bits;
            *reinterpret_cast<uint32_t*>(stage + kTileA + off) = lo_bits;
          }
          // Q_a for this channel and the pass's 8 a's
          float2 q[kAPass];
          const uint32_t base_ph = top32_mul(ku, pc.u_lo, pc.u_hi);
#pragma unroll
          for (int al = 0; al < kAPass; ++al) {
            const uint32_t ja = static_cast<uint32_t>(a.j_begin + j_pass + al * kM);
            q[al] = nu_ok ? unit_phasor(base_ph + top32_mul(ku * ja, pc.v_lo, pc.v_hi))
                          : make_float2(0.f, 0.f);
          }
          // Z_a = Q_a X for beams beta = pw + 8m, real embedding into B
#pragma unroll
          for (int m = 0; m < kBeams / kProdWarps; ++m) {
            const int beta = pw + kProdWarps * m;
            const int bg = group * kBeams + beta;
            float2 x = make_float2(0.f, 0.f);
            if (nu_ok && bg < a.n_series)
              x = __ldg(a.X + static_cast<int64_t>(bg) * a.x_series_stride +
                        static_cast<int64_t>(nu) * a.x_chan_stride + k);
#pragma unroll
            for (int al = 0; al < kAPass; ++al) {
              const float zr = x.x * q[al].x - x.y * q[al].y;
              const float zi = x.x * q[al].y + x.y * q[al].x;
              const int acc = al / kNA;
              const int row = ((al % kNA) * kBeams + beta) * 2;
              unsigned char* tb = stage + 2 * kTileA + acc * kTileB;
              *reinterpret_cast<uint32_t*>(tb + sw128(row, 2 * lane)) =
                  bf16x2_bits(__floats2bfloat162_rn(zr, -zi));
              *reinterpret_cast<uint32_t*>(tb + sw128(row + 1, 2 * lane)) =
                  bf16x2_bits(__floats2bfloat162_rn(zi, zr));
            }
          }
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          mbar_arrive(&full[st]);
        }
        if (!ok) break;
        // epilogue: accumulator my_acc, tensor-memory lanes of this quarter
        if (!__all_sync(0xffffffffu, mbar_wait(acc_full, p & 1, abort_flag))) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int b = quarter * 32 + lane;
        const bool real_only = (k == a.real_bin_a) || (k == a.real_bin_b);
#pragma unroll 1
        for (int c0 = 0; c0 < kN; c0 += 32) {
          uint32_t r[32];
          tmem_ld32(tmem + (static_cast<uint32_t>(quarter * 32) << 16) + my_acc * kN + c0, r);
#pragma unroll
          for (int h = 0; h < 16; ++h) {
            const int n = c0 + 2 * h;            // (a_in, beta, re) column
            const int a_in = n / (2 * kBeams);
            const int beta = (n % (2 * kBeams)) / 2;
            const int bg = group * kBeams + beta;
            const int jl = j_pass + (my_acc * kNA + a_in) * kM + b;
            if (bg < a.n_series && jl < a.n_dm) {
              const float re = __uint_as_float(r[2 * h]) * a.scale;
              const float im = real_only ? 0.f : __uint_as_float(r[2 * h + 1]) * a.scale;
              const int64_t o = static_cast<int64_t>(bg) * a.y_series_stride +
                                static_cast<int64_t>(jl) * a.y_dm_stride + k;
              if (a.out_kind == 2)
                static_cast<float*>(a.Y)[o] = re * re + im * im;
              else
                static_cast<float2*>(a.Y)[o] = make_float2(re, im);
            }
          }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        mbar_arrive(acc_empty);
        ++p;
      }
    }
    if (!ok) {
      *abort_flag = 1;
      if (a.status) atomicExch(a.status, FDD_ERR_TIMEOUT);
    }
  }

  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kTmemCols));
  }
}

}  // namespace

size_t mac_tc_smem_bytes() { return kStages * kStageBytes + 1024 + 128; }

int mac_tc_trials_per_pass() { return kDmsPass; }

cudaError_t mac_tc_prepare() {
  return cudaFuncSetAttribute(mac_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              static_cast<int>(mac_tc_smem_bytes()));
}

cudaError_t launch_mac_tc(const MacArgs& a, int n_sms, cudaStream_t s) {
  if (a.n_dm <= 0 || a.n_series <= 0 || a.n_bins <= 0) return cudaSuccess;
  const int grid = a.n_bins < n_sms ? a.n_bins : n_sms;
  MacArgs args = a;
  void* params[] = {&args};
  return cudaLaunchKernel(reinterpret_cast<const void*>(&mac_tc_kernel), dim3(grid),
                          dim3(kThreads), params, mac_tc_smem_bytes(), s);
}

}  // namespace fdd

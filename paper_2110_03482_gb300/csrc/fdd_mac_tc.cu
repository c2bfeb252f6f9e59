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
// with A = [Pr | Pi] (BF16 hi + lo: two MMAs; or BF16 alone) and B the real embedding
// [[Zr, -Zi], [Zi, Zr]] of Z (BF16), FP32 accumulation in tensor memory.
// M = 128 trials b, N = 256 = 4 a's x 32 beams x (re, im), K = 64 per stage
// (32 channels x (re, im)); one pass over the channels covers 4 a's = 512
// trials, and passes alternate between two accumulators in tensor memory.
// Calls with at most 16 series use groups of 16 beams instead: N = 256 = 8 a's
// x 16 beams x (re, im), 1024 trials per pass, no idle columns.
//
// Warp specialisation: warp 0 allocates tensor memory and one of its threads
// issues the MMAs; 16 producer warps evaluate P (exact fixed-point phase,
// MUFU sin/cos and short recurrences, hi/lo split) and Z = Q X for each stage
// straight into the 128-byte-swizzled K-major shared layout the MMA
// descriptors address, through a 3-stage mbarrier ring; 4 epilogue warps read
// one accumulator back (tcgen05.ld) and store it while the MMAs of the next
// pass fill the other.  Barriers count warps (one arrive per warp).
// Every wait is bounded: on timeout the kernel records FDD_ERR_TIMEOUT in the
// status word, stops, drains its own MMAs (bounded), frees its tensor memory
// and returns.
#include <cuda_bf16.h>

#include "fdd_device.cuh"
#include "fdd_internal.h"

namespace fdd {
namespace {

using dev::mbar_arrive;
using dev::mbar_arrive_warp;
using dev::mbar_init;
using dev::mbar_wait;
using dev::smem_u32;
using dev::top32_mul;
using dev::unit_phasor;

constexpr int kM = 128;                  // trials b per a (T)
constexpr int kN = 256;                  // accumulator columns
// Beams per group (kBeams, 16 or 32) is a template parameter: a pass covers
// kNA = kN / (2 kBeams) a's, i.e. kNA * kM trials.
template <int kBeams>
__host__ __device__ constexpr int dms_per_pass() { return kN / (2 * kBeams) * kM; }
constexpr int kKC = 32;                  // channels per stage
constexpr int kProdWarps = 16;
constexpr int kProd = 32 * kProdWarps;
constexpr int kEpiWarps = 4;             // one per tensor-memory lane quarter
constexpr int kEpi = 32 * kEpiWarps;
constexpr int kThreads = 32 + kEpi + kProd;
constexpr uint32_t kTileA = kM * 64 * 2;  // 16 KB
constexpr uint32_t kTileB = kN * 64 * 2;  // 32 KB
constexpr uint32_t kStageBytes = 2 * kTileA + kTileB;  // 64 KB
constexpr int kStages = 3;
constexpr int kAccBufs = 2;              // accumulators alternate between passes
constexpr uint32_t kTmemCols = kAccBufs * kN;

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

// kHiLo: phasors as BF16 hi + lo (two MMAs per K step); otherwise BF16 only.
template <bool kHiLo, int kBeams>
__global__ void __launch_bounds__(kThreads, 1) mac_tc_kernel(const MacArgs a) {
  static_assert(kBeams == 16 || kBeams == 32, "groups of 16 or 32 beams");
  constexpr int kNA = kN / (2 * kBeams);      // a's per pass
  constexpr int kDmsPass = dms_per_pass<kBeams>();
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(base + kStages * kStageBytes);
  uint64_t* full = bars;                        // [kStages]  producers -> MMA
  uint64_t* empty = bars + kStages;             // [kStages]  MMA commit -> producers
  uint64_t* acc_full = bars + 2 * kStages;      // [kAccBufs] MMA commit -> epilogue
  uint64_t* acc_empty = acc_full + kAccBufs;    // [kAccBufs] epilogue -> MMA
  uint64_t* drain = acc_empty + kAccBufs;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int i = 0; i < kStages; ++i) {
      mbar_init(&full[i], kProdWarps);  // one arrive per producer warp
      mbar_init(&empty[i], 1);
    }
    for (int i = 0; i < kAccBufs; ++i) {
      mbar_init(&acc_full[i], 1);
      mbar_init(&acc_empty[i], kEpiWarps);  // one arrive per epilogue warp
    }
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
      bool issued = false, ok = true;
      for (int k = blockIdx.x; k < a.n_bins && ok; k += gridDim.x) {
        for (int it = 0; it < items_per_bin && ok; ++it, ++p) {
          const uint32_t buf = p % kAccBufs;
          if (!mbar_wait(&acc_empty[buf], ((p / kAccBufs) & 1) ^ 1, abort_flag)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t d = tmem + buf * kN;
          for (int t = 0; t < n_tiles; ++t, ++s) {
            const uint32_t st = s % kStages;
            if (!mbar_wait(&full[st], (s / kStages) & 1, abort_flag)) {
              ok = false;
              break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t stage = smem_u32(base + st * kStageBytes);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
              const uint64_t bd = smem_desc(stage + 2 * kTileA + kk * 32);
              const uint64_t ahi = smem_desc(stage + kk * 32);
              const uint64_t alo = smem_desc(stage + kTileA + kk * 32);
              const uint32_t accum = (t > 0 || kk > 0) ? 1u : 0u;
              asm volatile(
                  "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
                  " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d),
                  "l"(ahi), "l"(bd), "r"(kIdesc), "r"(accum));
              if (kHiLo)
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d),
                    "l"(alo), "l"(bd), "r"(kIdesc), "r"(1u));
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
                  smem_u32(&acc_full[buf]))
              : "memory");
        }
      }
      if (!ok) {
        *abort_flag = 1;
        if (a.status) atomicExch(a.status, FDD_ERR_TIMEOUT);
      }
      if (issued) {  // drain this thread's MMAs before tensor memory is freed
        asm volatile(
            "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_u32(drain))
            : "memory");
        volatile int never = 0;
        mbar_wait(drain, 0, &never);
      }
    }
  } else if (warp <= kEpiWarps) {
    // ------------------------------------------------------------ epilogue
    // Warp w reads tensor-memory lanes 32 (w mod 4) .. +31 (trials b), all 256
    // columns (a, beta, re|im) of the pass's accumulator, and stores Y.
    const int quarter = warp & 3;  // the lanes this warp may read
    const int b = quarter * 32 + lane;
    uint32_t p = 0;
    bool ok = true;
    for (int k = blockIdx.x; k < a.n_bins && ok; k += gridDim.x) {
      const bool real_only = (a.k_begin + k == a.real_bin_a) || (a.k_begin + k == a.real_bin_b);
      for (int it = 0; it < items_per_bin && ok; ++it, ++p) {
        const int group = it / n_pass;
        const int j_pass = (it % n_pass) * kDmsPass;
        const uint32_t buf = p % kAccBufs;
        if (!__all_sync(0xffffffffu, mbar_wait(&acc_full[buf], (p / kAccBufs) & 1, abort_flag))) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll 1
        for (int c0 = 0; c0 < kN; c0 += 32) {
          uint32_t r[32];
          tmem_ld32(tmem + (static_cast<uint32_t>(quarter * 32) << 16) + buf * kN + c0, r);
#pragma unroll
          for (int h = 0; h < 16; ++h) {
            const int n = c0 + 2 * h;  // (a_in, beta, re) column
            const int a_in = n / (2 * kBeams);
            const int beta = (n % (2 * kBeams)) / 2;
            const int bg = group * kBeams + beta;
            const int jl = j_pass + a_in * kM + b;
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
        mbar_arrive_warp(&acc_empty[buf]);
      }
    }
    if (!ok) {
      *abort_flag = 1;
      if (a.status) atomicExch(a.status, FDD_ERR_TIMEOUT);
    }
  } else {
    // ------------------------------------------------------------ producers
    // Producer warp pw (0..15) evaluates, for channel nu = tile*32 + lane:
    //   P_b for the 8 rows b = 8 pw .. 8 pw + 7 (one direct phasor, then the
    //   recurrence P_{b+1} = P_b R with R = exp(2 pi i k v), at most 7 steps),
    //   Q_a for the pass's kNA a's (Q_0 direct, Q_{a+1} = Q_a R^128),
    //   Z_a = Q_a X for the beams beta = pw (and pw + 16 in 32-beam groups).
    // X and the phase constants of the next tile are loaded one stage ahead.
    const int pw = warp - 1 - kEpiWarps;           // 0..15
    constexpr int kRows = kM / kProdWarps;         // P rows per warp (8)
    constexpr int kBeamsPerWarp = kBeams / kProdWarps;  // 1 or 2
    // Store offsets that do not change between stages (see sw128): the P
    // rows of this warp, and the Z rows (al*kBeams + pw + 16m)*2 + e, whose
    // position within an 8-row group depends only on pw and e.
    const uint32_t lane_chunk = static_cast<uint32_t>((lane >> 2) << 4);
    const uint32_t p_base = static_cast<uint32_t>(pw * 1024 + (lane & 3) * 4);
    uint32_t z_base[2];
#pragma unroll
    for (int e = 0; e < 2; ++e) z_base[e] = sw128(2 * pw + e, 2 * lane);  // rows < 32
    uint32_t s = 0;
    bool ok = true;
    for (int k = blockIdx.x; k < a.n_bins && ok; k += gridDim.x) {
      const uint32_t ku = static_cast<uint32_t>(a.k_begin + k);  // absolute bin
      for (int it = 0; it < items_per_bin && ok; ++it) {
        const int group = it / n_pass;
        const int j_pass = (it % n_pass) * kDmsPass;
        PhaseConst pc_next = {0u, 0u, 0u, 0u};
        float2 x_next[kBeamsPerWarp];
        {
          const int nu = lane;
          if (nu < a.n_chan) pc_next = a.pc[nu];
#pragma unroll
          for (int m = 0; m < kBeamsPerWarp; ++m) {
            const int bg = group * kBeams + pw + kProdWarps * m;
            x_next[m] = (nu < a.n_chan && bg < a.n_series)
                            ? __ldg(a.X + static_cast<int64_t>(k) * a.x_bin_stride +
                                    static_cast<int64_t>(bg) * a.x_series_stride +
                                    static_cast<int64_t>(nu) * a.x_chan_stride)
                            : make_float2(0.f, 0.f);
          }
        }
        for (int t = 0; t < n_tiles; ++t, ++s) {
          const int nu = t * kKC + lane;
          const bool nu_ok = nu < a.n_chan;
          const PhaseConst pc = pc_next;
          float2 x[kBeamsPerWarp];
#pragma unroll
          for (int m = 0; m < kBeamsPerWarp; ++m) x[m] = x_next[m];
          if (t + 1 < n_tiles) {  // prefetch the next tile
            const int nn = nu + kKC;
            pc_next = nn < a.n_chan ? a.pc[nn] : PhaseConst{0u, 0u, 0u, 0u};
#pragma unroll
            for (int m = 0; m < kBeamsPerWarp; ++m) {
              const int bg = group * kBeams + pw + kProdWarps * m;
              x_next[m] = (nn < a.n_chan && bg < a.n_series)
                              ? __ldg(a.X + static_cast<int64_t>(k) * a.x_bin_stride +
                                      static_cast<int64_t>(bg) * a.x_series_stride +
                                      static_cast<int64_t>(nn) * a.x_chan_stride)
                              : make_float2(0.f, 0.f);
            }
          }
          // phasors in registers before touching the stage
          float2 r1 = make_float2(0.f, 0.f), pb = r1, qa = r1, r128 = r1;
          if (nu_ok) {
            r1 = unit_phasor(top32_mul(ku, pc.v_lo, pc.v_hi));
            pb = unit_phasor(top32_mul(ku * static_cast<uint32_t>(pw * kRows), pc.v_lo, pc.v_hi));
            r128 = unit_phasor(top32_mul(ku * static_cast<uint32_t>(kM), pc.v_lo, pc.v_hi));
            const uint32_t ja = static_cast<uint32_t>(a.j_begin + j_pass);
            qa = unit_phasor(top32_mul(ku, pc.u_lo, pc.u_hi) + top32_mul(ku * ja, pc.v_lo, pc.v_hi));
          }
          const uint32_t st = s % kStages;
          if (!__all_sync(0xffffffffu, mbar_wait(&empty[st], ((s / kStages) & 1) ^ 1, abort_flag))) {
            ok = false;
            break;
          }
          unsigned char* stage = base + st * kStageBytes;
          // P rows b = 8 pw + i fill one 8-row swizzle group: the 16-byte chunk
          // of column pair 2*lane is (lane/4) ^ i, the rest is a constant.
#pragma unroll
          for (int i = 0; i < kRows; ++i) {
            const __nv_bfloat162 hi = __floats2bfloat162_rn(pb.x, pb.y);
            const uint32_t hb = bf16x2_bits(hi);
            // residual P - hi (the hi halves widened back to FP32)
            const float2 res = __ffma2_rn(make_float2(__uint_as_float(hb << 16),
                                                      __uint_as_float(hb & 0xFFFF0000u)),
                                          make_float2(-1.f, -1.f), pb);
            const uint32_t off = p_base + i * 128 + ((lane_chunk ^ (i << 4)));
            *reinterpret_cast<uint32_t*>(stage + off) = hb;
            if (kHiLo)
              *reinterpret_cast<uint32_t*>(stage + kTileA + off) =
                  bf16x2_bits(__floats2bfloat162_rn(res.x, res.y));
            // P <- P R as a paired multiply-add: (pr, pi) r1r + (-pi, pr) r1i
            pb = __ffma2_rn(make_float2(-pb.y, pb.x), make_float2(r1.y, r1.y),
                            __fmul2_rn(pb, make_float2(r1.x, r1.x)));
          }
          unsigned char* tb = stage + 2 * kTileA;
#pragma unroll
          for (int al = 0; al < kNA; ++al) {
#pragma unroll
            for (int m = 0; m < kBeamsPerWarp; ++m) {
              // Z = X Q as (xr, xr)(qr, qi) + (-xi, xi)(qi, qr)
              const float2 z = __ffma2_rn(make_float2(-x[m].y, x[m].y), make_float2(qa.y, qa.x),
                                          __fmul2_rn(make_float2(x[m].x, x[m].x), qa));
              const uint32_t zb = bf16x2_bits(__floats2bfloat162_rn(z.x, z.y));
              // rows (al*kBeams + beta)*2 + {0, 1}: per-thread base + a constant
              const uint32_t row_off = static_cast<uint32_t>((kBeams / 4 * al + 4 * m) * 1024);
              *reinterpret_cast<uint32_t*>(tb + z_base[0] + row_off) = zb ^ 0x80000000u;  // (zr, -zi)
              *reinterpret_cast<uint32_t*>(tb + z_base[1] + row_off) = __byte_perm(zb, 0, 0x1032);  // (zi, zr)
            }
            qa = __ffma2_rn(make_float2(-qa.y, qa.x), make_float2(r128.y, r128.y),
                            __fmul2_rn(qa, make_float2(r128.x, r128.x)));
          }
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          if (!a.test_withhold) mbar_arrive_warp(&full[st]);
        }
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

int mac_tc_beams_per_group(int n_series) { return n_series <= 16 ? 16 : 32; }

int mac_tc_trials_per_pass(int n_series) {
  return mac_tc_beams_per_group(n_series) == 16 ? dms_per_pass<16>() : dms_per_pass<32>();
}

cudaError_t mac_tc_prepare() {
  const void* fns[] = {reinterpret_cast<const void*>(&mac_tc_kernel<true, 32>),
                       reinterpret_cast<const void*>(&mac_tc_kernel<false, 32>),
                       reinterpret_cast<const void*>(&mac_tc_kernel<true, 16>),
                       reinterpret_cast<const void*>(&mac_tc_kernel<false, 16>)};
  for (const void* fn : fns) {
    const cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               static_cast<int>(mac_tc_smem_bytes()));
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

static cudaError_t launch_mac_tc_block(const MacArgs& a, bool hi_lo, int n_sms, cudaStream_t s);

size_t mac_tc_scratch_bytes(int n_series, int n_chan, int64_t n_bins) {
  const size_t per_bin = sizeof(float2) * static_cast<size_t>(n_series) * n_chan;
  const size_t cap = size_t(2) << 30;
  int64_t kb = static_cast<int64_t>(cap / per_bin);
  if (kb < 1) kb = 1;
  if (kb > n_bins) kb = n_bins;
  return per_bin * static_cast<size_t>(kb);
}

cudaError_t launch_mac_tc(const MacArgs& a, bool hi_lo, int n_sms, float2* scratch,
                          size_t scratch_bytes, cudaStream_t s) {
  if (a.n_dm <= 0 || a.n_series <= 0 || a.n_bins <= 0) return cudaSuccess;
  if (a.x_series_stride != a.x_chan_stride * a.n_chan) return cudaErrorInvalidValue;
  const int64_t rows = static_cast<int64_t>(a.n_series) * a.n_chan;
  const int64_t kb = static_cast<int64_t>(scratch_bytes / (sizeof(float2) * rows));
  if (!scratch || kb < 1) return cudaErrorInvalidValue;
  const size_t y_elem = a.out_kind == 2 ? sizeof(float) : sizeof(float2);
  for (int64_t k0 = 0; k0 < a.n_bins; k0 += kb) {
    const int nb = static_cast<int>((a.n_bins - k0) < kb ? (a.n_bins - k0) : kb);
    BinTransposeArgs t{a.X, a.x_chan_stride, rows, k0, nb, scratch};
    cudaError_t e = launch_bin_transpose(t, s);
    if (e != cudaSuccess) return e;
    MacArgs b = a;
    b.X = scratch;
    b.x_bin_stride = rows;
    b.x_series_stride = a.n_chan;
    b.x_chan_stride = 1;
    b.n_bins = nb;
    b.k_begin = a.k_begin + static_cast<int>(k0);
    b.Y = static_cast<char*>(a.Y) + y_elem * static_cast<size_t>(k0);
    e = launch_mac_tc_block(b, hi_lo, n_sms, s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

static cudaError_t launch_mac_tc_block(const MacArgs& a, bool hi_lo, int n_sms, cudaStream_t s) {
  const int grid = a.n_bins < n_sms ? a.n_bins : n_sms;
  MacArgs args = a;
  void* params[] = {&args};
  const bool g16 = mac_tc_beams_per_group(a.n_series) == 16;
  const void* fn =
      hi_lo ? (g16 ? reinterpret_cast<const void*>(&mac_tc_kernel<true, 16>)
                   : reinterpret_cast<const void*>(&mac_tc_kernel<true, 32>))
            : (g16 ? reinterpret_cast<const void*>(&mac_tc_kernel<false, 16>)
                   : reinterpret_cast<const void*>(&mac_tc_kernel<false, 32>));
  return cudaLaunchKernel(fn, dim3(grid),
                          dim3(kThreads), params, mac_tc_smem_bytes(), s);
}

}  // namespace fdd

// fdd_mac_tc.cu -- phase-rotate-and-sum on the tensor cores (tcgen05 + TMEM)
// for many beams sharing the same Fourier bins (the tensor-core and
// phasor-reuse directions of Sect. 5 of the paper).
//
// With the trial index split j = aT + b (T = 128, or 256 on a CTA pair), the
// phasor of Eq. 4 factorises as W(aT + b) = Q_a P_b (see fdd_mac_fp32.cu), so
// for one bin k and beams beta
//
//   Y[aT + b][beta] = sum_nu P_b[nu] Z_a[nu][beta],   Z_a = Q_a X[nu][beta],
//
// i.e. for every group of a's one complex GEMM of (T x N_nu) phasors P by
// (N_nu x beams) data.  It runs on tcgen05 as two real GEMMs that share one B
// operand.  With K = (nu, re|im) and B[(a, beta)][(nu, c)] = (Zr, Zi)[nu]:
//
//   D_re[b][(a, beta)] = sum_K A_re[b][K] B[(a, beta)][K],   A_re = (Pr, -Pi),
//   D_im[b][(a, beta)] = sum_K A_im[b][K] B[(a, beta)][K],   A_im = (Pi,  Pr),
//
// i.e. Re and Im of P Z.  Operands are BF16 (phasors hi + lo: four MMAs per K
// step; or hi alone: two) or FP16 (two MMAs; each bin's data scaled by a power
// of two so its largest component lands near 2^14, undone in the epilogue),
// accumulation FP32 in tensor memory.  M = 128
// trials b per CTA, N = 256 (a, beta) pairs (8 a's x 32 beams, or 16 a's x 16
// beams for calls with at most 16 series), K = 64 per stage (32 channels x
// (re, im)).  D_re and D_im fill all 512 tensor-memory columns, so one pass
// over the channels covers 1024 trials (2048 in 16-beam groups), twice that
// on a CTA pair (M = 256 over two SMs, each CTA building half of B): every P
// tile the producers build serves 256 output columns, and every Z value is
// written to shared memory once.
//
// Warp specialisation: warp 0 allocates tensor memory and one of its threads
// issues the MMAs; 16 producer warps evaluate P (exact fixed-point phase,
// MUFU sin/cos and short recurrences, hi/lo split) and Z = Q X for each stage
// straight into the 128-byte-swizzled K-major shared layout the MMA
// descriptors address, through an mbarrier ring (2 stages of 96 KB with hi +
// lo phasors, 3 of 64 KB without; a pair's CTA holds half of B: 2 of 80 KB
// or 4 of 48 KB); 4 epilogue warps read the accumulators
// back (tcgen05.ld) and store them, while the producers already fill the ring
// for the next pass.  The kernel writes Y bin-major, [bin][series][trial], so
// each warp store covers 256 contiguous bytes; launch_mac_tc then moves it
// into the caller's layout (bins innermost) with an HBM-bound transpose.
// (Stored straight into that layout, each 8-byte value of one bin is its own
// partial sector, and those scattered stores cost more than the transpose.)
// Barriers count warps (one arrive per warp).  Every wait is bounded: on
// timeout the kernel records FDD_ERR_TIMEOUT in the status word, stops,
// drains its own MMAs (bounded), frees its tensor memory and returns.
#include <atomic>

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

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

constexpr int kM = 128;                  // trials b per CTA (tensor-memory lanes)
constexpr int kN = 256;                  // (a, beta) columns of each accumulator
// Trials per a: T = 128 for one CTA; a CTA pair (kPair, one MMA of M = 256
// over both CTAs' tensor cores) takes T = 256, rows b < 128 in the first CTA.
template <bool kPair>
__host__ __device__ constexpr int trials_per_a() { return kPair ? 2 * kM : kM; }
// Beams per group (kBeams, 16 or 32) is a template parameter: a pass covers
// kN / kBeams a's, i.e. kN / kBeams * T trials.
template <int kBeams, bool kPair>
__host__ __device__ constexpr int dms_per_pass() { return kN / kBeams * trials_per_a<kPair>(); }
constexpr int kKC = 32;                  // channels per stage of 16-bit operands
constexpr int kProdWarps = 16;
constexpr int kEpiWarps = 4;             // one per tensor-memory lane quarter
constexpr int kThreads = 32 + 32 * kEpiWarps + 32 * kProdWarps;
constexpr uint32_t kTileA = kM * 64 * 2;  // 16 KB
constexpr uint32_t kTileB = kN * 64 * 2;  // 32 KB
constexpr uint32_t kRingBytes = 192 * 1024;
// Stage layout: A_re hi, A_im hi (, A_re lo, A_im lo), then B (a CTA of a
// pair holds half of B's rows).
template <bool kHiLo, bool kPair>
struct Ring {
  static constexpr int kATiles = kHiLo ? 4 : 2;
  static constexpr uint32_t kBOff = kATiles * kTileA;
  static constexpr uint32_t kStageBytes = kBOff + (kPair ? kTileB / 2 : kTileB);
  static constexpr int kStages = kRingBytes / kStageBytes;  // 2 or 3; a pair 2 or 4
};
constexpr uint32_t kTmemCols = 2 * kN;   // D_re | D_im

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

// Operand precisions of the kernel (from fdd_params.precision).
enum TcPrec { kBf16HiLo = 0, kBf16 = 1, kF16 = 2, kF8 = 3 };

// Instruction descriptor: D FP32, A and B both BF16 (format 1) or both FP16
// (format 0) under kind::f16, both E4M3 (format 0) under kind::f8f6f4; both
// K-major, N and M.
// n: the MMA's N, a multiple of 16 in [16, kN] (a pass's last a's may be
// fewer than the kN / kBeams of a full pass); m: 128, or 256 for a CTA pair.
template <int kPrec>
__host__ __device__ constexpr uint32_t idesc(int n, int m) {
  return (1u << 4) | ((kPrec == kF16 || kPrec == kF8) ? 0u : ((1u << 7) | (1u << 10))) |
         (static_cast<uint32_t>(n >> 3) << 17) | (static_cast<uint32_t>(m >> 4) << 24);
}

// a's of the pass from trial j_pass: all kNA of a full pass, fewer (whole
// a's of kT trials) where the trials end within it
__device__ __forceinline__ int pass_as(int n_dm, int j_pass, int kNA, int kT) {
  const int left = (n_dm - j_pass + kT - 1) / kT;
  return left < kNA ? left : kNA;
}

__device__ __forceinline__ uint32_t bf16x2_bits(__nv_bfloat162 v) {
  return *reinterpret_cast<uint32_t*>(&v);
}

// Four bytes of one K-major row for kCpl channels: (re, im) of one channel in
// the 16-bit types (re in the low half), or (re0, im0, re1, im1) of two
// adjacent channels in FP8 E4M3 (re0 in the lowest byte).
template <int kPrec>
__device__ __forceinline__ uint32_t pack2(float x, float y);
template <int kPrec, int kCpl>
__device__ __forceinline__ uint32_t pack_word(const float2 (&v)[kCpl]) {
  if constexpr (kPrec == kF8) {
    const uint32_t lo = __nv_cvt_float2_to_fp8x2(v[0], __NV_SATFINITE, __NV_E4M3);
    const uint32_t hi = __nv_cvt_float2_to_fp8x2(v[kCpl - 1], __NV_SATFINITE, __NV_E4M3);
    return lo | (hi << 16);
  } else {
    return pack2<kPrec>(v[0].x, v[0].y);
  }
}
// (re, im) -> (re, -im) and -> (im, re) on every channel of a packed word.
template <int kPrec>
__device__ __forceinline__ constexpr uint32_t neg_im_mask() {
  return kPrec == kF8 ? 0x80008000u : 0x80000000u;
}
template <int kPrec>
__device__ __forceinline__ uint32_t swap_re_im(uint32_t w) {
  return __byte_perm(w, 0, kPrec == kF8 ? 0x2301 : 0x1032);
}

// (x, y) rounded to the kernel's 16-bit operand type, x in the low half.
template <int kPrec>
__device__ __forceinline__ uint32_t pack2(float x, float y) {
  if constexpr (kPrec == kF16) {
    __half2 h = __floats2half2_rn(x, y);
    return *reinterpret_cast<uint32_t*>(&h);
  } else {
    return bf16x2_bits(__floats2bfloat162_rn(x, y));
  }
}

// Data scale of a bin whose largest |re| or |im| is m, for the operand types
// of limited range: with E the biased exponent of m (m < 2^(E - 126)), the
// power of two 2^(T + 126 - E), so that m times it is below 2^T and every
// component of Z = Q X (|Z| <= sqrt(2) m) stays below 2^(T + 0.5): T = 14 for
// FP16 (largest 65504), T = 8 for FP8 E4M3 (largest 448).  Powers of two keep
// the scaling and its undoing exact.
template <int kPrec>
__device__ __forceinline__ float bin_scale(float m) {
  constexpr int kT = kPrec == kF8 ? 8 : 14;
  const int e = static_cast<int>((__float_as_uint(m) >> 23) & 0xFFu);
  int f = kT + 253 - e;  // biased exponent of 2^(T + 126 - E)
  f = f < 1 ? 1 : (f > 253 ? 253 : f);
  return __uint_as_float(static_cast<uint32_t>(f) << 23);
}

// 16 consecutive FP32 columns of this warp's 32 tensor-memory lanes, from two
// places at once (one wait for both loads).
__device__ __forceinline__ void tmem_ld16x2(uint32_t ta, uint32_t tb, uint32_t (&r)[16],
                                            uint32_t (&q)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(ta));
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15}, [%16];"
      : "=r"(q[0]), "=r"(q[1]), "=r"(q[2]), "=r"(q[3]), "=r"(q[4]), "=r"(q[5]), "=r"(q[6]),
        "=r"(q[7]), "=r"(q[8]), "=r"(q[9]), "=r"(q[10]), "=r"(q[11]), "=r"(q[12]), "=r"(q[13]),
        "=r"(q[14]), "=r"(q[15])
      : "r"(tb));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// D (+)= A B^T for one K step of 32 bytes: M = 128 (256 over a CTA pair),
// N up to 256, FP32 out; 16 elements of 16 bits (kind::f16) or 32 of FP8 E4M3
// (kind::f8f6f4).  A CTA pair's MMA, issued by the first CTA, reads each
// CTA's 128 rows of A and its N / 2 rows of B at the same shared-memory
// offsets and writes each CTA's 128 rows of D into its own tensor memory.
template <int kPrec, bool kPair>
__device__ __forceinline__ void mma16(uint32_t d, uint64_t adesc, uint64_t bdesc,
                                      uint32_t accum, uint32_t id) {
  if constexpr (kPrec == kF8 && kPair) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::2.kind::f8f6f4 [%0], %1, %2, %3, p;\n}" ::"r"(d),
        "l"(adesc), "l"(bdesc), "r"(id), "r"(accum));
  } else if constexpr (kPrec == kF8) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}" ::"r"(d),
        "l"(adesc), "l"(bdesc), "r"(id), "r"(accum));
  } else if constexpr (kPair) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d),
        "l"(adesc), "l"(bdesc), "r"(id), "r"(accum));
  } else {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d),
        "l"(adesc), "l"(bdesc), "r"(id), "r"(accum));
  }
}

// Completion of this thread's earlier MMAs arrives once on the barrier at
// this shared-memory offset: in this CTA, or in both CTAs of a pair.
template <bool kPair>
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  if constexpr (kPair) {
    const uint16_t both = 3;
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64"
        " [%0], %1;" ::"r"(smem_u32(bar)),
        "h"(both)
        : "memory");
  } else {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar))
        : "memory");
  }
}

// The same, arriving on this CTA's barrier only.
template <bool kPair>
__device__ __forceinline__ void mma_commit_one(uint64_t* bar) {
  if constexpr (kPair) {
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar))
        : "memory");
  } else {
    mma_commit<false>(bar);
  }
}

// ---- CTA pairs (clusters of two): rank, pair index, barriers in the first CTA
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cluster_index() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cluster_count() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%nclusterid.x;" : "=r"(r));
  return r;
}
// Every thread of both CTAs: earlier accesses (release) before later ones
// (acquire) of any thread of the pair.
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release;\nbarrier.cluster.wait.acquire;" ::: "memory");
}
// Bounded wait at cluster scope (arrivals from the other CTA of the pair).
__device__ __forceinline__ bool mbar_wait_cluster(uint64_t* bar, uint32_t parity,
                                                  volatile int* abort_flag) {
  const long long t0 = clock64();
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    if (done) return true;
    if (*abort_flag) return false;
    if (clock64() - t0 > dev::kWaitCycles) return false;
  }
}
template <bool kPair>
__device__ __forceinline__ bool wait_bar(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
  if constexpr (kPair)
    return mbar_wait_cluster(bar, parity, abort_flag);
  else
    return mbar_wait(bar, parity, abort_flag);
}

// 21 warps at one CTA per SM: one of the four schedulers holds six of them,
// and a scheduler's 16384 registers cap the kernel at 80 per thread.
// kPrec: kBf16HiLo (phasors as BF16 hi + lo, four MMAs per K step), kBf16
// (BF16 only), kF16 (FP16 phasors and scaled FP16 data) or kF8 (FP8 E4M3
// phasors and scaled E4M3 data, kind::f8f6f4, 64 channels per stage).
// kPair: launched in clusters of two CTAs, each pair working on one bin at a
// time with T = 256: the first CTA's MMA warp issues M = 256 MMAs over both
// CTAs (rows b < 128 from the first CTA, the rest from the second), each CTA
// builds its own 128 rows of P and half of the pass's Z columns (the first
// or the second half of its a's), so a CTA builds half the Z values per MMA
// it would alone.  Producers and epilogue warps arrive on their own CTA's
// barriers; in the second CTA one thread of warp 0 forwards each completed
// stage and read-out to the first CTA's barriers (one cluster-scope release
// per stage instead of one per producer warp, which cost more than the
// pairing saved), and the MMAs' completion reaches both CTAs' barriers.
template <int kPrec, int kBeams, bool kPair>
__global__ void __launch_bounds__(kThreads, 1) mac_tc_kernel(const MacArgs a) {
  static_assert(kBeams == 16 || kBeams == 32, "groups of 16 or 32 beams");
  constexpr bool kHiLo = kPrec == kBf16HiLo;
  constexpr bool kScaled = kPrec == kF16 || kPrec == kF8;  // per-bin data scale
  constexpr int kCpl = kPrec == kF8 ? 2 : 1;               // channels per producer lane
  constexpr int kKCp = kKC * kCpl;                         // channels per stage
  constexpr int kT = trials_per_a<kPair>();   // trials per a
  constexpr int kNA = kN / kBeams;            // a's per pass (8 or 16)
  constexpr int kNAc = kPair ? kNA / 2 : kNA;  // a's whose Z this CTA builds
  constexpr int kDmsPass = dms_per_pass<kBeams, kPair>();
  constexpr int kStages = Ring<kHiLo, kPair>::kStages;
  constexpr uint32_t kStageBytes = Ring<kHiLo, kPair>::kStageBytes;
  constexpr uint32_t kBOff = Ring<kHiLo, kPair>::kBOff;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(base + kRingBytes);
  uint64_t* full = bars;                        // [kStages]  producers -> MMA
  uint64_t* empty = bars + kStages;             // [kStages]  MMA commit -> producers
  uint64_t* acc_full = bars + 2 * kStages;      // MMA commit -> epilogue
  uint64_t* acc_empty = acc_full + 1;           // epilogue -> MMA
  uint64_t* drain = acc_empty + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  // this CTA's place in its pair (0 alone), the unit of bins and their count
  const int rank = kPair ? static_cast<int>(cluster_rank()) : 0;
  const int unit = kPair ? static_cast<int>(cluster_index()) : static_cast<int>(blockIdx.x);
  const int n_units = kPair ? static_cast<int>(cluster_count()) : static_cast<int>(gridDim.x);
  constexpr int kCtas = kPair ? 2 : 1;
  if (threadIdx.x == 0) {
    for (int i = 0; i < kStages; ++i) {
      // one arrive per producer warp; in a pair's first CTA one more from the
      // second CTA's forwarder
      mbar_init(&full[i], kProdWarps + (kPair && rank == 0 ? 1 : 0));
      mbar_init(&empty[i], 1);
    }
    mbar_init(acc_full, 1);
    mbar_init(acc_empty, kEpiWarps + (kPair && rank == 0 ? 1 : 0));  // likewise
    mbar_init(drain, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  if (warp == 0) {
    if constexpr (kPair) {
      asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                       smem_u32(tmem_slot)),
                   "r"(kTmemCols));
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;");
    } else {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                       smem_u32(tmem_slot)),
                   "r"(kTmemCols));
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if constexpr (kPair) cluster_sync();  // both CTAs' barriers exist before any remote arrive
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  const int n_groups = (a.n_series + kBeams - 1) / kBeams;
  const int n_pass = (a.n_dm + kDmsPass - 1) / kDmsPass;
  const int n_tiles = (a.n_chan + kKCp - 1) / kKCp;
  const int items_per_bin = n_groups * n_pass;
  // a's of a pass with n_a of them: the MMA's (even for a pair, whose two
  // CTAs hold half each) and, per CTA, how many and from which one it builds
  auto mma_as = [&](int n_a) { return kPair ? (n_a + 1) & ~1 : n_a; };
  auto cta_first_a = [&](int n_a) { return kPair ? rank * (mma_as(n_a) / 2) : 0; };
  auto cta_as = [&](int n_a) { return kPair ? mma_as(n_a) / 2 : n_a; };

  if (warp == 0) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0 && rank == 0) {
      uint32_t s = 0, p = 0;
      bool issued = false, ok = true;
      for (int k = unit; k < a.n_bins && ok; k += n_units) {
        for (int it = 0; it < items_per_bin && ok; ++it, ++p) {
          // the epilogue (of both CTAs) has read the previous pass out of tensor memory
          if (!wait_bar<kPair>(acc_empty, (p & 1) ^ 1, abort_flag)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          // N of this pass: its a's times the group's beams
          const int n_a = pass_as(a.n_dm, (it % n_pass) * kDmsPass, kNA, kT);
          const uint32_t id = idesc<kPrec>(mma_as(n_a) * kBeams, kCtas * kM);
          for (int t = 0; t < n_tiles; ++t, ++s) {
            const uint32_t st = s % kStages;
            if (!wait_bar<kPair>(&full[st], (s / kStages) & 1, abort_flag)) {
              ok = false;
              break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t stage = smem_u32(base + st * kStageBytes);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
              const uint64_t bd = smem_desc(stage + kBOff + kk * 32);
              const uint32_t accum = (t > 0 || kk > 0) ? 1u : 0u;
              mma16<kPrec, kPair>(tmem, smem_desc(stage + kk * 32), bd, accum, id);  // re, hi
              mma16<kPrec, kPair>(tmem + kN, smem_desc(stage + kTileA + kk * 32), bd, accum,
                                  id);  // im, hi
              if (kHiLo) {
                mma16<kPrec, kPair>(tmem, smem_desc(stage + 2 * kTileA + kk * 32), bd, 1u,
                                    id);  // re, lo
                mma16<kPrec, kPair>(tmem + kN, smem_desc(stage + 3 * kTileA + kk * 32), bd, 1u,
                                    id);  // im, lo
              }
            }
            issued = true;
            mma_commit<kPair>(&empty[st]);
          }
          if (!ok) break;
          mma_commit<kPair>(acc_full);
        }
      }
      if (!ok) {
        *abort_flag = 1;
        if (a.status) atomicExch(a.status, FDD_ERR_TIMEOUT);
      }
      if (issued) {  // drain this thread's MMAs before tensor memory is freed
        mma_commit_one<kPair>(drain);
        volatile int never = 0;
        mbar_wait(drain, 0, &never);
      }
    } else if (kPair && lane == 0) {
      // forwarder of a pair's second CTA: each stage its producers filled and
      // each pass its epilogue read out (their arrives, CTA scope) is passed
      // on as one arrive on the first CTA's barrier at cluster scope, so that
      // no producer or epilogue warp waits on a cluster-scope release of its
      // own loads and stores in flight
      uint32_t s = 0, p = 0;
      bool ok = true;
      auto forward = [&](uint64_t* bar) {
        uint32_t remote;
        asm volatile("mapa.shared::cluster.u32 %0, %1, 0;" : "=r"(remote) : "r"(smem_u32(bar)));
        asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(remote)
                     : "memory");
      };
      for (int k = unit; k < a.n_bins && ok; k += n_units) {
        for (int it = 0; it < items_per_bin && ok; ++it, ++p) {
          // the previous pass read out here (the first CTA's MMAs wait for it)
          if (p > 0) {
            if (!mbar_wait(acc_empty, (p - 1) & 1, abort_flag)) {
              ok = false;
              break;
            }
            forward(acc_empty);
          }
          for (int t = 0; t < n_tiles; ++t, ++s) {
            const uint32_t st = s % kStages;
            if (!mbar_wait(&full[st], (s / kStages) & 1, abort_flag)) {
              ok = false;
              break;
            }
            forward(&full[st]);
          }
        }
      }
      if (!ok) {
        *abort_flag = 1;
        if (a.status) atomicExch(a.status, FDD_ERR_TIMEOUT);
      }
    }
  } else if (warp <= kEpiWarps) {
    // ------------------------------------------------------------ epilogue
    // Warp w reads tensor-memory lanes 32 (w mod 4) .. +31 (trials b of this
    // CTA) of D_re and D_im, all (a, beta) columns, and stores
    // Y[k][beta][aT + b]: the warp's 32 lanes write 32 consecutive trials.
    const int quarter = warp & 3;  // the lanes this warp may read
    const int b = rank * kM + quarter * 32 + lane;
    const uint32_t t_lanes = tmem + (static_cast<uint32_t>(quarter * 32) << 16);
    uint32_t p = 0;
    bool ok = true;
    for (int k = unit; k < a.n_bins && ok; k += n_units) {
      const bool real_only = (a.k_begin + k == a.real_bin_a) || (a.k_begin + k == a.real_bin_b);
      // FP16: undo the bin's data scale (a power of two, so exactly)
      const float sy = kScaled ? a.scale / bin_scale<kPrec>(a.bin_absmax[k]) : a.scale;
      const float2 sc = make_float2(sy, real_only ? 0.f : sy);
      const int64_t o_bin = static_cast<int64_t>(k) * a.y_bin_stride;
      for (int it = 0; it < items_per_bin && ok; ++it, ++p) {
        const int group = it / n_pass;
        const int j_pass = (it % n_pass) * kDmsPass;
        if (!__all_sync(0xffffffffu, wait_bar<kPair>(acc_full, p & 1, abort_flag))) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // columns of the pass's a's that have trials
        const int n_cols = pass_as(a.n_dm, j_pass, kNA, kT) * kBeams;
#pragma unroll 1
        for (int c0 = 0; c0 < n_cols; c0 += 16) {
          uint32_t re[16], im[16];
          tmem_ld16x2(t_lanes + c0, t_lanes + kN + c0, re, im);
          // the 16 columns share a_in = c0 / kBeams; beams beta0 .. beta0 + 15
          const int bg0 = group * kBeams + c0 % kBeams;
          const int jl = j_pass + (c0 / kBeams) * kT + b;
          const int n_valid = a.n_series - bg0;  // beams of this chunk in range (may be <= 0)
          if (jl < a.n_dm && n_valid > 0) {
            const int64_t o0 = o_bin + static_cast<int64_t>(bg0) * a.y_series_stride +
                               static_cast<int64_t>(jl) * a.y_dm_stride;
            if (a.out_kind == 2) {
              float* q = static_cast<float*>(a.Y) + o0;
#pragma unroll
              for (int h = 0; h < 16; ++h) {
                const float2 y =
                    __fmul2_rn(make_float2(__uint_as_float(re[h]), __uint_as_float(im[h])), sc);
                if (h < n_valid) q[h * a.y_series_stride] = y.x * y.x + y.y * y.y;
              }
            } else {
              float2* q = static_cast<float2*>(a.Y) + o0;
#pragma unroll
              for (int h = 0; h < 16; ++h) {
                const float2 y =
                    __fmul2_rn(make_float2(__uint_as_float(re[h]), __uint_as_float(im[h])), sc);
                if (h < n_valid) q[h * a.y_series_stride] = y;
              }
            }
          }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        mbar_arrive_warp(acc_empty);  // (a pair's second CTA forwards it)
      }
    }
    if (!ok) {
      *abort_flag = 1;
      if (a.status) atomicExch(a.status, FDD_ERR_TIMEOUT);
    }
  } else {
    // ------------------------------------------------------------ producers
    // Producer warp pw (0..15) evaluates, for the channels nu = tile * kKCp +
    // kCpl * lane + cl (cl < kCpl: one channel per lane for 16-bit operands,
    // two adjacent ones for 8-bit, so every lane writes four bytes per row):
    //   P_b for the 8 rows b = 128 rank + 8 pw .. + 7 (one direct phasor,
    //   then the recurrence P_{b+1} = P_b R with R = exp(2 pi i k v), at most
    //   7 steps), stored as the A_re and A_im rows (hi, and lo = P - hi);
    //   Q_a for this CTA's a's of the pass as two chains (Q of each chain's
    //   first a direct, then Q_{a+1} = Q_a R^T),
    //   Z_a = Q_a X for the beams beta = pw (and pw + 16 in 32-beam groups).
    // X and the phase constants run two tiles ahead.
    const int pw = warp - 1 - kEpiWarps;           // 0..15
    constexpr int kRows = kM / kProdWarps;         // P rows per warp (8)
    constexpr int kBeamsPerWarp = kBeams / kProdWarps;  // 1 or 2
    constexpr int kHalfA = kNAc / 2;               // a's per Q chain
    constexpr int kProdUnroll = (kHiLo || kPrec == kF8) ? 1 : 2;
    // Store offsets that do not change between stages (see sw128): the P
    // rows of this warp, and the B rows a_local * kBeams + pw + 16 m, whose
    // position within an 8-row group is pw mod 8.  A lane's four bytes sit
    // at the same place for either operand width.
    const uint32_t lane_chunk = static_cast<uint32_t>((lane >> 2) << 4);
    const uint32_t p_base = static_cast<uint32_t>(pw * 1024 + (lane & 3) * 4);
    const uint32_t z_base = sw128(pw, 2 * lane);  // row pw < 16
    const uint32_t b_first = static_cast<uint32_t>(rank * kM + pw * kRows);  // first P row's b
    uint32_t s = 0;
    bool ok = true;
    for (int k = unit; k < a.n_bins && ok; k += n_units) {
      // absolute bin of the phasors (groups of bins sharing a reference bin
      // under spin-frequency-dependent grids step by the group size)
      const uint32_t ku = static_cast<uint32_t>(a.k_begin + k * (a.k_step > 0 ? a.k_step : 1));
      const float sx = kScaled ? bin_scale<kPrec>(a.bin_absmax[k]) : 1.f;  // data scale
      for (int it = 0; it < items_per_bin && ok; ++it) {
        const int group = it / n_pass;
        const int j_pass = (it % n_pass) * kDmsPass;
        const int n_a = pass_as(a.n_dm, j_pass, kNA, kT);  // a's of this pass with trials
        const int a_first = cta_first_a(n_a);              // this CTA's first a
        const int n_mine = cta_as(n_a);                    // and its count
        auto load_pc = [&](int nn) {
          return nn < a.n_chan ? a.pc[nn] : PhaseConst{0u, 0u, 0u, 0u};
        };
        auto load_x = [&](int nn, int m) {
          const int bg = group * kBeams + pw + kProdWarps * m;
          return (nn < a.n_chan && bg < a.n_series)
                     ? __ldg(a.X + static_cast<int64_t>(k) * a.x_bin_stride +
                             static_cast<int64_t>(bg) * a.x_series_stride +
                             static_cast<int64_t>(nn) * a.x_chan_stride)
                     : make_float2(0.f, 0.f);
        };
        // a_local (< kNAc) is stored where this CTA holds it and it has trials
        auto keep = [&](int a_local) { return a_local < n_mine && a_first + a_local < n_a; };
        PhaseConst pc_n1[kCpl], pc_n2[kCpl];
        float2 x_n1[kCpl][kBeamsPerWarp], x_n2[kCpl][kBeamsPerWarp];
#pragma unroll
        for (int cl = 0; cl < kCpl; ++cl) {
          pc_n1[cl] = load_pc(kCpl * lane + cl);
          pc_n2[cl] = load_pc(kKCp + kCpl * lane + cl);
#pragma unroll
          for (int m = 0; m < kBeamsPerWarp; ++m) {
            x_n1[cl][m] = load_x(kCpl * lane + cl, m);
            x_n2[cl][m] = load_x(kKCp + kCpl * lane + cl, m);
          }
        }
        // (16-bit forms unrolled by two: the register sets of the tile after
        // next and the next one trade names instead of being copied, so a
        // prefetched value is first read two stages after its load; measured
        // 1-2 % faster for FP16, while hi+lo and FP8, short of registers,
        // spilled and lost as much)
#pragma unroll (kProdUnroll)
        for (int t = 0; t < n_tiles; ++t, ++s) {
          const int nu0 = t * kKCp + kCpl * lane;
          PhaseConst pc[kCpl];
          float2 x[kCpl][kBeamsPerWarp];
#pragma unroll
          for (int cl = 0; cl < kCpl; ++cl) {
            pc[cl] = pc_n1[cl];
            pc_n1[cl] = pc_n2[cl];
#pragma unroll
            for (int m = 0; m < kBeamsPerWarp; ++m) {
              x[cl][m] = kScaled ? make_float2(x_n1[cl][m].x * sx, x_n1[cl][m].y * sx)
                                 : x_n1[cl][m];
              x_n1[cl][m] = x_n2[cl][m];
            }
            if (t + 2 < n_tiles) {  // prefetch the tile after next
              const int nn = nu0 + 2 * kKCp + cl;
              pc_n2[cl] = load_pc(nn);
#pragma unroll
              for (int m = 0; m < kBeamsPerWarp; ++m) x_n2[cl][m] = load_x(nn, m);
            }
          }
          // phasors in registers before touching the stage (zero beyond n_chan)
          float2 r1[kCpl], pb[kCpl], rT[kCpl], qa[kCpl], qb[kCpl];
#pragma unroll
          for (int cl = 0; cl < kCpl; ++cl) {
            r1[cl] = pb[cl] = rT[cl] = qa[cl] = qb[cl] = make_float2(0.f, 0.f);
            if (nu0 + cl < a.n_chan) {
              const PhaseConst& q = pc[cl];
              r1[cl] = unit_phasor(top32_mul(ku, q.v_lo, q.v_hi));
              pb[cl] = unit_phasor(top32_mul(ku * b_first, q.v_lo, q.v_hi));
              rT[cl] = unit_phasor(top32_mul(ku * static_cast<uint32_t>(kT), q.v_lo, q.v_hi));
              const uint32_t ja =
                  static_cast<uint32_t>(a.j_begin + j_pass + a_first * kT);  // first a's trial
              const uint32_t ph_u = top32_mul(ku, q.u_lo, q.u_hi);
              qa[cl] = unit_phasor(ph_u + top32_mul(ku * ja, q.v_lo, q.v_hi));
              qb[cl] = unit_phasor(ph_u + top32_mul(ku * (ja + static_cast<uint32_t>(kHalfA * kT)),
                                                    q.v_lo, q.v_hi));
            }
          }
          const uint32_t st = s % kStages;
          if (!__all_sync(0xffffffffu,
                          wait_bar<kPair>(&empty[st], ((s / kStages) & 1) ^ 1, abort_flag))) {
            ok = false;
            break;
          }
          unsigned char* stage = base + st * kStageBytes;
          // A rows b = 8 pw + i fill one 8-row swizzle group: the 16-byte chunk
          // of the lane's four bytes is (lane/4) ^ i, the rest is a constant.
#pragma unroll
          for (int i = 0; i < kRows; ++i) {
            const uint32_t hb = pack_word<kPrec, kCpl>(pb);  // (pr, pi) per channel
            const uint32_t off = p_base + i * 128 + ((lane_chunk ^ (i << 4)));
            *reinterpret_cast<uint32_t*>(stage + off) = hb ^ neg_im_mask<kPrec>();       // (pr, -pi)
            *reinterpret_cast<uint32_t*>(stage + kTileA + off) = swap_re_im<kPrec>(hb);  // (pi, pr)
            if (kHiLo) {
              // residual P - hi (the hi halves widened back to FP32)
              const float2 res = __ffma2_rn(make_float2(__uint_as_float(hb << 16),
                                                        __uint_as_float(hb & 0xFFFF0000u)),
                                            make_float2(-1.f, -1.f), pb[0]);
              const uint32_t lb = bf16x2_bits(__floats2bfloat162_rn(res.x, res.y));
              *reinterpret_cast<uint32_t*>(stage + 2 * kTileA + off) = lb ^ 0x80000000u;
              *reinterpret_cast<uint32_t*>(stage + 3 * kTileA + off) = __byte_perm(lb, 0, 0x1032);
            }
            // P <- P R as a paired multiply-add: (pr, pi) r1r + (-pi, pr) r1i
#pragma unroll
            for (int cl = 0; cl < kCpl; ++cl)
              pb[cl] = __ffma2_rn(make_float2(-pb[cl].y, pb[cl].x), make_float2(r1[cl].y, r1[cl].y),
                                  __fmul2_rn(pb[cl], make_float2(r1[cl].x, r1[cl].x)));
          }
          unsigned char* tb = stage + kBOff;
          if constexpr (kPrec == kF16) {
            // FP16: Z = X Q in paired half arithmetic, straight into the stored
            // format: xr (qr, qi) + xi (-qi, qr), Q converted once per a
            __half2 xr2[kBeamsPerWarp], xi2[kBeamsPerWarp];
#pragma unroll
            for (int m = 0; m < kBeamsPerWarp; ++m) {
              xr2[m] = __float2half2_rn(x[0][m].x);
              xi2[m] = __float2half2_rn(x[0][m].y);
            }
#pragma unroll
            for (int al = 0; al < kHalfA; ++al) {
              const __half2 qa2 = __floats2half2_rn(qa[0].x, qa[0].y);
              const __half2 qas = __floats2half2_rn(-qa[0].y, qa[0].x);
              const __half2 qb2 = __floats2half2_rn(qb[0].x, qb[0].y);
              const __half2 qbs = __floats2half2_rn(-qb[0].y, qb[0].x);
#pragma unroll
              for (int m = 0; m < kBeamsPerWarp; ++m) {
                // (a's this CTA does not hold, or without trials, are not read by its MMAs)
                if (keep(al)) {
                  const __half2 za = __hfma2(xr2[m], qa2, __hmul2(xi2[m], qas));
                  const uint32_t ra = static_cast<uint32_t>((kBeams / 8 * al + 2 * m) * 1024);
                  *reinterpret_cast<__half2*>(tb + z_base + ra) = za;
                }
                if (keep(al + kHalfA)) {
                  const __half2 zb = __hfma2(xr2[m], qb2, __hmul2(xi2[m], qbs));
                  const uint32_t rb =
                      static_cast<uint32_t>((kBeams / 8 * (al + kHalfA) + 2 * m) * 1024);
                  *reinterpret_cast<__half2*>(tb + z_base + rb) = zb;
                }
              }
              qa[0] = __ffma2_rn(make_float2(-qa[0].y, qa[0].x), make_float2(rT[0].y, rT[0].y),
                                 __fmul2_rn(qa[0], make_float2(rT[0].x, rT[0].x)));
              qb[0] = __ffma2_rn(make_float2(-qb[0].y, qb[0].x), make_float2(rT[0].y, rT[0].y),
                                 __fmul2_rn(qb[0], make_float2(rT[0].x, rT[0].x)));
            }
          } else {
#pragma unroll
          for (int al = 0; al < kHalfA; ++al) {
#pragma unroll
            for (int m = 0; m < kBeamsPerWarp; ++m) {
              // Z = X Q as (xr, xr)(qr, qi) + (-xi, xi)(qi, qr), for a = al and al + kHalfA
              float2 za[kCpl], zb[kCpl];
#pragma unroll
              for (int cl = 0; cl < kCpl; ++cl) {
                const float2 xv = x[cl][m];
                za[cl] = __ffma2_rn(make_float2(-xv.y, xv.y), make_float2(qa[cl].y, qa[cl].x),
                                    __fmul2_rn(make_float2(xv.x, xv.x), qa[cl]));
                zb[cl] = __ffma2_rn(make_float2(-xv.y, xv.y), make_float2(qb[cl].y, qb[cl].x),
                                    __fmul2_rn(make_float2(xv.x, xv.x), qb[cl]));
              }
              // row a_local * kBeams + pw + 16 m: z_base + (kBeams / 8 * a_local + 2 m) groups
              // (a's this CTA does not hold, or without trials, are not read by its MMAs)
              const uint32_t ra = static_cast<uint32_t>((kBeams / 8 * al + 2 * m) * 1024);
              const uint32_t rb = static_cast<uint32_t>((kBeams / 8 * (al + kHalfA) + 2 * m) * 1024);
              if (keep(al)) *reinterpret_cast<uint32_t*>(tb + z_base + ra) = pack_word<kPrec, kCpl>(za);
              if (keep(al + kHalfA))
                *reinterpret_cast<uint32_t*>(tb + z_base + rb) = pack_word<kPrec, kCpl>(zb);
            }
#pragma unroll
            for (int cl = 0; cl < kCpl; ++cl) {
              qa[cl] = __ffma2_rn(make_float2(-qa[cl].y, qa[cl].x), make_float2(rT[cl].y, rT[cl].y),
                                  __fmul2_rn(qa[cl], make_float2(rT[cl].x, rT[cl].x)));
              qb[cl] = __ffma2_rn(make_float2(-qb[cl].y, qb[cl].x), make_float2(rT[cl].y, rT[cl].y),
                                  __fmul2_rn(qb[cl], make_float2(rT[cl].x, rT[cl].x)));
            }
          }
          }
          // this thread's stores before the MMAs' reads (async proxy); the
          // arrive is local (a pair's second CTA forwards the stage)
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
  // a pair: the first CTA's MMAs have drained (its warp 0 waited above) and
  // no thread of either CTA arrives remotely any more
  if constexpr (kPair) cluster_sync();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if constexpr (kPair)
      asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                   "r"(kTmemCols));
    else
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                   "r"(kTmemCols));
  }
}

}  // namespace

size_t mac_tc_smem_bytes() { return kRingBytes + 1024 + 128; }

int mac_tc_beams_per_group(int n_series) { return n_series <= 16 ? 16 : 32; }

int mac_tc_trials_per_pass(int n_series, bool pair) {
  const bool g16 = mac_tc_beams_per_group(n_series) == 16;
  return pair ? (g16 ? dms_per_pass<16, true>() : dms_per_pass<32, true>())
              : (g16 ? dms_per_pass<16, false>() : dms_per_pass<32, false>());
}

int mac_tc_trials_per_a(bool pair) { return pair ? trials_per_a<true>() : trials_per_a<false>(); }

namespace {
template <int kPrec, int kBeams, bool kPair>
const void* tc_fn() {
  return reinterpret_cast<const void*>(&mac_tc_kernel<kPrec, kBeams, kPair>);
}
template <bool kPair>
const void* tc_fn(int prec, bool g16) {
  switch (prec) {
    case kBf16HiLo: return g16 ? tc_fn<kBf16HiLo, 16, kPair>() : tc_fn<kBf16HiLo, 32, kPair>();
    case kBf16: return g16 ? tc_fn<kBf16, 16, kPair>() : tc_fn<kBf16, 32, kPair>();
    case kF16: return g16 ? tc_fn<kF16, 16, kPair>() : tc_fn<kF16, 32, kPair>();
    default: return g16 ? tc_fn<kF8, 16, kPair>() : tc_fn<kF8, 32, kPair>();
  }
}
cudaLaunchConfig_t pair_config(int n_pairs, cudaLaunchAttribute* attr, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(2 * n_pairs);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = mac_tc_smem_bytes();
  cfg.stream = s;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cfg;
}
// Pairs resident at once per pair kernel (precision x group size), per device
constexpr int kMaxDevices = 64;
std::atomic<int> g_pairs[kMaxDevices][8];
}  // namespace

cudaError_t mac_tc_prepare() {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  for (int prec = 0; prec < 4; ++prec) {
    for (int g = 0; g < 2; ++g) {
      for (const void* fn : {tc_fn<false>(prec, g == 1), tc_fn<true>(prec, g == 1)}) {
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(mac_tc_smem_bytes()));
        if (e != cudaSuccess) return e;
      }
      if (dev < kMaxDevices) {
        cudaLaunchAttribute attr[1];
        const cudaLaunchConfig_t cfg = pair_config(1, attr, nullptr);
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, tc_fn<true>(prec, g == 1), &cfg) != cudaSuccess) {
          cudaGetLastError();
          n = 0;
        }
        g_pairs[dev][prec * 2 + g].store(n);
      }
    }
  }
  return cudaSuccess;
}

static cudaError_t launch_mac_tc_block(const MacArgs& a, int prec, int n_sms, cudaStream_t s);

namespace {
constexpr size_t kScratchAlign = 256;
constexpr size_t kScratchCap = size_t(3) << 30;
size_t align_up(size_t p) { return (p + kScratchAlign - 1) & ~(kScratchAlign - 1); }
// Scratch bytes per bin of a block: the bin-major spectra (when the caller's
// are bins innermost) and the bin-major output (when the caller's is).
size_t block_bytes_per_bin(bool x_in_place, bool y_in_place, int n_series, int n_chan, int n_dm,
                           size_t y_elem) {
  return (x_in_place ? 0 : sizeof(float2) * static_cast<size_t>(n_series) * n_chan) +
         (y_in_place ? 0 : y_elem * static_cast<size_t>(n_series) * n_dm);
}
int tc_prec(int precision) {
  return precision == FDD_PREC_BF16_HILO ? kBf16HiLo
         : precision == FDD_PREC_BF16    ? kBf16
         : precision == FDD_PREC_FP16    ? kF16
         : precision == FDD_PREC_FP8     ? kF8
                                         : -1;
}
}  // namespace

size_t mac_tc_scratch_bytes(int n_series, int n_chan, int n_dm, int64_t n_bins) {
  // the per-bin FP16 maxima of every bin, then blocks of both bin-major sides
  const size_t per_bin = block_bytes_per_bin(false, false, n_series, n_chan, n_dm, sizeof(float2));
  int64_t kb = static_cast<int64_t>(kScratchCap / per_bin);
  if (kb < 1) kb = 1;
  if (kb > n_bins) kb = n_bins;
  return align_up(sizeof(unsigned int) * static_cast<size_t>(n_bins)) +
         per_bin * static_cast<size_t>(kb) + 2 * kScratchAlign;
}

cudaError_t launch_mac_tc_direct(const MacArgs& a, int precision, int n_sms, cudaStream_t s) {
  if (a.n_dm <= 0 || a.n_series <= 0 || a.n_bins <= 0) return cudaSuccess;
  const int prec = tc_prec(precision);
  if (prec < 0 || a.x_bin_stride <= 0 || a.y_bin_stride <= 0 || a.x_chan_stride != 1)
    return cudaErrorInvalidValue;
  return launch_mac_tc_block(a, prec, n_sms, s);
}

size_t mac_tc_min_scratch(int n_series, int n_chan, int n_dm, int64_t n_bins) {
  return align_up(sizeof(unsigned int) * static_cast<size_t>(n_bins)) +
         block_bytes_per_bin(false, false, n_series, n_chan, n_dm, sizeof(float2)) +
         2 * kScratchAlign;
}

cudaError_t launch_mac_tc(const MacArgs& a, int precision, int n_sms, float2* scratch,
                          size_t scratch_bytes, cudaStream_t s) {
  if (a.n_dm <= 0 || a.n_series <= 0 || a.n_bins <= 0) return cudaSuccess;
  const int prec = tc_prec(precision);
  if (prec < 0 || !scratch) return cudaErrorInvalidValue;
  const bool x_in_place = a.x_bin_stride > 0;
  const bool y_in_place = a.y_bin_stride > 0;
  if (x_in_place && a.x_chan_stride != 1) return cudaErrorInvalidValue;
  if (!x_in_place && a.x_series_stride != a.x_chan_stride * a.n_chan) return cudaErrorInvalidValue;
  // scratch: [n_bins] per-bin maxima (FP16), then a block of bin-major
  // spectra and a block of bin-major output, as the caller's layouts need
  unsigned int* absmax = reinterpret_cast<unsigned int*>(scratch);
  const size_t head = align_up(sizeof(unsigned int) * static_cast<size_t>(a.n_bins));
  const size_t y_elem = a.out_kind == 2 ? sizeof(float) : sizeof(float2);
  cudaError_t e;
  if (x_in_place && y_in_place) {
    if ((prec == kF16 || prec == kF8) && !a.absmax_ready) {
      BinAbsmaxArgs t{a.X, a.x_bin_stride, a.n_series * a.n_chan, a.n_bins, absmax};
      if ((e = launch_bin_absmax(t, s)) != cudaSuccess) return e;
    }
    MacArgs b = a;
    b.bin_absmax = reinterpret_cast<const float*>(absmax);
    return launch_mac_tc_block(b, prec, n_sms, s);
  }
  const size_t per_bin =
      block_bytes_per_bin(x_in_place, y_in_place, a.n_series, a.n_chan, a.n_dm, y_elem);
  if (scratch_bytes < head + 2 * kScratchAlign) return cudaErrorInvalidValue;
  const int64_t kb = static_cast<int64_t>((scratch_bytes - head - 2 * kScratchAlign) / per_bin);
  if (kb < 1) return cudaErrorInvalidValue;
  char* blk = reinterpret_cast<char*>(scratch) + head;
  float2* x_scratch = reinterpret_cast<float2*>(blk);
  const size_t x_block = x_in_place ? 0 : sizeof(float2) * static_cast<size_t>(kb) * a.n_series *
                                              a.n_chan;
  void* y_scratch = blk + align_up(x_block);
  const int64_t rows = static_cast<int64_t>(a.n_series) * a.n_chan;
  const bool scaled = prec == kF16 || prec == kF8;
  if (scaled && x_in_place && !a.absmax_ready) {
    BinAbsmaxArgs t{a.X, a.x_bin_stride, a.n_series * a.n_chan, a.n_bins, absmax};
    if ((e = launch_bin_absmax(t, s)) != cudaSuccess) return e;
  }
  for (int64_t k0 = 0; k0 < a.n_bins; k0 += kb) {
    const int nb = static_cast<int>((a.n_bins - k0) < kb ? (a.n_bins - k0) : kb);
    MacArgs c = a;
    c.n_bins = nb;
    c.k_begin = a.k_begin + static_cast<int>(k0);
    c.bin_absmax = reinterpret_cast<const float*>(absmax + k0);
    if (x_in_place) {
      c.X = a.X + k0 * a.x_bin_stride;
    } else {
      if (scaled) {
        e = cudaMemsetAsync(absmax + k0, 0, sizeof(unsigned int) * static_cast<size_t>(nb), s);
        if (e != cudaSuccess) return e;
      }
      BinTransposeArgs t{a.X, a.x_chan_stride, rows, k0, nb, x_scratch,
                         scaled ? absmax + k0 : nullptr};
      if ((e = launch_bin_transpose(t, s)) != cudaSuccess) return e;
      c.X = x_scratch;
      c.x_bin_stride = rows;
      c.x_series_stride = a.n_chan;
      c.x_chan_stride = 1;
    }
    if (y_in_place) {
      c.Y = static_cast<char*>(a.Y) + y_elem * static_cast<size_t>(k0 * a.y_bin_stride);
    } else {
      c.Y = y_scratch;
      c.y_bin_stride = static_cast<int64_t>(a.n_series) * a.n_dm;
      c.y_series_stride = a.n_dm;
      c.y_dm_stride = 1;
    }
    if ((e = launch_mac_tc_block(c, prec, n_sms, s)) != cudaSuccess) return e;
    if (!y_in_place) {
      BinUntransposeArgs u{y_scratch, static_cast<int>(y_elem), a.n_series, a.n_dm, nb,
                           static_cast<char*>(a.Y) + y_elem * static_cast<size_t>(k0),
                           a.y_series_stride, a.y_dm_stride};
      if ((e = launch_bin_untranspose(u, s)) != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

static cudaError_t launch_mac_tc_block(const MacArgs& a, int prec, int n_sms, cudaStream_t s) {
  MacArgs args = a;
  void* params[] = {&args};
  const bool g16 = mac_tc_beams_per_group(a.n_series) == 16;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  // the CTA-pair form where the plan chose it: persistent pairs, as many as
  // are resident at once, at most one per bin (none fit: the one-CTA form)
  int n_pairs = dev < kMaxDevices ? g_pairs[dev][prec * 2 + (g16 ? 1 : 0)].load() : 0;
  if (!a.tc_pair) n_pairs = 0;
  if (n_pairs > n_sms / 2) n_pairs = n_sms / 2;
  if (n_pairs > a.n_bins) n_pairs = a.n_bins;
  note_launches(1);
  if (n_pairs >= 1) {
    cudaLaunchAttribute attr[1];
    const cudaLaunchConfig_t cfg = pair_config(n_pairs, attr, s);
    return cudaLaunchKernelExC(&cfg, tc_fn<true>(prec, g16), params);
  }
  const int grid = a.n_bins < n_sms ? a.n_bins : n_sms;
  return cudaLaunchKernel(tc_fn<false>(prec, g16), dim3(grid), dim3(kThreads), params,
                          mac_tc_smem_bytes(), s);
}

}  // namespace fdd

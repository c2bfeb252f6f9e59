// Device helpers shared by the phase-rotate-and-sum kernels: exact
// fixed-point phases, unit phasors, and mbarriers with bounded waits.
#pragma once

#include <stdint.h>

namespace fdd {
namespace dev {

// Upper bound of any wait in these kernels (~2 s at 2 GHz); a wait that runs
// out reports a timeout instead of hanging the GPU.
constexpr long long kWaitCycles = 4000000000LL;

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

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

// Arrive (release semantics: this thread's earlier shared-memory accesses are
// ordered before the phase completes).
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}" ::"r"(
                   smem_u32(bar))
               : "memory");
}

// One arrive for the whole (converged) warp: __syncwarp orders every lane's
// earlier shared-memory accesses before lane 0's release arrive, so a barrier
// counts warps instead of threads (fewer same-address atomics per phase).
__device__ __forceinline__ void mbar_arrive_warp(uint64_t* bar) {
  __syncwarp();
  if ((threadIdx.x & 31) == 0) mbar_arrive(bar);
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

}  // namespace dev
}  // namespace fdd

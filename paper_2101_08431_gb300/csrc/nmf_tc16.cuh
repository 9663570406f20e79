// Helpers shared by the rank-16 tensor-core passes (nmf_tc16s.cuh,
// nmf_tc16r.cuh): the BF16 hi/lo split of FP32 values and the bounded waits
// on mbarriers (2 s of wall time, or until another role of the CTA has
// given up and raised the abort flag).
#pragma once

#include <cuda_bf16.h>

#include "nmf_nnls.cuh"
#include "nmf_sweep.cuh"
#include "nmf_tc.cuh"
#include "nmf_tc16.h"
#include "nmf_lane16.cuh"

namespace nmfgb {
namespace tc16 {

__device__ __forceinline__ uint16_t bf16_bits(float f) {
  return __bfloat16_as_ushort(__float2bfloat16_rn(f));
}
__device__ __forceinline__ float bf16_val(uint16_t u) { return __uint_as_float((uint32_t)u << 16); }
// two FP32 values rounded to nearest-even BF16 by one packed conversion:
// a in the low half of the word, b in the high half
__device__ __forceinline__ uint32_t bf16x2_bits(float a, float b) {
  uint32_t r;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(b), "f"(a));
  return r;
}
// hi/lo split of two FP32 values, packed two BF16 per word (a in the low
// halves): hi = bf16(v), lo = bf16(v - hi), the subtraction exact in FP32.
// Two packed conversions per pair: the scalar form's four conversions paced
// the GEMM kernels' converter warps.
__device__ __forceinline__ void split2(float a, float b, uint32_t& hi, uint32_t& lo) {
  hi = bf16x2_bits(a, b);
  lo = bf16x2_bits(a - __uint_as_float(hi << 16), b - __uint_as_float(hi & 0xffff0000u));
}

constexpr unsigned long long WAIT_NS = 2000000000ull;   // bound of every wait: 2 s of wall time

__device__ __forceinline__ unsigned long long gtime() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ bool flag_set(int* flag) { return *reinterpret_cast<volatile int*>(flag) != 0; }
// Bounded waits: false after WAIT_NS (limit_ns), or as soon as another role of
// the CTA has given up (which it announces through *abort_flag).
template <bool CLUSTER>
__device__ __forceinline__ bool bwait_flag(int* abort_flag, uint64_t* bar, uint32_t parity,
                                           unsigned long long limit_ns = WAIT_NS) {
  const unsigned long long t0 = gtime();
  for (unsigned i = 0;; ++i) {
    if (CLUSTER ? mbar_try_wait_cluster(bar, parity) : mbar_try_wait(bar, parity)) return true;
    if ((i & 63) == 63) {
      if (flag_set(abort_flag)) return false;
      if (gtime() - t0 > limit_ns) break;
    }
  }
  atomicExch(abort_flag, 1);
  return false;
}
}  // namespace tc16
}  // namespace nmfgb

// Accumulation policies of the M pass (B = X^T M_tile and P += M_tile Y^T).
//
//   ArF32 : FP32 operands, FP32 FMA accumulation (bulk sweeps of the mixed form)
//   ArF64 : FP64 operands and accumulation (the FP64 form, and the plain
//           FP64-accumulated refinement of FP32 M)
//   ArInc : incremental contraction for the refinement sweeps of the mixed
//           form: FP32 operands and FP32 accumulation like ArF32, but of the
//           change of X (and of Y) since the last compensated sweep, whose
//           contractions are added back in FP64 (Problem::Bref, Pref)
//   ArDF  : compensated FP32 ("double-float") accumulation of FP32 M times
//           FP64 factors, for the refinement sweeps of the mixed form.  A
//           factor value x is carried as hi + lo with hi = fl32(x),
//           lo = fl32(x - hi); each term m * hi is formed exactly as p + e
//           (p = fl(m hi), e = fma(m, hi, -p)), p is added to the running
//           high word with Knuth's TwoSum (the rounding error is recovered
//           exactly), and e, m * lo and the recovered errors go to the low
//           word.  About 11 FP32 instructions per term instead of one FP64
//           FMA, on a part whose FP32 rate is ~60x its FP64 rate; the sums
//           carry ~44 significant bits.
//
// Every policy provides: V (staged factor value), A (accumulator), P (type
// of the stored P partials), R (type of the cross-warp and cross-CTA sums of
// B: FP32 instructions only where the pass itself avoids FP64), load_x /
// yval (staging of X from its stored copies, of y from FP64), zero, vzero,
// madd, add, shfl_xor, to_double, to_p, to_r, radd, rshfl_xor, r_to_double,
// EPS (the epsilon of the NNLS entering tolerance for sweeps computed with
// this policy), INC (the incremental form) and REFINE (one step of iterative
// refinement in the table-driven column solves).
#pragma once

#include "nmf_common.cuh"

namespace nmfgb {

struct alignas(8) DF {
  float hi, lo;
};

// Double-float addition (Knuth's TwoSum of the high words, then the low
// words, renormalised): the cross-warp and cross-CTA reduction type of the
// FP32 and compensated passes (FP32 instructions only).
__device__ __forceinline__ float df_two_sum(float a, float b, float& err) {
  const float s = __fadd_rn(a, b);
  const float bb = __fadd_rn(s, -a);
  err = __fadd_rn(__fadd_rn(a, -__fadd_rn(s, -bb)), __fadd_rn(b, -bb));
  return s;
}
__device__ __forceinline__ DF df_add(DF a, DF b) {
  float err;
  const float s = df_two_sum(a.hi, b.hi, err);
  const float lo = __fadd_rn(__fadd_rn(a.lo, b.lo), err);
  const float h = __fadd_rn(s, lo);
  return {h, __fadd_rn(lo, -__fadd_rn(h, -s))};
}
__device__ __forceinline__ DF df_shfl_xor(DF a, int o) {
  return {__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o)};
}

// Arithmetic on the stored partials of P = M Y^T (the row pass sums the
// cluster partials in their own type and converts once).
template <typename T>
struct PartOps;
template <>
struct PartOps<float> {
  __device__ static float zero() { return 0.f; }
  __device__ static float add(float a, float b) { return a + b; }
  __device__ static double to_double(float a) { return (double)a; }
};
template <>
struct PartOps<double> {
  __device__ static double zero() { return 0.0; }
  __device__ static double add(double a, double b) { return a + b; }
  __device__ static double to_double(double a) { return a; }
};
template <>
struct PartOps<DF> {
  __device__ static DF zero() { return {0.f, 0.f}; }
  __device__ static DF add(DF a, DF b) { return df_add(a, b); }
  __device__ static double to_double(DF a) { return (double)a.hi + (double)a.lo; }
};

struct ArF32 {
  using V = float;
  using A = float;
  using P = float;
  static constexpr bool XD = false;   // X is staged from its FP32 copy
  static constexpr bool INC = false;
  static constexpr bool REFINE = false;   // B is FP32-accurate: no refinement step in the solves
  static constexpr bool PACC_SMEM = false;   // P accumulators in registers
  // the FP64 column solves take the FP64 entering tolerance: a coarser one
  // leaves out variables whose small gradient hides a large value where G is
  // ill conditioned
  static constexpr double EPS = 2.220446049250313e-16;
  using R = DF;   // cross-warp / cross-CTA reduction of B
  __device__ static V load_x(const Problem& p, int b, size_t i) { return p.X32[b][i]; }
  __device__ static V vzero() { return 0.f; }
  __device__ static R to_r(A a) { return {a, 0.f}; }
  __device__ static R radd(R a, R b) { return df_add(a, b); }
  __device__ static R rshfl_xor(R a, int o) { return df_shfl_xor(a, o); }
  __device__ static double r_to_double(R a) { return (double)a.hi + (double)a.lo; }
  __device__ static V yval(double y) { return (float)y; }
  __device__ static A zero() { return 0.f; }
  template <typename TM>
  __device__ static A madd(TM m, V v, A a) { return __fmaf_rn((float)m, v, a); }
  __device__ static A add(A a, A b) { return __fadd_rn(a, b); }
  __device__ static A shfl_xor(A a, int o) { return __shfl_xor_sync(0xffffffffu, a, o); }
  __device__ static double to_double(A a) { return (double)a; }
  __device__ static P to_p(A a) { return a; }
};

struct ArF64 {
  using V = double;
  using A = double;
  using P = double;
  static constexpr bool XD = true;
  static constexpr bool INC = false;
  static constexpr bool REFINE = true;    // one refinement step of the table solve
  static constexpr bool PACC_SMEM = false;
  static constexpr double EPS = 2.220446049250313e-16;
  using R = double;
  __device__ static V load_x(const Problem& p, int b, size_t i) { return p.X[b][i]; }
  __device__ static V vzero() { return 0.0; }
  __device__ static R to_r(A a) { return a; }
  __device__ static R radd(R a, R b) { return __dadd_rn(a, b); }
  __device__ static R rshfl_xor(R a, int o) { return __shfl_xor_sync(0xffffffffu, a, o); }
  __device__ static double r_to_double(R a) { return a; }
  __device__ static V yval(double y) { return y; }
  __device__ static A zero() { return 0.0; }
  template <typename TM>
  __device__ static A madd(TM m, V v, A a) { return __fma_rn((double)m, v, a); }
  __device__ static A add(A a, A b) { return __dadd_rn(a, b); }
  __device__ static A shfl_xor(A a, int o) { return __shfl_xor_sync(0xffffffffu, a, o); }
  __device__ static double to_double(A a) { return a; }
  __device__ static P to_p(A a) { return a; }
};

struct ArDF {
  using V = DF;
  using A = DF;
  using P = DF;   // partials stay double-float: no FP64 instruction in the epilogue
  static constexpr bool XD = true;
  static constexpr bool INC = false;
  static constexpr bool REFINE = true;
  static constexpr double EPS = 5.684341886080802e-14;   // 2^-44
  // the P accumulators (two words each) live in shared memory, so that a
  // CTA holds as many rows as in the FP32 pass (no cluster exchange)
  static constexpr bool PACC_SMEM = true;
  __device__ static V split(double x) {
    const float hi = __double2float_rn(x);
    return {hi, __double2float_rn(x - (double)hi)};
  }
  using R = DF;
  // the split of X is formed by the row pass that produced it (X32, X32lo)
  __device__ static V load_x(const Problem& p, int b, size_t i) { return {p.X32[b][i], p.X32lo[b][i]}; }
  __device__ static V vzero() { return {0.f, 0.f}; }
  __device__ static R to_r(A a) { return a; }
  __device__ static R radd(R a, R b) { return df_add(a, b); }
  __device__ static R rshfl_xor(R a, int o) { return df_shfl_xor(a, o); }
  __device__ static double r_to_double(R a) { return (double)a.hi + (double)a.lo; }
  __device__ static V yval(double y) { return split(y); }
  __device__ static A zero() { return {0.f, 0.f}; }
  // Knuth's TwoSum: s + err == a + b exactly.
  __device__ static float two_sum(float a, float b, float& err) { return df_two_sum(a, b, err); }
  __device__ static A madd(float m, V v, A a) {
    const float p = __fmul_rn(m, v.hi);
    const float e = __fmaf_rn(m, v.hi, -p);            // m * v.hi == p + e exactly
    float err;
    const float s = two_sum(a.hi, p, err);
    return {s, __fadd_rn(a.lo, __fadd_rn(err, __fmaf_rn(m, v.lo, e)))};
  }
  __device__ static A add(A a, A b) { return df_add(a, b); }
  __device__ static A shfl_xor(A a, int o) { return df_shfl_xor(a, o); }
  __device__ static double to_double(A a) { return (double)a.hi + (double)a.lo; }
  __device__ static P to_p(A a) { return a; }
};

struct ArInc {
  using V = float;
  using A = float;
  using P = float;     // partials of M (Y - Yref)^T
  // FP64-class solves (one refinement step): B and P are FP64-accurate
  static constexpr bool XD = true;
  static constexpr bool INC = true;
  // the FP64 table solve's own error (~2^-53 cond) is far below that of B
  // (~2^-44 cond): no refinement step
  static constexpr bool REFINE = false;
  static constexpr bool PACC_SMEM = false;
  static constexpr double EPS = 5.684341886080802e-14;   // 2^-44, as the compensated pass
  using R = DF;
  // the row pass that produced X wrote fl32(X - Xref)
  __device__ static V load_x(const Problem& p, int b, size_t i) { return p.Xd32[b][i]; }
  __device__ static V vzero() { return 0.f; }
  __device__ static R to_r(A a) { return {a, 0.f}; }
  __device__ static R radd(R a, R b) { return df_add(a, b); }
  __device__ static R rshfl_xor(R a, int o) { return df_shfl_xor(a, o); }
  __device__ static double r_to_double(R a) { return (double)a.hi + (double)a.lo; }
  __device__ static V yval(double dy) { return (float)dy; }   // called with y - yref
  __device__ static A zero() { return 0.f; }
  template <typename TM>
  __device__ static A madd(TM m, V v, A a) { return __fmaf_rn((float)m, v, a); }
  __device__ static A add(A a, A b) { return __fadd_rn(a, b); }
  __device__ static A shfl_xor(A a, int o) { return __shfl_xor_sync(0xffffffffu, a, o); }
  __device__ static double to_double(A a) { return (double)a; }
  __device__ static P to_p(A a) { return a; }
};

// Reduce-scatter of VP = 2^p <= 32 accumulators held by every lane: lane l
// ends with the warp-wide sum of accumulator (l & (VP-1)), in fixed order.
template <typename AR, int VP>
__device__ __forceinline__ typename AR::A warp_reduce_scatter_ar(typename AR::A (&v)[VP]) {
  static_assert(VP >= 1 && VP <= 32 && (VP & (VP - 1)) == 0, "VP must be a power of two <= 32");
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = VP / 2; o >= 1; o >>= 1) {
    const bool upper = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < o; ++i) {
      const typename AR::A keep = upper ? v[i + o] : v[i];
      const typename AR::A send = upper ? v[i] : v[i + o];
      v[i] = AR::add(keep, AR::shfl_xor(send, o));
    }
  }
  typename AR::A r = v[0];
#pragma unroll
  for (int o = VP; o < 32; o <<= 1) r = AR::add(r, AR::shfl_xor(r, o));
  return r;
}

}  // namespace nmfgb

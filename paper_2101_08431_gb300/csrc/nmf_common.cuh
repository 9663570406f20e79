// Shared device-side definitions of the GB300 streaming-NMF library:
// device state, launch descriptors, PTX wrappers (mbarrier, bulk async copy)
// and fixed-order reductions.  Everything here is part of the CUDA path; the
// CPU oracle has its own, separate implementation of the method.
#pragma once

#include <type_traits>

#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace nmfgb {

namespace cg = cooperative_groups;

constexpr int KMAX = 16;           // largest rank the kernels are built for
constexpr int STAT_CAP = 64;       // per-iterate statistics ring
constexpr int NSTAT = 16;          // doubles per statistics record
constexpr int NYT = 11;            // KKT / objective terms of the Y half (per cluster)
constexpr int NXT = 10;            // terms of the X half (per row block)
constexpr int CACHE_N = 8;         // inverse-cache entries per CTA
constexpr long long SPIN_LIMIT = 1ll << 26;   // bounded waits (about a second)

// error bits in DevState::err
constexpr unsigned ERR_TIMEOUT = 1u;
constexpr unsigned ERR_NONFINITE = 2u;
constexpr unsigned ERR_CONFIG = 4u;

// Y-half terms, for the iterate (X_t, Y_t) entering a sweep:
//   graY_j = G y_j - b_j with b_j = X_t^T M_{:,j} and G = X_t^T X_t
enum YTerm { YT_NEG = 0, YT_COMP, YT_BNORM2, YT_BY, YT_YGY, YT_YMAX, YT_YNORM2, YT_DY2,
             YT_CHANGED, YT_NOTCONV, YT_ENTER };
// X-half terms, for the iterate (X_{t+1}, Y_{t+1}) leaving a sweep:
//   graX_i = H x_i - P_i with H = Y Y^T and P = M Y^T
enum XTerm { XT_NEG = 0, XT_COMP, XT_PNORM2, XT_XMAX, XT_XNORM2, XT_DX2, XT_XP,
             XT_CHANGED, XT_NOTCONV, XT_VALID };
// statistics record of iterate t
enum Stat { ST_ITER = 0, ST_F, ST_EABS, ST_REL, ST_STEP, ST_NEG, ST_COMP, ST_SG, ST_XYMAX,
            ST_CHANGED_COLS, ST_CHANGED_ROWS, ST_NOTCONV, ST_FP64, ST_MSQ, ST_VALID, ST_ENTER };

// Device-resident control block of one problem.
struct DevState {
  int iter;          // index t of the current iterate (buffers t & 1)
  int done;          // set by the finalize when a stopping test holds
  unsigned err;      // ERR_* bits
  unsigned xblocks_done;   // last-block counter of the X kernel
  int stop_reason;   // 1 = rel-KKT target, 2 = step tolerance
  int pass_var;      // device-driven mixed schedule: variant of the next sweep's passes
  int since_best;    // sweeps since the best FP32-pass relative KKT improved by 2%
  int fp64_sweeps;   // sweeps whose tail ran with an FP64-class M pass (counts up)
  int gtab_valid;    // the subset table of G in global memory belongs to the current G
  double stats[STAT_CAP][NSTAT];
  double xiter[2][NXT];     // X-half terms of the iterate held in buffers 0 / 1
  double msq;               // ||M||_F^2 of the resident window
  double best_rel;          // device-driven mixed schedule: best FP32-pass relative KKT (<= 0: none)
};

// Arithmetic of one M pass.
enum Variant {
  VAR_F32 = 0,   // FP32 M, FP32 contraction (mixed precision, bulk sweeps)
  VAR_REF = 1,   // FP32 M, FP64 contraction (mixed precision, refinement sweeps)
  VAR_F64 = 2,   // FP64 M, FP64 contraction (the plain FP64 form)
  VAR_DF = 3,    // FP32 M, compensated FP32 contraction (mixed precision, refinement sweeps)
  VAR_INC = 4,   // FP32 M, incremental contraction: references from the last compensated
                 // sweep plus the FP32 contraction of the change of X and Y since it
  NVAR = 5
};

// One problem as the kernels see it.
struct Problem {
  int n, m, k;            // rows, resident columns, rank
  int ld;                 // leading dimension of M (elements, multiple of 32)
  int mcap;               // ring capacity (columns)
  int head;               // physical column of logical column 0
  const void* M;          // ld x mcap, column-major, float or double
  double* X[2];           // n x k row-major, FP64
  float* X32[2];          // FP32 copy of X
  float* X32lo[2];        // fl32(x - fl32(x)): low word of X for the compensated pass
  double* Y[2];           // k x mcap column-major (physical column order), FP64
  uint32_t* ymask[2];     // passive set of each column
  uint32_t* xmask[2];     // passive set of each row
  double* G;              // k x k, X^T X of the current iterate
  double* Gtab;           // k <= 8: inv(G_PP) for every passive set P (2^k x k x k)
  int* Gok;               // k <= 8: 1 where the table entry is valid
  double* Hg;             // k <= 8, tab_global: H = Y Y^T of this sweep (k x k)
  double* Htab;           // k <= 8, tab_global: its subset table (2^k x k x k)
  int* Hok;
  int tab_global;         // 1: the tables of G and H are built once per sweep into global
                          // memory (G by the row pass's tail, H by the batch's H stage)
  int gtab_tail;          // 1: the table of G alone is built by the row pass's tail
  const double* colsq;    // ||M_{:,j}||^2 per physical column
  void* Ppart;            // [Q][ld][k] partial M Y^T (accumulate type)
  double* Hpart;          // [Q][k][k]
  double* Yterms;         // [Q][NYT]
  double* Xpart;          // [nxblk][k*k + NXT], for k = 16 then [ceil(nxblk / XGROUP)] group partials
  unsigned* xgt;          // k = 16: group tickets of the row pass's block sums (self-resetting);
                          // nullptr: the last block sums every block
  DevState* st;
  double kkt_target;      // <= 0 disables
  double kkt_abs_target;  // <= 0 disables
  double stol;            // <= 0 disables
  int warm;               // 0 cold, 1 previous sweep (new columns are seeded at append),
                          // 2 chain: column j from column j - 1's new solution
  int fp64_pass;          // 1 when this sweep's M pass runs in FP64
  // device-driven mixed schedule (batched form): FP32 passes until the
  // relative KKT reaches mixed_switch or has not improved by 2% for
  // stall_sweeps sweeps, then compensated passes (DevState::pass_var)
  int auto_mixed;
  int stall_sweeps;
  double mixed_switch;
  // incremental contractions (VAR_INC) of the mixed form.  A compensated sweep
  // with record_refs = 1 stores its exact-to-~44-bit contractions as
  // references: Bref_j = X_t^T M_{:,j} with Xref = X_t, and Pref = M Y_{t+1}^T
  // with Yref = Y_{t+1}.  An incremental sweep (inc = 1) forms
  // B_j = Bref_j + (X - Xref)^T M_{:,j} and P = Pref + M (Y - Yref)^T, the
  // change terms contracted in FP32: their rounding is 2^-24 of the change,
  // not of the contraction.  Every row pass of either kind writes
  // Xd32 = fl32(X_{t+1} - Xref) for the next incremental sweep.
  double* Bref;           // k x mcap (physical column order)
  double* Yref;           // k x mcap (physical column order)
  double* Pref;           // n x k row-major
  double* Xref;           // n x k row-major
  float* Xd32[2];         // n x k row-major, by iterate parity
  int inc;                // 1: this sweep is incremental
  int record_refs;        // 1: this (compensated) sweep records the references
};

enum Mode { MODE_SWEEP = 0, MODE_PRIME = 1, MODE_KKT = 2 };

constexpr int XGROUP = 16;   // row-pass blocks per group partial (Problem::xgt)

// ---------------------------------------------------------------------------
// PTX wrappers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}

// Release store / acquire load of a 32-bit flag at GPU scope.
__device__ __forceinline__ void st_release_u32(unsigned* a, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(a), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* a) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(a) : "memory");
  return v;
}

__device__ __forceinline__ void mbar_inval(uint64_t* bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Arrive (release, cluster scope) on the mbarrier at the same offset in the
// shared memory of cluster rank `rank`.
__device__ __forceinline__ void mbar_arrive_remote(uint64_t* bar, uint32_t rank) {
  uint32_t raddr;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(raddr) : "r"(smem_u32(bar)), "r"(rank));
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(raddr) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait_cluster(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ bool mbar_wait_cluster(uint64_t* bar, uint32_t parity) {
  for (long long i = 0; i < SPIN_LIMIT; ++i)
    if (mbar_try_wait_cluster(bar, parity)) return true;
  return false;
}

// Named barrier over the first `count` threads of the block (id != 0).
__device__ __forceinline__ void named_sync(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait on an mbarrier phase; false after SPIN_LIMIT polls.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  for (long long i = 0; i < SPIN_LIMIT; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// 1-D bulk asynchronous copy global -> shared (the TMA engine), completion
// counted in bytes on the mbarrier.  dst, src 16-byte aligned, bytes % 16 == 0.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// FP64 compares, min and max are several times slower than FP64 FMAs on
// this part; for finite values the sign and order tests below run on the
// IEEE bit patterns with integer instructions instead.
__device__ __forceinline__ long long dbits(double x) { return __double_as_longlong(x); }
__device__ __forceinline__ bool dpos(double x) { return dbits(x) > 0; }            // x > 0
__device__ __forceinline__ bool dneg(double x) { return dbits(x) < 0 && x != 0.0; } // x < 0
// max of two non-negative values
__device__ __forceinline__ double dmax_nn(double a, double b) { return dbits(a) >= dbits(b) ? a : b; }
// w > t for t >= 0 (any w)
__device__ __forceinline__ bool dgt_nn(double w, double t) { return dbits(w) > dbits(t); }
// min(g, 0) and max(g, 0)
__device__ __forceinline__ double dminz(double g) { return dbits(g) < 0 ? g : 0.0; }
__device__ __forceinline__ double dmaxz(double g) { return dbits(g) > 0 ? g : 0.0; }
__device__ __forceinline__ double dabs(double x) { return __longlong_as_double(dbits(x) & 0x7fffffffffffffffll); }

// Fused multiply-add in the precision of the operands (no implicit promotion).
__device__ __forceinline__ float fmad(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fmad(double a, double b, double c) { return __fma_rn(a, b, c); }

// ---------------------------------------------------------------------------
// Warp reductions (fixed lane order => deterministic)
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
template <typename T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Reduce-scatter of V = 2^p <= 32 values held by every lane: afterwards lane l
// holds the warp-wide sum of value (l & (V-1)).  V-1 + 5-p shuffles.
template <int V, typename T>
__device__ __forceinline__ T warp_reduce_scatter(T (&v)[V]) {
  static_assert(V >= 1 && V <= 32 && (V & (V - 1)) == 0, "V must be a power of two <= 32");
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = V / 2; o >= 1; o >>= 1) {
    const bool upper = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < o; ++i) {
      T keep = upper ? v[i + o] : v[i];
      T send = upper ? v[i] : v[i + o];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
  T r = v[0];
#pragma unroll
  for (int o = V; o < 32; o <<= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
  return r;
}

__device__ __forceinline__ int pow2ceil_int(int v) {
  int p = 1;
  while (p < v) p <<= 1;
  return p;
}

__device__ __forceinline__ void set_err(DevState* st, unsigned bits) { atomicOr(&st->err, bits); }

}  // namespace nmfgb

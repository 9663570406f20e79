// Warm-started Lawson-Hanson NNLS for one k-variable subproblem per thread
// (problem "qp" of Sec. 2: min 1/2 y'Gy - b'y, y >= 0, with G = X^T X for a
// column of Y or G = Y Y^T for a row of X).
//
// GB300 design notes.  FP64 on this part is slow (about 1/60 of FP32, a
// dependent FMA takes tens of ns and a divide hundreds), so the solver never
// refactors G from scratch per column.  It keeps A = inv(G_PP) for the
// current passive set P and changes it by one-rank bordering / downdating
// when a variable enters or leaves (one reciprocal and O(k^2) FMAs each) --
// the paper's remark that the factorization of the previous solve can be
// reused (Sec. 2).  A per-CTA cache holds inv(G_PP) for the passive sets of
// sampled neighbouring columns, so that a column whose passive set did not
// change costs two k x k mat-vecs: z = A b and w = b - G z.
//
// Decisions shared with the oracle (same readings, separate code):
//   entering test w_i > tol, tol = 10 k eps (max|b| + max_i G_ii max|y|),
//   lowest index first on ties, Schur pivot <= 1e-14 max_i G_ii blocks the
//   variable, an entering variable whose first value is <= 0 is blocked,
//   at most 5k + 10 outer iterations.
#pragma once

#include "nmf_common.cuh"

namespace nmfgb {

// 1/x in FP64 by Newton-Raphson refinement r <- r (2 - x r) of an FP32
// reciprocal seed: the error squares each step (2^-23 -> 2^-46 -> rounding),
// two FMAs per step instead of the long FP64 divide.  Arguments outside the
// FP32 normal range fall back to the division.
__device__ __forceinline__ double rcp64(double x) {
  const long long ab = dbits(x) & 0x7fffffffffffffffll;   // |x| as an ordered integer
  if (!(ab > 0x39b4484bfeebc2a0ll && ab < 0x4629c4ab5c06e0d3ll)) return 1.0 / x;   // 1e-30 .. 1e30
  double r = (double)__frcp_rn((float)x);
  double e = __fma_rn(-x, r, 1.0);
  r = __fma_rn(r, e, r);
  e = __fma_rn(-x, r, 1.0);
  return __fma_rn(r, e, r);
}

// sum_c [c in P] a[c] * b[c] as a pairwise tree (dependency depth 1 + log2 K)
template <int K>
__device__ __forceinline__ double dot_masked(const double* a, const double (&b)[K], uint32_t P) {
  double t[K];
#pragma unroll
  for (int c = 0; c < K; ++c) t[c] = ((P >> c) & 1u) ? a[c] * b[c] : 0.0;
#pragma unroll
  for (int w = 1; w < K; w <<= 1)
#pragma unroll
    for (int c = 0; c + w < K; c += 2 * w) t[c] += t[c + w];
  return t[0];
}

// Arithmetic of the lane-parallel solver in its value type: FP64 for the
// FP64-class passes; FP32 for the FP32 pass, whose right-hand sides are
// FP32-accurate (IEEE-ordered bit patterns for sign and order tests, the
// correctly rounded FP32 reciprocal).
template <typename V>
struct VOps;
template <>
struct VOps<double> {
  __device__ static long long bits(double x) { return __double_as_longlong(x); }
  __device__ static double rcp(double x) { return rcp64(x); }
  __device__ static double absv(double x) { return dabs(x); }
};
template <>
struct VOps<float> {
  __device__ static int bits(float x) { return __float_as_int(x); }
  __device__ static float rcp(float x) { return __frcp_rn(x); }
  __device__ static float absv(float x) { return fabsf(x); }
};
template <typename V>
__device__ __forceinline__ bool vpos(V x) { return VOps<V>::bits(x) > 0; }   // x > 0
template <typename V>
__device__ __forceinline__ V vmax_nn(V a, V b) { return VOps<V>::bits(a) >= VOps<V>::bits(b) ? a : b; }

template <int K, typename V>
__device__ __forceinline__ V dot_masked_v(const V* a, const V (&b)[K], uint32_t P) {
  V t[K];
#pragma unroll
  for (int c = 0; c < K; ++c) t[c] = ((P >> c) & 1u) ? a[c] * b[c] : V(0);
#pragma unroll
  for (int w = 1; w < K; w <<= 1)
#pragma unroll
    for (int c = 0; c + w < K; c += 2 * w) t[c] += t[c + w];
  return t[0];
}

template <int K>
struct InvCache {
  int n;
  uint32_t mask[CACHE_N];
  double inv[CACHE_N][K * K];
};

template <int K>
struct NnlsSolver {
  const double* G;   // k x k row-major (shared memory)
  double gmax;
  double pivot_min;
  double eps;

  __device__ void init(const double* Gs, double eps_) {
    G = Gs;
    double g = 0.0;
#pragma unroll
    for (int a = 0; a < K; ++a) g = dmax_nn(g, dabs(Gs[a * K + a]));
    gmax = g;
    pivot_min = 1e-14 * g;
    eps = eps_;
  }

  // A = inv(G_PP) -> inv(G_{P+i}); false (A unchanged) if the Schur pivot is
  // not above pivot_min.
  __device__ bool add(double* A, uint32_t P, int i) const {
    double gi[K], u[K];
#pragma unroll
    for (int c = 0; c < K; ++c) gi[c] = G[c * K + i];
#pragma unroll
    for (int a = 0; a < K; ++a) u[a] = ((P >> a) & 1u) ? dot_masked<K>(A + a * K, gi, P) : 0.0;
    const double s = G[i * K + i] - dot_masked<K>(G + i * K, u, P);
    if (!(s > pivot_min)) return false;
    const double rs = rcp64(s);
#pragma unroll
    for (int a = 0; a < K; ++a) {
      if (!((P >> a) & 1u)) continue;
      const double ua = u[a] * rs;
#pragma unroll
      for (int c = 0; c < K; ++c)
        if ((P >> c) & 1u) A[a * K + c] = fmad(ua, u[c], A[a * K + c]);
      A[a * K + i] = -ua;
      A[i * K + a] = -ua;
    }
    A[i * K + i] = rs;
    return true;
  }

  // A = inv(G_PP) with i in P -> inv(G_{P-i}).
  __device__ void remove(double* A, uint32_t P, int i) const {
    const double rd = rcp64(A[i * K + i]);
    double ci[K];
#pragma unroll
    for (int a = 0; a < K; ++a) ci[a] = (((P >> a) & 1u) && a != i) ? A[a * K + i] : 0.0;
#pragma unroll
    for (int a = 0; a < K; ++a) {
      if (!((P >> a) & 1u) || a == i) continue;
      const double f = ci[a] * rd;
#pragma unroll
      for (int c = 0; c < K; ++c)
        if (((P >> c) & 1u) && c != i) A[a * K + c] = fmad(-f, ci[c], A[a * K + c]);
    }
  }

  // inv(G_PP) from scratch, variables added in ascending order; variables
  // whose pivot fails are dropped from the returned mask and set in *blocked.
  __device__ uint32_t build(double* A, uint32_t P, uint32_t* blocked) const {
    uint32_t Q = 0;
#pragma unroll 1
    for (int i = 0; i < K; ++i) {
      if (!((P >> i) & 1u)) continue;
      if (add(A, Q, i)) Q |= 1u << i;
      else if (blocked) *blocked |= 1u << i;
    }
    return Q;
  }

  __device__ void apply(const double* A, uint32_t P, const double (&b)[K], double (&z)[K]) const {
#pragma unroll
    for (int a = 0; a < K; ++a) z[a] = ((P >> a) & 1u) ? dot_masked<K>(A + a * K, b, P) : 0.0;
  }

  // w = b - G y, returns the entering index (or -1) for the outer loop.
  __device__ int entering(const double (&b)[K], const double (&y)[K], uint32_t P, uint32_t blocked,
                          double bmax) const {
    double ymax = 0.0;
#pragma unroll
    for (int a = 0; a < K; ++a) ymax = fmax(ymax, y[a]);
    const double tol = 10.0 * K * eps * (bmax + gmax * ymax);
    int t = -1;
    double best = tol;
#pragma unroll
    for (int a = 0; a < K; ++a) {
      const double w = b[a] - dot_masked<K>(G + a * K, y, 0xffffffffu);
      const bool cand = !(((P | blocked) >> a) & 1u);
      if (cand && w > best) {
        best = w;
        t = a;
      }
    }
    return t;
  }

  // Inner loop of Lawson-Hanson from the feasible y (y_P > 0).  t_in is the
  // variable that just entered (or -1 on a warm start).
  __device__ void inner(double* A, const double (&b)[K], double (&y)[K], uint32_t& P,
                        uint32_t& blocked, int t_in) const {
    bool first = true;
#pragma unroll 1
    for (int it = 0; it <= K + 1; ++it) {
      if (!P) {
#pragma unroll
        for (int a = 0; a < K; ++a) y[a] = 0.0;
        return;
      }
      double z[K];
      apply(A, P, b, z);
      if (first && t_in >= 0) {
        double zt = 0.0;
#pragma unroll
        for (int a = 0; a < K; ++a)
          if (a == t_in) zt = z[a];
        if (!(zt > 0.0)) {
          remove(A, P, t_in);
          P &= ~(1u << t_in);
          blocked |= 1u << t_in;
          return;
        }
      }
      first = false;
      bool feasible = true;
#pragma unroll
      for (int a = 0; a < K; ++a)
        if (((P >> a) & 1u) && !(z[a] > 0.0)) feasible = false;
      if (feasible) {
#pragma unroll
        for (int a = 0; a < K; ++a) y[a] = ((P >> a) & 1u) ? z[a] : 0.0;
        return;
      }
      double alpha = 2.0;
      int q = -1;
#pragma unroll
      for (int a = 0; a < K; ++a) {
        if (!((P >> a) & 1u) || z[a] > 0.0) continue;
        const double r = y[a] * rcp64(y[a] - z[a]);
        if (r < alpha) {
          alpha = r;
          q = a;
        }
      }
      if (q < 0) {   // only reachable through NaN: take the first infeasible one
        alpha = 0.0;
#pragma unroll
        for (int a = K - 1; a >= 0; --a)
          if (((P >> a) & 1u) && !(z[a] > 0.0)) q = a;
      }
#pragma unroll
      for (int a = 0; a < K; ++a)
        if ((P >> a) & 1u) y[a] = fmad(alpha, z[a] - y[a], y[a]);
      // drop q and every passive variable that reached zero
      uint32_t drop = 1u << q;
#pragma unroll
      for (int a = 0; a < K; ++a)
        if (((P >> a) & 1u) && !(y[a] > 0.0)) drop |= 1u << a;
#pragma unroll 1
      for (int a = 0; a < K; ++a) {
        if (!((drop >> a) & 1u)) continue;
        remove(A, P, a);
        P &= ~(1u << a);
      }
#pragma unroll
      for (int a = 0; a < K; ++a)
        if ((drop >> a) & 1u) y[a] = 0.0;
    }
  }

  // Full solve.  y holds the warm start on entry (>= 0; ignored when cold)
  // and the solution on exit; A is per-thread scratch of K*K doubles.
  // Returns 0 when converged, 1 at the iteration cap.  *mask_out gets the
  // support of y.
  __device__ __noinline__ int solve(double* A, const double (&b)[K], double (&y)[K], bool warm,
                                    const InvCache<K>* cache, uint32_t* mask_out) const {
    uint32_t P = 0, blocked = 0;
    double bmax = 0.0;
#pragma unroll
    for (int a = 0; a < K; ++a) {
      bmax = fmax(bmax, fabs(b[a]));
      if (warm && y[a] > 0.0) P |= 1u << a;
      else y[a] = 0.0;
    }
    int hit = -1;
    if (P && cache) {
      for (int e = 0; e < cache->n; ++e)
        if (cache->mask[e] == P) {
          hit = e;
          break;
        }
    }
    if (hit >= 0) {
      // fast path: the passive set of the warm start is still optimal
      const double* C = cache->inv[hit];
      double z[K];
      apply(C, P, b, z);
      bool feasible = true;
#pragma unroll
      for (int a = 0; a < K; ++a)
        if (((P >> a) & 1u) && !(z[a] > 0.0)) feasible = false;
      if (feasible && entering(b, z, P, 0u, bmax) < 0) {
#pragma unroll
        for (int a = 0; a < K; ++a) y[a] = ((P >> a) & 1u) ? z[a] : 0.0;
        *mask_out = P;
        return 0;
      }
#pragma unroll
      for (int e = 0; e < K * K; ++e) A[e] = C[e];
    } else if (P) {
      const uint32_t Q = build(A, P, &blocked);
#pragma unroll
      for (int a = 0; a < K; ++a)
        if (((P & ~Q) >> a) & 1u) y[a] = 0.0;
      P = Q;
    }
    if (P) inner(A, b, y, P, blocked, -1);
    int status = 1;
#pragma unroll 1
    for (int outer = 0; outer < 5 * K + 10; ++outer) {
      const int t = entering(b, y, P, blocked, bmax);
      if (t < 0) {
        status = 0;
        break;
      }
      if (!add(A, P, t)) {
        blocked |= 1u << t;
        continue;
      }
      P |= 1u << t;
      inner(A, b, y, P, blocked, t);
    }
    uint32_t mask = 0;
#pragma unroll
    for (int a = 0; a < K; ++a)
      if (y[a] > 0.0) mask |= 1u << a;
    *mask_out = mask;
    return status;
  }
};

// ---------------------------------------------------------------------------
// Subset-inverse table (k <= 8): inv(G_PP) for every nonempty passive set P,
// entry P at tab[P * K * K] (row-major K x K, meaningful on P x P only).
// Built upward: the entry of P is the entry of P minus its highest index h,
// bordered with h (one reciprocal, O(K^2) FMAs) -- the same pivots as a
// Cholesky factorization of G_PP in ascending index order, so the oracle's
// pivot test applies unchanged.  All subsets of one level are built in
// parallel, so the dependency depth is K bordering steps.  ok[P] = 0 marks a
// subset whose pivot failed (or that inherits a failure).
// ---------------------------------------------------------------------------
template <int K>
__device__ void build_subset_table(const NnlsSolver<K>& S, double* tab, int* ok) {
  constexpr int NS = 1 << K;
  for (int L = 1; L <= K; ++L) {
    for (int P = (int)threadIdx.x; P < NS; P += (int)blockDim.x) {
      if (P == 0 || __popc(P) != L) continue;
      const int h = 31 - __clz(P);
      const int parent = P & ~(1 << h);
      double* A = tab + (size_t)P * K * K;
      bool good = true;
      if (parent) {
        const double* B = tab + (size_t)parent * K * K;
#pragma unroll
        for (int e = 0; e < K * K; ++e) A[e] = B[e];
        good = ok[parent] != 0;
      }
      good = good && S.add(A, (uint32_t)parent, h);
      ok[P] = good ? 1 : 0;
    }
    __syncthreads();
  }
}

// Lawson-Hanson driven by the subset table: every solve on a passive set P
// is z0 = A_P b_P followed by one step of iterative refinement
// z = z0 + A_P (b - G z0)_P, so the result is accurate even though the
// table entries were built by repeated bordering.  The entering test uses
// the residual b - G z0.  Returns 0 converged, 1 iteration cap, -1 when a
// needed table entry is marked degenerate (the caller then falls back to the
// incremental solver).
template <int K>
__device__ __forceinline__ int table_nnls(const NnlsSolver<K>& S, const double* tab, const int* ok,
                                          const double (&b)[K], double (&y)[K], bool warm,
                                          uint32_t* mask_out) {
  uint32_t P = 0, blocked = 0;
  double bmax = 0.0;
#pragma unroll
  for (int a = 0; a < K; ++a) {
    bmax = dmax_nn(bmax, dabs(b[a]));
    if (warm && dpos(y[a])) P |= 1u << a;
    else y[a] = 0.0;
  }
  int t_in = -1;
  int status = 1;
#pragma unroll 1
  for (int it = 0; it < 6 * K + 12; ++it) {
    double z[K], r[K];
    if (P) {
      if (!ok[P]) return -1;
      const double* A = tab + (size_t)P * K * K;
      double z0[K], rp[K];
#pragma unroll
      for (int a = 0; a < K; ++a) z0[a] = ((P >> a) & 1u) ? dot_masked<K>(A + a * K, b, P) : 0.0;
#pragma unroll
      for (int a = 0; a < K; ++a) r[a] = b[a] - dot_masked<K>(S.G + a * K, z0, P);
#pragma unroll
      for (int a = 0; a < K; ++a) rp[a] = ((P >> a) & 1u) ? r[a] : 0.0;
#pragma unroll
      for (int a = 0; a < K; ++a) z[a] = ((P >> a) & 1u) ? z0[a] + dot_masked<K>(A + a * K, rp, P) : 0.0;
    } else {
#pragma unroll
      for (int a = 0; a < K; ++a) {
        z[a] = 0.0;
        r[a] = b[a];
      }
    }
    uint32_t nonpos = 0;   // passive variables whose value is not positive
#pragma unroll
    for (int a = 0; a < K; ++a)
      if (((P >> a) & 1u) && !dpos(z[a])) nonpos |= 1u << a;
    if (t_in >= 0) {          // the entering variable must come out positive
      const int tt = t_in;
      t_in = -1;
      if ((nonpos >> tt) & 1u) {
        P &= ~(1u << tt);
        blocked |= 1u << tt;
        continue;             // y unchanged (y_tt = 0); re-solve on P
      }
    }
    if (nonpos) {
      // step from y towards z until the first passive variable reaches zero
      double alpha = 2.0;
      int q = -1;
#pragma unroll
      for (int a = 0; a < K; ++a) {
        if (!((nonpos >> a) & 1u)) continue;
        const double rr = y[a] * rcp64(y[a] - z[a]);
        if (rr < alpha) {
          alpha = rr;
          q = a;
        }
      }
      if (q < 0) {
        alpha = 0.0;
        q = __ffs(nonpos) - 1;
      }
      uint32_t drop = 1u << q;
#pragma unroll
      for (int a = 0; a < K; ++a) {
        if (!((P >> a) & 1u)) continue;
        y[a] = fmad(alpha, z[a] - y[a], y[a]);
        if (!dpos(y[a])) drop |= 1u << a;
      }
#pragma unroll
      for (int a = 0; a < K; ++a)
        if ((drop >> a) & 1u) y[a] = 0.0;
      P &= ~drop;
      continue;
    }
    double ymax = 0.0;
#pragma unroll
    for (int a = 0; a < K; ++a) {
      y[a] = ((P >> a) & 1u) ? z[a] : 0.0;
      ymax = dmax_nn(ymax, y[a]);
    }
    // entering test on w = b - G y (the residual of the unrefined solve)
    const double tol = 10.0 * K * S.eps * (bmax + S.gmax * ymax);
    uint32_t cand = 0;
#pragma unroll
    for (int a = 0; a < K; ++a)
      if (!(((P | blocked) >> a) & 1u) && dgt_nn(r[a], tol)) cand |= 1u << a;
    if (!cand) {
      status = 0;
      break;
    }
    int t = -1;
    double best = tol;
#pragma unroll
    for (int a = 0; a < K; ++a)
      if (((cand >> a) & 1u) && dgt_nn(r[a], best)) {
        best = r[a];
        t = a;
      }
    P |= 1u << t;
    t_in = t;
  }
  uint32_t mask = 0;
#pragma unroll
  for (int a = 0; a < K; ++a)
    if (dpos(y[a])) mask |= 1u << a;
  *mask_out = mask;
  return status;
}

// ---------------------------------------------------------------------------
// Lane-parallel Lawson-Hanson for k <= 8 with the subset table.
//
// FP64 on this part costs roughly one sub-partition FP64-unit pass per warp
// instruction whatever the number of active lanes, so a solver that keeps
// one column per lane pays for K-fold unrolled scalar work.  Here a warp
// solves 32 / KP columns at once, lane = column slot * KP + component a
// (KP = K rounded up to a power of two): every mat-vec is K FMAs per lane
// with the other components fetched by shuffles (integer pipe), and every
// per-column decision (feasibility, entering test, step ratio) is a ballot or
// an integer max/min over the KP-lane group.
// ---------------------------------------------------------------------------
template <int K>
struct LaneGroup {
  static constexpr int KP = K <= 1 ? 1 : K <= 2 ? 2 : K <= 4 ? 4 : 8;   // lanes per column
  static constexpr int CPW = 32 / KP;                                    // columns per warp
  static constexpr uint32_t GMASK = (KP == 32) ? 0xffffffffu : ((1u << KP) - 1u);
  int lane, a, base;
  __device__ void init() {
    lane = threadIdx.x & 31;
    a = lane & (KP - 1);
    base = lane & ~(KP - 1);
  }
  template <typename V>
  __device__ V from(V v, int c) const { return __shfl_sync(0xffffffffu, v, base + c); }
  // the group's bits of a warp ballot, bit a of the result = lane base + a
  __device__ uint32_t bits(bool pred) const { return (__ballot_sync(0xffffffffu, pred) >> base) & GMASK; }
  // max over the group of non-negative values (integer order of the bits)
  template <typename V>
  __device__ V max_nn(V v) const {
#pragma unroll
    for (int o = 1; o < KP; o <<= 1) v = vmax_nn(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
  }
};

// The subset table built level by level by lane groups: in level L every
// group of KP lanes takes one subset P with L elements and borders
// inv(G_{P-h}) (h the highest index of P) into inv(G_PP), lane a computing
// row a.  The arithmetic is that of NnlsSolver::add in the same order, so
// the entries equal those of build_subset_table; entries outside P are 0.
// The subsets of a level are enumerated in increasing order from warp
// ballots (no table in memory: after an L2 flush a memory lookup would wait
// behind the TMA stream of M).  Called by the `nthreads` threads starting at
// thread t0 (both multiples of 32); sync() must be a barrier over exactly
// those threads.  Warps without a subset in a round skip its arithmetic.
template <int K, typename V, typename Sync>
__device__ void build_subset_table_lanes_v(const V* Gm, V pivot_min, V* tab, int* ok, int t0, int nthreads,
                                           Sync sync) {
  static_assert(K <= 8, "subset tables are built for k <= 8");
  constexpr int KP = LaneGroup<K>::KP, CPW = LaneGroup<K>::CPW;
  constexpr int NC = (1 << K) - 1;              // candidate subsets 1 .. 2^K - 1
  constexpr int NB = (NC + 31) / 32;            // ballot words
  LaneGroup<K> g;
  g.init();
  const int local = (int)threadIdx.x - t0;
  const int group = local / KP, ngroups = nthreads / KP;
  const int wgroup = (local >> 5) * CPW;        // first group of this warp
  if (local == 0) ok[0] = 1;
#pragma unroll 1
  for (int L = 1; L <= K; ++L) {
    uint32_t words[NB];
    int ntask = 0;
#pragma unroll
    for (int w = 0; w < NB; ++w) {
      const int v = w * 32 + g.lane + 1;
      words[w] = __ballot_sync(0xffffffffu, v <= NC && __popc(v) == L);
      ntask += __popc(words[w]);
    }
#pragma unroll 1
    for (int base = 0; base < ntask; base += ngroups) {
      if (base + wgroup >= ntask) continue;     // warp-uniform
      const int task = base + group;
      const bool valid = task < ntask;
      uint32_t P = 1u;
      if (valid) {
        int r = task;
#pragma unroll
        for (int w = 0; w < NB; ++w) {
          const int c = __popc(words[w]);
          if (r >= 0 && r < c) P = (uint32_t)(w * 32 + 1 + (int)__fns(words[w], 0, r + 1));
          r -= c;
        }
      }
      const int h = 31 - __clz(P);
      const uint32_t par = P & ~(1u << h);
      const V* A = tab + (size_t)par * K * K;
      V gi[K];
#pragma unroll
      for (int c = 0; c < K; ++c) gi[c] = Gm[c * K + h];
      const bool ina = g.a < K && ((par >> g.a) & 1u);
      const V u = ina ? dot_masked_v<K, V>(A + g.a * K, gi, par) : V(0);
      V t = ina ? Gm[h * K + g.a] * u : V(0);
#pragma unroll
      for (int o = 1; o < KP; o <<= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      const V sp = Gm[h * K + h] - t;
      const bool good = valid && (par == 0 || ok[par] != 0) && (sp > pivot_min);
      const V rs = VOps<V>::rcp(sp);
      const V ua = u * rs;
      V* D = tab + (size_t)P * K * K + g.a * K;
#pragma unroll
      for (int c = 0; c < K; ++c) {
        const V uc = g.from(u, c);
        if (valid && g.a < K) {
          V v = V(0);
          if (ina) {
            if ((par >> c) & 1u) v = fmad(ua, uc, A[g.a * K + c]);
            else if (c == h) v = -ua;
          } else if (g.a == h) {
            if ((par >> c) & 1u) v = -(uc * rs);
            else if (c == h) v = rs;
          }
          D[c] = v;
        }
      }
      if (valid && g.a == 0) ok[P] = good ? 1 : 0;
    }
    sync();
  }
}

// The FP64 table of NnlsSolver's G (the same arithmetic as its bordering).
template <int K, typename Sync>
__device__ void build_subset_table_lanes(const NnlsSolver<K>& S, double* tab, int* ok, int t0, int nthreads,
                                         Sync sync) {
  build_subset_table_lanes_v<K, double>(S.G, S.pivot_min, tab, ok, t0, nthreads, sync);
}

// The subset table with every subset independent of the others: a group of
// KP lanes takes a subset P and inverts G_PP by Gauss-Jordan elimination in
// ascending index order (lane a holds row a of [G_PP | I]); the pivots are
// the Schur complements the bordering method tests, so the degenerate
// entries are the same, and the dependency chain is |P| pivot steps instead
// of k levels of bordering (a subset's inverse does not wait for its
// parent's).  For small k, where all 2^k - 1 subsets fit the groups of one
// round.  Called by the `nthreads` threads starting at thread t0 (multiples
// of 32); needs no barrier of its own.
template <int K>
__device__ void build_subset_table_gj(const double* Gm, double pivot_min, double* tab, int* ok, int t0,
                                      int nthreads) {
  static_assert(K <= 8, "subset tables are built for k <= 8");
  constexpr int NC = (1 << K) - 1;
  LaneGroup<K> g;
  g.init();
  const int local = (int)threadIdx.x - t0;
  const int group = local / LaneGroup<K>::KP, ngroups = nthreads / LaneGroup<K>::KP;
  const int nrounds = (NC + ngroups - 1) / ngroups;
#pragma unroll 1
  for (int rd = 0; rd < nrounds; ++rd) {   // rounds are warp-uniform: every lane runs every round
    const int task = rd * ngroups + group;
    const bool valid = task < NC;
    const uint32_t P = valid ? (uint32_t)(task + 1) : 1u;
    const bool ina = g.a < K && ((P >> g.a) & 1u);
    double R[K], I[K];
#pragma unroll
    for (int c = 0; c < K; ++c) {
      R[c] = (ina && ((P >> c) & 1u)) ? Gm[g.a * K + c] : 0.0;
      I[c] = (ina && c == g.a) ? 1.0 : 0.0;
    }
    bool good = true;
#pragma unroll
    for (int pv = 0; pv < K; ++pv) {
      // every lane of the warp runs every pivot step (the shuffles are
      // full-warp); a step whose index is not in the group's P changes nothing
      const bool inpv = (P >> pv) & 1u;
      const double piv = g.from(R[pv], pv);
      if (inpv) good = good && piv > pivot_min;
      const double rinv = VOps<double>::rcp(inpv ? piv : 1.0);
      const double f = R[pv] * rinv;   // this row's multiple of the pivot row
#pragma unroll
      for (int c = 0; c < K; ++c) {
        const double rp = g.from(R[c], pv), ip = g.from(I[c], pv);
        if (inpv && g.a == pv) {
          R[c] *= rinv;
          I[c] *= rinv;
        } else if (inpv && ina) {
          R[c] = fmad(-f, rp, R[c]);
          I[c] = fmad(-f, ip, I[c]);
        }
      }
    }
    if (valid && g.a < K) {
      double* D = tab + (size_t)P * K * K + g.a * K;
#pragma unroll
      for (int c = 0; c < K; ++c) D[c] = ina ? I[c] : 0.0;
    }
    if (valid && g.a == 0) ok[P] = good ? 1 : 0;
  }
  if (local == 0) ok[0] = 1;
}

// Solve the columns held by the warp.  Per lane: b = component a of the
// right-hand side, y = component a of the warm start (in) / solution (out),
// grow = row a of G (K values, registers).  tab / ok: subset table of G.
// Every collective (shuffle, ballot) is executed by all lanes in the same
// order; the per-column state machine acts through predicates only.
// Returns per lane the column's status (0 converged, 1 iteration cap, -1 a
// needed table entry is degenerate) and its passive set in *mask.
template <int K, typename V = double>
__device__ __forceinline__ int lane_table_nnls(const LaneGroup<K>& g, const V* tab, const int* ok,
                                               const V (&grow)[K], V gmax, V eps, V b, V& y, bool warm,
                                               bool active, bool refine, uint32_t* mask, int* entered = nullptr) {
  using O = VOps<V>;
  constexpr int KP = LaneGroup<K>::KP;
  const bool comp = active && g.a < K;
  V bc[K];
#pragma unroll
  for (int c = 0; c < K; ++c) bc[c] = g.from(b, c);
  const V bmax = g.max_nn(comp ? O::absv(b) : V(0));
  const bool ypos = comp && warm && vpos(y);
  uint32_t P = g.bits(ypos);
  if (!ypos) y = V(0);
  uint32_t blocked = 0;
  int t_in = -1, status = active ? 1 : 0, n_in = 0;
  bool done = !active;
#pragma unroll 1
  for (int it = 0; it < 6 * K + 12; ++it) {
    if (P && !done && !ok[P]) {
      status = -1;
      done = true;
    }
    if (__all_sync(0xffffffffu, done)) break;
    const bool inP = !done && ((P >> g.a) & 1u);
    const V* A = tab + (size_t)(inP ? P : 0) * K * K + g.a * K;
    V z0 = V(0);
    if (inP) {
#pragma unroll
      for (int c = 0; c < K; ++c)
        if ((P >> c) & 1u) z0 = fmad(A[c], bc[c], z0);
    }
    V r = b;   // r = b - G z0, all components
#pragma unroll
    for (int c = 0; c < K; ++c) r = fmad(-grow[c], g.from(z0, c), r);
    V z = z0;
    if (refine) {   // one step of iterative refinement on P
      const V rp = inP ? r : V(0);
      V corr = V(0);
#pragma unroll
      for (int c = 0; c < K; ++c) {
        const V rc = g.from(rp, c);
        if (inP && ((P >> c) & 1u)) corr = fmad(A[c], rc, corr);
      }
      z = z0 + corr;
    }
    const uint32_t nonpos = g.bits(comp && inP && !vpos(z));
    // a just-entered variable that does not come out positive is blocked
    bool reject = false;
    if (t_in >= 0) reject = (nonpos >> t_in) & 1u;
    // Lawson-Hanson step (columns with nonpos != 0 and no rejection)
    const bool stepping = !done && !reject && nonpos;
    V yn = V(0);
    uint32_t drop = 0;
    if (__any_sync(0xffffffffu, stepping)) {
      const bool mine = stepping && ((nonpos >> g.a) & 1u);
      V ratio = V(2);
      if (mine) {
        ratio = y * O::rcp(y - z);
        if (!(O::bits(ratio) >= 0)) ratio = V(0);
      }
      V amin = ratio;
#pragma unroll
      for (int o = 1; o < KP; o <<= 1) {
        const V w = __shfl_xor_sync(0xffffffffu, amin, o);
        amin = O::bits(w) < O::bits(amin) ? w : amin;
      }
      const uint32_t atmin = g.bits(mine && O::bits(ratio) == O::bits(amin));
      const V alpha = atmin ? amin : V(0);
      yn = (stepping && inP) ? fmad(alpha, z - y, y) : V(0);
      const int q = stepping ? __ffs(atmin ? atmin : nonpos) - 1 : 0;
      drop = g.bits(stepping && comp && inP && !vpos(yn));
      if (stepping) drop |= 1u << q;
    }
    // entering test (feasible columns): w = b - G y, the residual of the solve
    const bool feas = !done && !reject && !nonpos;
    const V yf = (feas && comp && inP) ? z : V(0);
    const V ymax = g.max_nn(yf);
    const V tol = V(10) * V(K) * eps * (bmax + gmax * ymax);
    const bool cand = feas && comp && !(((P | blocked) >> g.a) & 1u) && O::bits(r) > O::bits(tol);
    const uint32_t cands = g.bits(cand);
    V best = cand ? r : V(0);
#pragma unroll
    for (int o = 1; o < KP; o <<= 1) best = vmax_nn(best, __shfl_xor_sync(0xffffffffu, best, o));
    const uint32_t at = g.bits(cand && O::bits(r) == O::bits(best));
    // apply the per-column transition
    if (!done) {
      if (reject) {
        P &= ~(1u << t_in);
        blocked |= 1u << t_in;
        t_in = -1;
      } else if (nonpos) {
        t_in = -1;
        y = ((drop >> g.a) & 1u) ? V(0) : yn;
        P &= ~drop;
      } else {
        t_in = -1;
        y = yf;
        if (!cands) {
          status = 0;
          done = true;
        } else {
          const int t = __ffs(at) - 1;
          P |= 1u << t;
          t_in = t;
          ++n_in;
        }
      }
    }
  }
  *mask = g.bits(comp && vpos(y));
  if (entered) *entered = n_in;
  return status;
}

// Build the per-CTA inverse cache from up to CACHE_N sampled passive sets
// (called by every thread of the block; G must be in shared memory).
template <int K>
__device__ void build_cache(InvCache<K>* cache, const NnlsSolver<K>& S, const uint32_t* samples,
                            int nsamples) {
  if (threadIdx.x == 0) {
    int n = 0;
    for (int s = 0; s < nsamples; ++s) {
      const uint32_t msk = samples[s];
      if (!msk) continue;
      bool seen = false;
      for (int e = 0; e < n; ++e) seen |= cache->mask[e] == msk;
      if (!seen && n < CACHE_N) cache->mask[n++] = msk;
    }
    cache->n = n;
  }
  __syncthreads();
  const int e = threadIdx.x;
  if (e < cache->n) {
    uint32_t blocked = 0;
    const uint32_t Q = S.build(cache->inv[e], cache->mask[e], &blocked);
    if (Q != cache->mask[e]) cache->mask[e] = 0xffffffffu;   // degenerate: never matches
  }
  __syncthreads();
}

// Warp-level version of build_cache (called by the 32 lanes of one warp).
template <int K>
__device__ void build_cache_warp(InvCache<K>* cache, const NnlsSolver<K>& S, const uint32_t* samples,
                                 int nsamples) {
  const int lane = threadIdx.x & 31;
  if (lane == 0) {
    int n = 0;
    for (int s = 0; s < nsamples; ++s) {
      const uint32_t msk = samples[s];
      if (!msk) continue;
      bool seen = false;
      for (int e = 0; e < n; ++e) seen |= cache->mask[e] == msk;
      if (!seen && n < CACHE_N) cache->mask[n++] = msk;
    }
    cache->n = n;
  }
  __syncwarp();
  if (lane < cache->n) {
    uint32_t blocked = 0;
    const uint32_t Q = S.build(cache->inv[lane], cache->mask[lane], &blocked);
    if (Q != cache->mask[lane]) cache->mask[lane] = 0xffffffffu;
  }
  __syncwarp();
}

}  // namespace nmfgb

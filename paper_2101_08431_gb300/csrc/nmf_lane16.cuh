// Lawson-Hanson NNLS of 16-variable problems on 16-lane groups (lane a <->
// variable a): the column solves of the rank-16 tensor-core M pass and the
// row solves of the rank-16 row pass.
#pragma once

#include "nmf_common.cuh"
#include "nmf_nnls.cuh"

namespace nmfgb {

// ---------------------------------------------------------------------------
// One 16-variable problem on a 16-lane group (lane a <-> variable a), the same algorithm and decisions as the one-thread solver:
// warm start from the support of y, entering test w_a > tol with
// tol = 10 k eps (max|b| + max G_aa max|y|), lowest index on ties, Schur
// pivot <= 1e-14 max G_aa blocks the variable, at most 5k + 10 outer steps.
// A = inv(G_PP) is kept row-distributed (lane a holds row a) and carried from
// column to column: a column whose warm passive set equals the carried one
// costs two lane-parallel mat-vecs.  V is the value type of the solve.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float vrcp(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double vrcp(double x) { return rcp64(x); }
// bit patterns as signed integers: for values >= 0 (and -0) and negative
// sentinels their order is that of the values, so maxima and arg-maxima of
// such values take integer instructions instead of FP64 ones
__device__ __forceinline__ int vbits(float x) { return __float_as_int(x); }
__device__ __forceinline__ long long vbits(double x) { return __double_as_longlong(x); }
// x != 0 (either sign of zero) on the bit pattern
__device__ __forceinline__ bool vnz(float x) { return ((unsigned)__float_as_int(x) << 1) != 0u; }
__device__ __forceinline__ bool vnz(double x) { return ((unsigned long long)__double_as_longlong(x) << 1) != 0ull; }

template <typename V>
struct LaneNnls16 {
  static constexpr int K = 16;
  static constexpr int UPD_MAX = 48;   // rank-one updates of a carried inverse before it is rebuilt
  const V (*Gp)[K + 1];
  V A[K];             // row a of inv(G_PcPc)
  uint32_t Pc;        // passive set of the carried inverse
  int upd;            // rank-one updates since it was built
  V gmax, pivot_min, eps;
  int a, base;
  unsigned gm;

  __device__ void init(const V (*G)[K + 1], V eps_) {
    Gp = G;
    const int lane = threadIdx.x & 31;
    a = lane & 15;
    base = lane & 16;
    gm = 0xFFFFu << base;
    V g = 0;
#pragma unroll
    for (int c = 0; c < K; ++c) g = fmax(g, fabs(G[c][c]));
    gmax = g;
    pivot_min = (V)1e-14 * g;
    eps = eps_;
#pragma unroll
    for (int c = 0; c < K; ++c) A[c] = 0;
    Pc = 0;
    upd = 0;
  }
  __device__ __forceinline__ V bc(V v, int c) const { return __shfl_sync(gm, v, base + c); }
  __device__ __forceinline__ V gsum(V v) const {
#pragma unroll
    for (int o = 8; o >= 1; o >>= 1) v += __shfl_xor_sync(gm, v, o);
    return v;
  }
  // maximum over the group of values >= 0 (NaN only from non-finite input)
  __device__ __forceinline__ V gmaxv(V v) const {
#pragma unroll
    for (int o = 8; o >= 1; o >>= 1) {
      const V w = __shfl_xor_sync(gm, v, o);
      v = vbits(w) > vbits(v) ? w : v;
    }
    return v;
  }
  __device__ __forceinline__ uint32_t gballot(bool p) const { return (__ballot_sync(gm, p) >> base) & 0xFFFFu; }
  __device__ __forceinline__ bool in(uint32_t P) const { return (P >> a) & 1u; }

  // Loops over the 16 variables skip, by branches uniform on the group, the
  // variables whose terms are exact zeros (outside P, or y_c == 0): the same
  // sums in the same accumulators as over all 16, for a fraction of the
  // instructions (each FP64 warp instruction holds a sub-partition's FP64
  // unit for tens of cycles on this part).
  // z_P = A b_P (zero outside P)
  __device__ V apply(uint32_t P, V b) const {
    V z0 = 0, z1 = 0, z2 = 0, z3 = 0;
#pragma unroll
    for (int c = 0; c < K; ++c) {
      if ((P >> c) & 1u) {
        const V v = bc(b, c);
        if ((c & 3) == 0) z0 = fmad(A[c], v, z0);
        else if ((c & 3) == 1) z1 = fmad(A[c], v, z1);
        else if ((c & 3) == 2) z2 = fmad(A[c], v, z2);
        else z3 = fmad(A[c], v, z3);
      }
    }
    return in(P) ? (z0 + z1) + (z2 + z3) : (V)0;
  }
  // (G y)_a
  __device__ V gdot(V y) const {
    const uint32_t S = gballot(vnz(y));
    V s0 = 0, s1 = 0, s2 = 0, s3 = 0;
#pragma unroll
    for (int c = 0; c < K; ++c) {
      if ((S >> c) & 1u) {
        const V v = bc(y, c);
        if ((c & 3) == 0) s0 = fmad(Gp[a][c], v, s0);
        else if ((c & 3) == 1) s1 = fmad(Gp[a][c], v, s1);
        else if ((c & 3) == 2) s2 = fmad(Gp[a][c], v, s2);
        else s3 = fmad(Gp[a][c], v, s3);
      }
    }
    return (s0 + s1) + (s2 + s3);
  }
  // entering variable of the outer loop (or -1)
  __device__ int entering(V b, V y, uint32_t P, uint32_t blocked, V bmax) const {
    const V ymax = gmaxv(y);
    const V tol = (V)(10.0 * K) * eps * (bmax + gmax * ymax);
    const V w = b - gdot(y);
    const bool cand = !(((P | blocked) >> a) & 1u) && w > tol;
    V bw = cand ? w : (V)-1;   // candidates: w > tol >= 0
    int bi = cand ? a : 99;
#pragma unroll
    for (int o = 8; o >= 1; o >>= 1) {
      const V ow = __shfl_xor_sync(gm, bw, o);
      const int oi = __shfl_xor_sync(gm, bi, o);
      if (vbits(ow) > vbits(bw) || (vbits(ow) == vbits(bw) && oi < bi)) {
        bw = ow;
        bi = oi;
      }
    }
    return bi < K ? bi : -1;
  }
  // A = inv(G_PP) -> inv(G_{P+i}); false (A unchanged) if the pivot fails
  __device__ bool add(uint32_t P, int i) {
    V u0 = 0, u1 = 0;
#pragma unroll
    for (int c = 0; c < K; ++c) {
      if ((P >> c) & 1u) {
        const V g = Gp[i][c];   // G[i][c]: one shared-memory word for the group
        if (c & 1) u1 = fmad(A[c], g, u1);
        else u0 = fmad(A[c], g, u0);
      }
    }
    const V gia = Gp[i][a], gii = Gp[i][i];
    const V u = in(P) ? u0 + u1 : (V)0;
    const V s = gii - gsum(gia * u);
    if (!(s > pivot_min)) return false;
    const V rs = vrcp(s);
    const V ua = u * rs;
    const bool pa = in(P);
#pragma unroll
    for (int c = 0; c < K; ++c) {
      if ((P >> c) & 1u) {
        // lane i: -u_c / s; the lanes of P: A_ac + u_a u_c / s (one FMA for both)
        const V uc = bc(u, c);
        const V nv = fmad(a == i ? -rs : ua, uc, a == i ? (V)0 : A[c]);
        if (a == i || pa) A[c] = nv;
      } else if (c == i) {
        if (a == i) A[c] = rs;
        else if (pa) A[c] = -ua;
      } else if (a == i) {
        A[c] = (V)0;
      }
    }
    ++upd;
    return true;
  }
  // A = inv(G_PP), i in P -> inv(G_{P-i})
  __device__ void remove(uint32_t P, int i) {
    V cia = 0;
#pragma unroll
    for (int c = 0; c < K; ++c)
      if (c == i) cia = A[c];
    const V rd = vrcp(bc(cia, i));
    const V f = cia * rd;
    const bool keep = in(P) && a != i;
#pragma unroll
    for (int c = 0; c < K; ++c) {
      if (((P >> c) & 1u) && c != i) {
        const V cc = bc(cia, c);
        if (keep) A[c] = fmad(-f, cc, A[c]);
      }
    }
    ++upd;
  }
  // carried inverse -> inverse for P (variables whose pivot fails are blocked)
  __device__ uint32_t rebase(uint32_t P, uint32_t& blocked) {
    const uint32_t diff = Pc ^ P;
    if (Pc == 0 || upd > UPD_MAX || __popc(diff) > __popc(P)) {
      uint32_t Q = 0, rest = P;
      upd = 0;
      while (rest) {
        const int i = __ffs(rest) - 1;
        rest &= rest - 1;
        if (add(Q, i)) Q |= 1u << i;
        else blocked |= 1u << i;
      }
      Pc = Q;
      return Q;
    }
    uint32_t out = Pc & ~P;
    while (out) {
      const int i = __ffs(out) - 1;
      out &= out - 1;
      remove(Pc, i);
      Pc &= ~(1u << i);
    }
    uint32_t inn = P & ~Pc;
    while (inn) {
      const int i = __ffs(inn) - 1;
      inn &= inn - 1;
      if (add(Pc, i)) Pc |= 1u << i;
      else blocked |= 1u << i;
    }
    return Pc;
  }
  // inner loop from the feasible y (y_P > 0); t_in just entered (or -1)
  __device__ void inner(V b, V& y, uint32_t& P, uint32_t& blocked, int t_in) {
    bool first = true;
#pragma unroll 1
    for (int it = 0; it <= K + 1; ++it) {
      if (!P) {
        y = 0;
        Pc = 0;
        return;
      }
      const V z = apply(P, b);
      if (first && t_in >= 0) {
        if (!(bc(z, t_in) > (V)0)) {
          remove(P, t_in);
          P &= ~(1u << t_in);
          Pc = P;
          blocked |= 1u << t_in;
          return;
        }
      }
      first = false;
      const uint32_t infeas = gballot(in(P) && !(z > (V)0));
      if (!infeas) {
        y = in(P) ? z : (V)0;
        return;
      }
      V r = 2;
      int ri = 99;
      if ((infeas >> a) & 1u) {
        r = y * vrcp(y - z);
        ri = a;
      }
#pragma unroll
      for (int o = 8; o >= 1; o >>= 1) {
        const V orr = __shfl_xor_sync(gm, r, o);
        const int oi = __shfl_xor_sync(gm, ri, o);
        if (orr < r || (orr == r && oi < ri)) {
          r = orr;
          ri = oi;
        }
      }
      V alpha = r;
      int q = (r < (V)2) ? ri : -1;
      if (q < 0) {   // only reachable through NaN: take the first infeasible one
        alpha = 0;
        q = __ffs(infeas) - 1;
      }
      if (in(P)) y = fmad(alpha, z - y, y);
      uint32_t drop = (1u << q) | gballot(in(P) && !(y > (V)0));
      if ((drop >> a) & 1u) y = 0;
      while (drop) {
        const int i = __ffs(drop) - 1;
        drop &= drop - 1;
        remove(P, i);
        P &= ~(1u << i);
      }
      Pc = P;
    }
  }
  // Full solve: y holds the warm start (lane a: component a) and the
  // solution on exit.  Returns 0 when converged, 1 at the iteration cap.
  __device__ int solve(V b, V& y, bool warm, uint32_t* mask_out) {
    uint32_t blocked = 0;
    const V bmax = gmaxv(fabs(b));
    if (!(warm && y > (V)0)) y = 0;
    uint32_t P = gballot(y > (V)0);
    if (P) {
      if (P == Pc) {
        const V z = apply(P, b);
        const bool feas = !gballot(in(P) && !(z > (V)0));
        if (feas && entering(b, z, P, 0u, bmax) < 0) {
          y = in(P) ? z : (V)0;
          *mask_out = P;
          return 0;
        }
      } else {
        const uint32_t Q = rebase(P, blocked);
        if (!in(Q)) y = 0;
        P = Q;
      }
      if (P) inner(b, y, P, blocked, -1);
    }
    int status = 1;
#pragma unroll 1
    for (int outer = 0; outer < 5 * K + 10; ++outer) {
      const int t = entering(b, y, P, blocked, bmax);
      if (t < 0) {
        status = 0;
        break;
      }
      if (P != Pc) {
        uint32_t bl2 = 0;
        P = rebase(P, bl2);
        blocked |= bl2;
      }
      if (!add(P, t)) {
        blocked |= 1u << t;
        continue;
      }
      P |= 1u << t;
      Pc = P;
      inner(b, y, P, blocked, t);
    }
    *mask_out = gballot(y > (V)0);
    return status;
  }
};

// ---------------------------------------------------------------------------
// FP32-predicted, FP64-accurate solve of one 16-variable problem on a 16-lane
// group.  An FP32 Lawson-Hanson solve (nf: its inverse of G_PP is carried
// from problem to problem) finds the passive set P and x in FP32; steps of
// iterative refinement x_P += inv(G_PP) (b - G x)_P -- the residual in FP64,
// the correction through the FP32 inverse -- bring x to FP64 accuracy (each
// step multiplies the error by ~2^-24 cond(G_PP)) until the correction is at
// most rtol max|x| (at most maxit steps; with `converge`, a refinement that
// has not reached rtol by then is not accepted).  x is accepted when the FP64
// optimality test holds: x_P > 0 and no gradient b - G x above the entering
// tolerance 10 k eps (max|b| + max G_aa max|x|) outside P.  A variable the
// test finds entering (the largest gradient, lowest index on ties) is added
// to P through the FP32 inverse and x refined again, at most twice (the
// FP32 solve's coarser tolerance leaves out such variables near an
// optimum).  G64: row a of G in FP64 (lane a).  Returns true when accepted
// (x, *mask set); otherwise x holds the refined point, a warm start for the
// FP64 solve.
// ---------------------------------------------------------------------------
// (b - G x)_a over the components in S (x is zero outside S: the terms
// skipped are exact zeros); S uniform on the group
__device__ __forceinline__ double resid64(const double* G64, double b, double x, unsigned gm, int base, uint32_t S) {
  double s0 = b, s1 = 0.0, s2 = 0.0, s3 = 0.0;
#pragma unroll
  for (int c = 0; c < 16; ++c) {
    if ((S >> c) & 1u) {
      const double v = __shfl_sync(gm, x, base + c);
      if ((c & 3) == 0) s0 = fmad(-G64[c], v, s0);
      else if ((c & 3) == 1) s1 = fmad(-G64[c], v, s1);
      else if ((c & 3) == 2) s2 = fmad(-G64[c], v, s2);
      else s3 = fmad(-G64[c], v, s3);
    }
  }
  return (s0 + s1) + (s2 + s3);
}

__device__ __forceinline__ bool predict_refine16(LaneNnls16<float>& nf, const double* G64, double gdiag_max, double b,
                                                 double& x, uint32_t* mask, int* status, bool warm, double eps,
                                                 double rtol, int maxit, bool converge) {
  constexpr int K = 16;
  float xv = (float)x;
  uint32_t P = 0;
  const int st = nf.solve((float)b, xv, warm, &P);
  *status = st;
  x = (double)xv;
  if (st != 0 || P != nf.Pc) return false;
  double bmax = dabs(b);
#pragma unroll
  for (int o = 8; o >= 1; o >>= 1) bmax = dmax_nn(bmax, __shfl_xor_sync(nf.gm, bmax, o));
  for (int round = 0; round < 3; ++round) {
    const bool inP = (P >> nf.a) & 1u;
    bool conv = false;
    for (int it = 0; it < maxit; ++it) {
      const double rr = resid64(G64, b, x, nf.gm, nf.base, P);   // x is zero outside P
      const float dz = nf.apply(P, (float)rr);
      if (inP) x += (double)dz;
      double dmax = inP ? dabs((double)dz) : 0.0, xmax = inP ? dabs(x) : 0.0;
#pragma unroll
      for (int o = 8; o >= 1; o >>= 1) {
        dmax = dmax_nn(dmax, __shfl_xor_sync(nf.gm, dmax, o));
        xmax = dmax_nn(xmax, __shfl_xor_sync(nf.gm, xmax, o));
      }
      if (dmax <= rtol * xmax) {
        conv = true;
        break;
      }
    }
    if (converge && !conv) return false;                // G_PP too ill conditioned for the FP32 inverse
    if (nf.gballot(inP && !(x > 0.0))) return false;   // infeasible: the FP64 solve decides
    const double w = resid64(G64, b, x, nf.gm, nf.base, P);
    double xmax = inP ? dabs(x) : 0.0;
#pragma unroll
    for (int o = 8; o >= 1; o >>= 1) xmax = dmax_nn(xmax, __shfl_xor_sync(nf.gm, xmax, o));
    const double tol = 10.0 * K * eps * (bmax + gdiag_max * xmax);
    const bool cand = !inP && w > tol;
    if (!nf.gballot(cand)) {
      if (!inP) x = 0.0;
      *mask = P;
      return true;
    }
    if (round == 2) break;
    // the largest entering gradient (lowest index on ties) joins P
    double bw = cand ? w : -1.0;
    int bi = cand ? nf.a : 99;
#pragma unroll
    for (int o = 8; o >= 1; o >>= 1) {
      const double ow = __shfl_xor_sync(nf.gm, bw, o);
      const int oi = __shfl_xor_sync(nf.gm, bi, o);
      if (vbits(ow) > vbits(bw) || (vbits(ow) == vbits(bw) && oi < bi)) {   // candidates w > tol >= 0
        bw = ow;
        bi = oi;
      }
    }
    if (bi >= K || !nf.add(P, bi)) return false;
    P |= 1u << bi;
    nf.Pc = P;
  }
  return false;
}

}  // namespace nmfgb

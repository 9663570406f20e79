// Rank-16 refinement passes of the mixed form where n is beyond the rows of
// the cluster-fused FP64-class kernels.  Like the k <= 8 refinement they come
// in two kinds (Sec. 2's sweep, with FP64-accurate contractions):
//
//   reference sweep   B = X^T M and P = M Y^T in compensated FP32
//                     ("double-float", ~44 significant bits; FP32 instructions
//                     only, on a part whose FP64 rate is ~1/60 of its FP32
//                     rate), FP64 column and row solves; it records
//                     B_ref = X_t^T M, Y_ref = Y_{t+1} (here) and X_ref,
//                     P_ref = M Y_{t+1}^T (the row pass)
//   incremental sweep B = B_ref + (X - X_ref)^T M, P = P_ref + M (Y - Y_ref)^T
//                     with the change terms on the tensor cores (the
//                     split-BF16 GEMMs of nmf_tc16s.cuh: their 2^-15 relative
//                     error is of the change, not of the contraction), FP64
//                     column and row solves
//
// dfb_kernel   B partials: CTA (row block of BR rows, column slice); X of the
//              block in shared memory as hi/lo FP32 pairs; warp w takes
//              columns w, w + 8, ... of the slice, lane l rows l + 32 t; the
//              16 double-float sums of a lane are reduce-scattered over the
//              warp and written as FP64 partials Bdf[row block][column]
// dfp_kernel   P partials: CTA (256 rows, column split), lane <-> row; y of a
//              chunk of columns in shared memory (hi/lo pairs, broadcast
//              reads); FP64 partials into Ppart[split][row]
// solve64_kernel  the FP64 column solves of both kinds (16-lane groups on
//              runs of columns ordered by passive set, carried inverse), FP64
//              KKT terms and H,
//              the records, and the split of Y - Y_ref for the incremental
//              P-GEMM
#pragma once

#include "nmf_arith.cuh"
#include "nmf_tc16s.cuh"

namespace nmfgb {
namespace tc16r {

using tc16s::xs_off;
constexpr int K = 16;
constexpr int BR = 512;       // rows of a B-partial block
constexpr int TB = 256;       // threads of dfb_kernel
constexpr int XSTR = 20;      // floats per row of the staged X (16 + 4: conflict-free 16-byte reads)
constexpr int TP = 256;       // threads (rows) of a dfp_kernel CTA
constexpr int PCH = 64;       // columns of y staged per chunk
constexpr int SOLVE_T = 256;

__host__ __device__ constexpr size_t dfb_smem() { return (size_t)2 * BR * XSTR * sizeof(float); }

// ---------------------------------------------------------------------------
// B partials: Bdf[rb][col][c] = sum over the block's rows of X_ic M_ij
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(TB, 2) dfb_kernel(Problem p, double* Bdf, RefPlan R) {
  extern __shared__ __align__(16) float xsm[];
  float* xh = xsm;
  float* xl = xsm + BR * XSTR;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (p.st->done) return;
  const int cur = p.st->iter & 1;
  const int rb = blockIdx.x % R.nrbB, slice = blockIdx.x / R.nrbB;
  const int r0 = rb * BR, rows = min(BR, p.ld - r0);
  for (int e = tid; e < BR * K; e += TB) {
    const int i = e >> 4, c = e & 15, row = r0 + i;
    const double x = (i < rows && row < p.n) ? p.X[cur][(size_t)row * K + c] : 0.0;
    const float hi = __double2float_rn(x);
    xh[i * XSTR + c] = hi;
    xl[i * XSTR + c] = __double2float_rn(x - (double)hi);
  }
  __syncthreads();
  const int c0 = (int)(((long long)slice * p.m) / R.slicesB), c1 = (int)(((long long)(slice + 1) * p.m) / R.slicesB);
  const float* M = static_cast<const float*>(p.M);
  const int nt = rows / 32;
  for (int col = c0 + warp; col < c1; col += TB / 32) {
    const float* mc = M + (size_t)wrap_col(p.head, col, p.mcap) * p.ld + r0;
    DF acc[K];
#pragma unroll
    for (int c = 0; c < K; ++c) acc[c] = ArDF::zero();
    float mv[BR / 32];   // the column's rows of the block, all loads in flight at once
#pragma unroll
    for (int t = 0; t < BR / 32; ++t) mv[t] = t < nt ? __ldg(mc + lane + 32 * t) : 0.f;
#pragma unroll
    for (int t = 0; t < BR / 32; ++t) {
      if (t >= nt) break;
      const int i = lane + 32 * t;
      const float m = mv[t];
      const float4* h4 = reinterpret_cast<const float4*>(xh + i * XSTR);
      const float4* l4 = reinterpret_cast<const float4*>(xl + i * XSTR);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float4 h = h4[q], l = l4[q];
        acc[4 * q + 0] = ArDF::madd(m, DF{h.x, l.x}, acc[4 * q + 0]);
        acc[4 * q + 1] = ArDF::madd(m, DF{h.y, l.y}, acc[4 * q + 1]);
        acc[4 * q + 2] = ArDF::madd(m, DF{h.z, l.z}, acc[4 * q + 2]);
        acc[4 * q + 3] = ArDF::madd(m, DF{h.w, l.w}, acc[4 * q + 3]);
      }
    }
    const DF s = warp_reduce_scatter_ar<ArDF, K>(acc);   // lane l: component l & 15
    if (lane < K) Bdf[((size_t)rb * p.mcap + col) * K + lane] = (double)s.hi + (double)s.lo;
  }
}

// ---------------------------------------------------------------------------
// P partials: Ppart[s][row][c] = sum over the split's columns of M_ij y_jc
// (y = Y[nxt] after a sweep's solves, Y[cur] in the priming pass)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(TP) dfp_kernel(Problem p, RefPlan R, int mode) {
  __shared__ __align__(16) float yh[PCH][K];
  __shared__ __align__(16) float yl[PCH][K];
  const int tid = threadIdx.x;
  if (p.st->done) return;
  const int yb = (p.st->iter & 1) ^ (mode == MODE_SWEEP ? 1 : 0);
  const int rb = blockIdx.x % R.nrbP, split = blockIdx.x / R.nrbP;
  const int row = rb * TP + tid;
  const int c0 = (int)(((long long)split * p.m) / R.SPd), c1 = (int)(((long long)(split + 1) * p.m) / R.SPd);
  const float* M = static_cast<const float*>(p.M);
  DF acc[K];
#pragma unroll
  for (int c = 0; c < K; ++c) acc[c] = ArDF::zero();
  for (int j0 = c0; j0 < c1; j0 += PCH) {
    const int nc = min(PCH, c1 - j0);
    __syncthreads();   // the previous chunk is consumed
    for (int e = tid; e < nc * K; e += TP) {
      const int jj = e >> 4, c = e & 15;
      const double y = p.Y[yb][(size_t)wrap_col(p.head, j0 + jj, p.mcap) * K + c];
      const float hi = __double2float_rn(y);
      yh[jj][c] = hi;
      yl[jj][c] = __double2float_rn(y - (double)hi);
    }
    __syncthreads();
    if (row < p.ld) {
      constexpr int PF = 8;   // columns whose M values are loaded ahead
      float mv[PF];
#pragma unroll
      for (int u = 0; u < PF; ++u)
        mv[u] = u < nc ? __ldg(M + (size_t)wrap_col(p.head, j0 + u, p.mcap) * p.ld + row) : 0.f;
      for (int jj = 0; jj < nc; ++jj) {
        const float m = mv[0];
#pragma unroll
        for (int u = 0; u < PF - 1; ++u) mv[u] = mv[u + 1];
        mv[PF - 1] = jj + PF < nc ? __ldg(M + (size_t)wrap_col(p.head, j0 + jj + PF, p.mcap) * p.ld + row) : 0.f;
        const float4* h4 = reinterpret_cast<const float4*>(&yh[jj][0]);
        const float4* l4 = reinterpret_cast<const float4*>(&yl[jj][0]);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float4 h = h4[q], l = l4[q];
          acc[4 * q + 0] = ArDF::madd(m, DF{h.x, l.x}, acc[4 * q + 0]);
          acc[4 * q + 1] = ArDF::madd(m, DF{h.y, l.y}, acc[4 * q + 1]);
          acc[4 * q + 2] = ArDF::madd(m, DF{h.z, l.z}, acc[4 * q + 2]);
          acc[4 * q + 3] = ArDF::madd(m, DF{h.w, l.w}, acc[4 * q + 3]);
        }
      }
    }
  }
  if (row < p.ld) {
    double* out = static_cast<double*>(p.Ppart) + ((size_t)split * p.ld + row) * K;
#pragma unroll
    for (int c = 0; c < K; ++c) out[c] = (double)acc[c].hi + (double)acc[c].lo;
  }
}

// ---------------------------------------------------------------------------
// FP64 column solves of the refinement sweeps.  kind REF: b = sum of the
// row-block partials of dfb_kernel, and with record_refs B_ref = b,
// Y_ref = the new y; kind INC: b = B_ref + the SB tensor-core partials of the
// change, and the split of y - Y_ref for the incremental P-GEMM.  KKT terms
// and H in FP64; the block partials are summed (tc16s::reduce_blocks) into
// Hpart[0], Yterms[0] and entries 1 .. Q-1 are zeroed (Q: the P partials of
// the pass).
// ---------------------------------------------------------------------------
enum Kind { REF = 0, INC = 1 };

__global__ void __launch_bounds__(SOLVE_T, 2) solve64_kernel(Problem p, tc16s::Bufs bf, const double* Bdf,
                                                             RefPlan R, int cpg, int nbpart, int Q, int kind,
                                                             int mode) {
  __shared__ double Gd[K][K + 1];
  __shared__ double wred[SOLVE_T / 32][tc16s::RED];
  __shared__ unsigned last;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  DevState* st = p.st;
  if (st->done) return;
  const int cur = st->iter & 1, nxt = cur ^ 1;
  for (int e = tid; e < K * K; e += SOLVE_T) Gd[e / K][e % K] = p.G[e];
  __syncthreads();
  LaneNnls16<double> nn;
  // FP64 solves with the tolerance constant of the compensated contractions
  nn.init(Gd, 5.684341886080802e-14);
  const int a = nn.a;
  const int ncols = p.m, ncolp = (ncols + tc16s::PG_COLS - 1) / tc16s::PG_COLS * tc16s::PG_COLS;
  const int gid = blockIdx.x * (SOLVE_T / 16) + (tid >> 4);
  const int cbeg = min(ncolp, gid * cpg), cend = min(ncolp, cbeg + cpg);
  const bool inc = kind == INC;
  double acc_t[NYT];
#pragma unroll
  for (int e = 0; e < NYT; ++e) acc_t[e] = 0.0;
  double hacc[9];   // lane a: H[a][(a + d) % 16], d = 0..8
#pragma unroll
  for (int d = 0; d < 9; ++d) hacc[d] = 0.0;
  for (int ci = cbeg; ci < cend; ++ci) {
    if (ci >= ncols) {
      if (inc && mode != MODE_KKT) {
        *reinterpret_cast<uint16_t*>(bf.Ys + xs_off(ci, a)) = 0;
        *reinterpret_cast<uint16_t*>(bf.Ys + xs_off(ci, K + a)) = 0;
      }
      continue;
    }
    const int col = bf.perm[ci];   // columns in the order of their passive sets (sort_cols_kernel)
    const int phys = wrap_col(p.head, col, p.mcap);
    const double yo = p.Y[cur][(size_t)phys * K + a];
    const uint32_t om = p.ymask[cur][phys];
    double b = 0.0;
    if (mode != MODE_PRIME) {
      if (inc) {
        double d = 0.0;
        for (int s = 0; s < nbpart; ++s) d += (double)bf.Bpart[((size_t)s * p.mcap + col) * K + a];
        b = p.Bref[(size_t)phys * K + a] + d;
      } else {
        for (int s = 0; s < nbpart; ++s) b += Bdf[((size_t)s * p.mcap + col) * K + a];
      }
    }
    double yn = yo;
    uint32_t msk = 0;
    int stt = 0;
    if (mode == MODE_SWEEP) stt = nn.solve(b, yn, p.warm != 0, &msk);
    if (mode != MODE_PRIME) {
      // Y-half KKT terms of the incoming iterate: g = G yo - b (component a)
      const double gy = nn.gdot(yo) - b;
      const double mn = dminz(gy), pos = dmaxz(gy) * yo;
      acc_t[YT_NEG] = fmad(mn, mn, acc_t[YT_NEG]);
      acc_t[YT_COMP] = fmad(pos, pos, acc_t[YT_COMP]);
      acc_t[YT_BNORM2] = fmad(b, b, acc_t[YT_BNORM2]);
      acc_t[YT_BY] = fmad(b, yo, acc_t[YT_BY]);
      acc_t[YT_YGY] = fmad(yo, gy + b, acc_t[YT_YGY]);
      acc_t[YT_YMAX] = dmax_nn(acc_t[YT_YMAX], yo);
      acc_t[YT_YNORM2] = fmad(yo, yo, acc_t[YT_YNORM2]);
      if (!isfinite(b)) set_err(st, ERR_NONFINITE);
    }
    if (mode == MODE_SWEEP) {
      acc_t[YT_DY2] = fmad(yn - yo, yn - yo, acc_t[YT_DY2]);
      if (a == 0) {
        acc_t[YT_CHANGED] += (om != msk) ? 1.0 : 0.0;
        acc_t[YT_NOTCONV] += (double)stt;
      }
      p.Y[nxt][(size_t)phys * K + a] = yn;
      if (a == 0) p.ymask[nxt][phys] = msk;
      if (!inc && p.record_refs) {
        p.Bref[(size_t)phys * K + a] = b;
        p.Yref[(size_t)phys * K + a] = yn;
      }
    } else if (mode == MODE_PRIME) {
      const uint32_t pm = (__ballot_sync(nn.gm, dpos(yo)) >> nn.base) & 0xFFFFu;
      if (a == 0) p.ymask[cur][phys] = pm;
    }
    if (mode != MODE_KKT) {
#pragma unroll
      for (int d = 0; d < 9; ++d) hacc[d] = fmad(yn, __shfl_sync(nn.gm, yn, nn.base + ((a + d) & 15)), hacc[d]);
      if (inc) {   // the change of y since the reference, split for the P-GEMM
        const float dy = __double2float_rn(yn - p.Yref[(size_t)phys * K + a]);
        const uint16_t h = tc16s::bf16_bits(dy);
        const uint16_t l = tc16s::bf16_bits(dy - tc16s::bf16_val(h));
        *reinterpret_cast<uint16_t*>(bf.Ys + xs_off(col, a)) = h;
        *reinterpret_cast<uint16_t*>(bf.Ys + xs_off(col, K + a)) = l;
      }
    }
  }
  // warp partials (fixed order: the two halves, then the triangle entries)
#pragma unroll
  for (int d = 0; d < 9; ++d) hacc[d] += __shfl_xor_sync(0xffffffffu, hacc[d], 16);
  if (lane < 16) {
#pragma unroll
    for (int d = 0; d < 9; ++d) {
      const int c = (a + d) & 15;
      if (d < 8 || a < 8) {
        wred[warp][a * K + c] = hacc[d];
        wred[warp][c * K + a] = hacc[d];
      }
    }
  }
#pragma unroll
  for (int e = 0; e < NYT; ++e) {
    const double v = (e == YT_YMAX) ? warp_max(acc_t[e]) : warp_sum(acc_t[e]);
    if (lane == 0) wred[warp][K * K + e] = v;
  }
  __syncthreads();
  constexpr int RED = tc16s::RED;
  double* myred = bf.red + (size_t)blockIdx.x * RED;
  for (int e = tid; e < RED; e += SOLVE_T) {
    double v = wred[0][e];
    for (int w = 1; w < SOLVE_T / 32; ++w) v = (e == K * K + YT_YMAX) ? dmax_nn(v, wred[w][e]) : v + wred[w][e];
    myred[e] = v;
  }
  const double* tot = tc16s::reduce_blocks(bf, &last);
  if (!tot) return;
  for (int e = tid; e < RED; e += SOLVE_T) {
    const double v = tot[e];
    if (e < K * K) {
      p.Hpart[e] = (mode == MODE_KKT) ? 0.0 : v;
      for (int q = 1; q < Q; ++q) p.Hpart[(size_t)q * K * K + e] = 0.0;
    } else {
      p.Yterms[e - K * K] = v;
      for (int q = 1; q < Q; ++q) p.Yterms[(size_t)q * NYT + e - K * K] = 0.0;
    }
  }
}

// split of X - X_ref for the incremental B-GEMM (rows >= n zero)
__global__ void xdsplit_kernel(Problem p, tc16s::Bufs bf) {
  if (p.st->done) return;
  const int cur = p.st->iter & 1;
  const int total = p.ld * K;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const int i = e >> 4, c = e & 15;
    const double x = i < p.n ? p.X[cur][(size_t)i * K + c] - p.Xref[(size_t)i * K + c] : 0.0;
    const uint16_t h = tc16s::bf16_bits((float)x);
    const uint16_t l = tc16s::bf16_bits((float)(x - (double)tc16s::bf16_val(h)));
    *reinterpret_cast<uint16_t*>(bf.Xs + xs_off(i, c)) = h;
    *reinterpret_cast<uint16_t*>(bf.Xs + xs_off(i, K + c)) = l;
  }
}

}  // namespace tc16r
}  // namespace nmfgb

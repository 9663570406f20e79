// The ANLS sweep on GB300 (Alg. "anls" of Sec. 2, Y-update first):
//
//   ypass  : one fused pass over M.  A cluster of C CTAs owns a contiguous
//            range of time columns; CTA c of the cluster owns rows
//            [c R, (c+1) R).  Column tiles of TJ columns are staged into
//            shared memory by the bulk-copy (TMA) engine through an S-deep
//            mbarrier ring.  Per tile: B = X^T M_tile (thread-owned rows,
//            reduce-scatter in the warp, fixed-order sums across warps and,
//            through distributed shared memory, across the cluster), one FP64
//            warm-started NNLS per column (problem "qp" with C = X), then
//            P += M_tile Y_tile^T and H += Y_tile Y_tile^T from the same
//            staged tile -- M is read from HBM exactly once per sweep.  The
//            same pass produces the Y-half KKT terms of the incoming iterate
//            (graY = G y - b, eq. "eqn:kkt").
//   xpass  : one thread per row of X: sums the P partials (fixed order),
//            solves the row NNLS (problem "qp" with C = Y^T), and the last
//            block to finish forms G = X^T X for the next sweep together with
//            the objective and KKT error of the iterate from the Grams
//            (Sec. 5.1), with no second read of M.
#pragma once

#include "nmf_arith.cuh"
#include "nmf_nnls.cuh"
#include "nmf_lane16.cuh"

namespace nmfgb {

// Compile-time tile shape of the M pass (AR: accumulation policy).  The CTA
// has NCW compute warps (rows, contraction, P update) and one NNLS warp.
template <typename TM, typename AR, int K>
struct YTraits {
  static constexpr bool WIDE = sizeof(typename AR::V) == 8;   // 8-byte staged factors
  static constexpr bool PSM = AR::PACC_SMEM;                   // P accumulators in shared memory
  static constexpr int T = 512;
  static constexpr int NCW = 15;                               // compute warps
  static constexpr int TC = NCW * 32;                          // compute threads
  static constexpr int RPT = (WIDE && !PSM) ? (K <= 4 ? 3 : (K <= 8 ? 2 : 1)) : (K <= 4 ? 7 : (K <= 8 ? 4 : 2));
  // shared-memory bytes of the P accumulators per owned row (PSM only)
  static constexpr int PACC_ROW_BYTES = PSM ? K * (int)sizeof(typename AR::A) : 0;
  static constexpr int TJ = WIDE ? (K <= 4 ? 4 : (K <= 8 ? 2 : 1)) : (K <= 4 ? 8 : (K <= 8 ? 4 : 2));
  static constexpr int V = TJ * K;
  static constexpr int VP = (V <= 1) ? 1 : (V <= 2) ? 2 : (V <= 4) ? 4 : (V <= 8) ? 8 : (V <= 16) ? 16 : 32;
  static_assert(V <= 32, "B tile must fit one warp reduce-scatter");
  static constexpr int ROWS = RPT * TC;                        // rows per CTA at most
  // value type of the column solves: FP64 in every pass.  (An FP32 solve
  // from an FP32 subset table carries about 2^-24 cond(G_PP), which exceeds
  // the FP32 contraction's own error wherever G is not well conditioned.)
  static constexpr bool F32NN = false;
  using NV = typename std::conditional<F32NN, float, double>::type;
  // the NNLS warp builds the table in shared memory: FP32 solves (k <= 8),
  // FP64 solves at k <= 6 (k = 7, 8: the FP64 table built by the row pass)
  static constexpr bool LOCAL_TAB = F32NN || K <= 6;
};

__host__ __device__ inline int wrap_col(int head, int j, int mcap) {
  int p = head + j;
  return p >= mcap ? p - mcap : p;
}

// Shared-memory layout of the M pass (dynamic smem, 128-byte aligned parts).
template <typename TM, typename AR, int K>
struct YSmem {
  using Tr = YTraits<TM, AR, K>;
  struct Small {
    uint64_t full[8];                  // stage barriers (S <= 8)
    uint64_t bready[2];                // B of a tile reduced (compute -> NNLS warp)
    uint64_t yready[2];                // y of a tile solved (NNLS warp -> compute)
    uint64_t xbar[2];                  // cluster exchange of B partials
    double G[K * K];
    double Hacc[K * K];
    double Bfull[2][Tr::VP];
    double Bpart[Tr::VP];
    typename AR::R red[Tr::NCW][Tr::VP];
    typename AR::R xch[2][8][Tr::VP];  // cluster exchange slots (C <= 8)
    double ybufD[2][Tr::TJ][K];
    typename AR::V ybufA[2][Tr::TJ][K];
    double yt[Tr::TJ][NYT];            // per-column-lane KKT / objective terms (k > 8)
    double lt[32][NYT];                // per-lane KKT / objective terms (k <= 8)
    uint32_t samples[CACHE_N];
    union {
      InvCache<K> cache;               // k > 8 only (no subset table)
      double lh[32][K];                // k <= 8: per-lane accumulators of H rows
    };
    // subset table of G built by the NNLS warp, in the value type of the
    // solve: FP32 for the FP32 pass, FP64 otherwise; Gn: G in that type
    typename Tr::NV gtab[Tr::LOCAL_TAB ? (1 << K) * K * K : 1];
    int gok[Tr::LOCAL_TAB ? (1 << K) : 1];
    typename Tr::NV Gn[K * K];
  };
  static constexpr size_t SMALL_BYTES = (sizeof(Small) + 127) & ~size_t(127);
  __host__ __device__ static constexpr size_t small_bytes() { return SMALL_BYTES; }
  __host__ __device__ static size_t stage_bytes(int R) { return size_t(Tr::TJ) * R * sizeof(TM); }
};

// The M pass of column group q (of Q) by one cluster of C CTAs, each owning
// R rows; smem_raw: the dynamic shared memory (small part, S stages, and the
// P accumulators when the policy keeps them there).  Called by all threads
// of the CTA; leaves every barrier it used invalidated, so that a persistent
// caller can run it again on the same memory.
template <typename TM, typename AR, int K>
__device__ __forceinline__ void ypass_body(const Problem& p, int mode, int S, int C, int R, int Q, int q,
                                           unsigned char* smem_raw) {
  using Tr = YTraits<TM, AR, K>;
  using Sm = YSmem<TM, AR, K>;
  using VT = typename AR::V;
  using AT = typename AR::A;
  constexpr int TC = Tr::TC, NCW = Tr::NCW, RPT = Tr::RPT, TJ = Tr::TJ, VP = Tr::VP;
  constexpr bool TABLE = K <= 8;
  typename Sm::Small& sm = *reinterpret_cast<typename Sm::Small*>(smem_raw);
  TM* stages = reinterpret_cast<TM*>(smem_raw + Sm::small_bytes());

  cg::cluster_group cluster = cg::this_cluster();
  const int crank = (int)cluster.block_rank();
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  DevState* st = p.st;
  if (st->done) return;                       // uniform: written by an earlier launch
  const int cur = st->iter & 1, nxt = cur ^ 1;

  const int c0 = (int)(((long long)q * p.m) / Q);
  const int c1 = (int)(((long long)(q + 1) * p.m) / Q);
  const int ncols = c1 - c0;
  const int ntiles = (ncols + TJ - 1) / TJ;
  const int r0 = crank * R;
  const int rows_c = max(0, min(R, p.ld - r0));
  const TM* M = static_cast<const TM*>(p.M);

  if (tid == 0) {
    for (int s = 0; s < S; ++s) mbar_init(&sm.full[s], 1);
    for (int b = 0; b < 2; ++b) {
      mbar_init(&sm.bready[b], 1);
      mbar_init(&sm.yready[b], 1);
      mbar_init(&sm.xbar[b], (uint32_t)(C * VP));
    }
    fence_mbar_init();
  }
  for (int e = tid; e < TJ * NYT; e += Tr::T) (&sm.yt[0][0])[e] = 0.0;
  for (int e = tid; e < K * K; e += Tr::T) sm.Hacc[e] = 0.0;
  if (C > 1) cluster.sync();
  else __syncthreads();

  auto issue = [&](int t, int s) {
    const int tj = min(TJ, ncols - t * TJ);
    const uint32_t bytes = (uint32_t)rows_c * (uint32_t)sizeof(TM);
    mbar_arrive_expect_tx(&sm.full[s], bytes * (uint32_t)tj);
    if (bytes) {
      TM* dst = stages + (size_t)s * TJ * R;
      for (int jj = 0; jj < tj; ++jj) {
        const int phys = wrap_col(p.head, c0 + t * TJ + jj, p.mcap);
        bulk_g2s(dst + (size_t)jj * R, M + (size_t)phys * p.ld + r0, bytes, &sm.full[s]);
      }
    }
  };
  bool timed_out = false;

  if (warp < NCW) {
    // ======================= compute warps ==================================
    if (tid == 0)
      for (int t = 0; t < min(S, ntiles); ++t) issue(t, t);
    VT xr[RPT][K];
    constexpr bool PSM = Tr::PSM;
    AT pacc[PSM ? 1 : RPT][K];
    // PSM: accumulators component-major behind the stages, ps[a * R + rr]
    AT* ps = reinterpret_cast<AT*>(smem_raw + Sm::small_bytes() + (size_t)S * Sm::stage_bytes(R));
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
      const int row = r0 + tid + r * TC;
      const bool ok = (tid + r * TC) < rows_c && row < p.n;
#pragma unroll
      for (int a = 0; a < K; ++a) {
        xr[r][a] = ok ? AR::load_x(p, cur, (size_t)row * K + a) : AR::vzero();
        if constexpr (PSM) {
          if (tid + r * TC < R) ps[(size_t)a * R + tid + r * TC] = AR::zero();
        } else {
          pacc[r][a] = AR::zero();
        }
      }
    }
    // Iteration t contracts tile t (t < ntiles) and then accumulates tile
    // t - 1 (t >= 1) once the NNLS warp has solved it: P += M_tile Y_tile^T
    // on the own rows and H += Y_tile Y_tile^T.  One code path keeps the row
    // accumulators in registers.
    for (int t = 0; t <= ntiles; ++t) {
      if (t < ntiles) {
        const int s = t % S, slot = t & 1;
        if (!mbar_wait(&sm.full[s], (uint32_t)((t / S) & 1))) timed_out = true;
        const TM* tile = stages + (size_t)s * TJ * R;
        // ---- B partial = X_rows^T M_tile over this thread's rows
        AT acc[VP];
#pragma unroll
        for (int e = 0; e < VP; ++e) acc[e] = AR::zero();
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
          const int rr = tid + r * TC;
          if (rr < rows_c) {
#pragma unroll
            for (int jj = 0; jj < TJ; ++jj) {
              const TM mv = tile[(size_t)jj * R + rr];
#pragma unroll
              for (int a = 0; a < K; ++a) acc[jj * K + a] = AR::madd(mv, xr[r][a], acc[jj * K + a]);
            }
          }
        }
        {
          const AT wsum = warp_reduce_scatter_ar<AR, VP>(acc);
          if (lane < VP) sm.red[warp][lane] = AR::to_r(wsum);
        }
        named_sync(1, TC);
        // 4 lanes per value, then a quad tree; sums in the pass's reduction
        // type R (double-float for the FP32 passes: no FP64 instruction here)
        using RT = typename AR::R;
        if (tid < ((4 * VP + 31) & ~31)) {
          const int v = tid >> 2, g = tid & 3;
          RT bs = AR::to_r(AR::zero());
          if (v < VP) {
#pragma unroll
            for (int w = g; w < NCW; w += 4) bs = AR::radd(bs, sm.red[w][v]);
          }
          bs = AR::radd(bs, AR::rshfl_xor(bs, 1));
          bs = AR::radd(bs, AR::rshfl_xor(bs, 2));
          if (g == 0 && v < VP) {
            if (C > 1) {
              // push this CTA's partial to every CTA of the cluster
              for (int rk = 0; rk < C; ++rk) {
                RT* dst = cluster.map_shared_rank(&sm.xch[slot][crank][v], rk);
                *dst = bs;
                mbar_arrive_remote(&sm.xbar[slot], (uint32_t)rk);
              }
            } else {
              sm.Bfull[slot][v] = AR::r_to_double(bs);
            }
          }
        }
        if (C > 1) {
          if (!mbar_wait_cluster(&sm.xbar[slot], (uint32_t)((t >> 1) & 1))) timed_out = true;
          if (tid < VP) {
            RT bs = sm.xch[slot][0][tid];
            for (int c = 1; c < C; ++c) bs = AR::radd(bs, sm.xch[slot][c][tid]);
            sm.Bfull[slot][tid] = AR::r_to_double(bs);
          }
        }
        named_sync(1, TC);
        if (tid == 0) mbar_arrive(&sm.bready[slot]);
      }
      if (t >= 1) {
        const int u = t - 1, ub = u & 1;
        if (!mbar_wait(&sm.yready[ub], (uint32_t)((u >> 1) & 1))) timed_out = true;
        if (mode != MODE_KKT) {
          const int tj = min(TJ, ncols - u * TJ);
          const TM* tile = stages + (size_t)(u % S) * TJ * R;
          if constexpr (PSM) {
            // accumulators in shared memory: a row loop unrolled twice keeps
            // the (long, compensated) body small for the instruction cache
            // and still gives 2 K independent chains; the tile's y values are
            // staged once
            VT yv[TJ][K];
#pragma unroll
            for (int jj = 0; jj < TJ; ++jj)
#pragma unroll
              for (int a = 0; a < K; ++a) yv[jj][a] = sm.ybufA[ub][jj][a];
#pragma unroll 2
            for (int rr = tid; rr < rows_c; rr += TC) {
              AT pa[K];
#pragma unroll
              for (int a = 0; a < K; ++a) pa[a] = ps[(size_t)a * R + rr];
#pragma unroll
              for (int jj = 0; jj < TJ; ++jj) {
                if (jj < tj) {
                  const TM mv = tile[(size_t)jj * R + rr];
#pragma unroll
                  for (int a = 0; a < K; ++a) pa[a] = AR::madd(mv, yv[jj][a], pa[a]);
                }
              }
#pragma unroll
              for (int a = 0; a < K; ++a) ps[(size_t)a * R + rr] = pa[a];
            }
          } else {
#pragma unroll
            for (int r = 0; r < RPT; ++r) {
              const int rr = tid + r * TC;
              if (rr < rows_c) {
#pragma unroll
                for (int jj = 0; jj < TJ; ++jj) {
                  if (jj < tj) {
                    const TM mv = tile[(size_t)jj * R + rr];
#pragma unroll
                    for (int a = 0; a < K; ++a)
                      pacc[PSM ? 0 : r][a] = AR::madd(mv, sm.ybufA[ub][jj][a], pacc[PSM ? 0 : r][a]);
                  }
                }
              }
            }
          }
          if (!TABLE && tid >= 32 && tid < 32 + K * K) {   // k > 8: pairwise tree over the tile's columns
            // (k <= 8: H is accumulated by the NNLS warp)
            const int e = tid - 32, a = e / K, c = e % K;
            double hp[TJ];
#pragma unroll
            for (int jj = 0; jj < TJ; ++jj) hp[jj] = jj < tj ? sm.ybufD[ub][jj][a] * sm.ybufD[ub][jj][c] : 0.0;
#pragma unroll
            for (int w = 1; w < TJ; w <<= 1)
#pragma unroll
              for (int jj = 0; jj + w < TJ; jj += 2 * w) hp[jj] += hp[jj + w];
            sm.Hacc[e] += hp[0];
          }
        }
        named_sync(1, TC);                       // every compute thread is done with stage u % S
        if (tid == 0 && u + S < ntiles) issue(u + S, u % S);
      }
    }

    // ---- epilogue: partials of this cluster
    if constexpr (TABLE) {
      // the NNLS warp's per-lane KKT terms and H accumulators, reduced in
      // the fixed butterfly orders of one warp each (a term over the 32
      // lanes; a column of H over the lane groups' column slots), one item
      // per compute warp
      constexpr int KP = LaneGroup<K>::KP;
      for (int item = warp; item < NYT + K; item += NCW) {
        if (item < NYT) {
          const double v0 = sm.lt[lane][item];
          const double v = (item == YT_YMAX) ? warp_max(v0) : warp_sum(v0);
          if (lane == 0) sm.yt[0][item] = v;
        } else {
          const int c = item - NYT;
          double v = sm.lh[lane][c];
#pragma unroll
          for (int o = KP; o < 32; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
          const int a = lane & (KP - 1);
          if (lane < KP && a < K) sm.Hacc[a * K + c] = v;
        }
      }
      named_sync(1, TC);
    }
    typename AR::P* Pp = static_cast<typename AR::P*>(p.Ppart);
    if (mode != MODE_KKT) {
#pragma unroll
      for (int r = 0; r < RPT; ++r) {
        const int rr = tid + r * TC;
        const int row = r0 + rr;
        if (rr < rows_c && row < p.n) {
#pragma unroll
          for (int a = 0; a < K; ++a)
            Pp[((size_t)q * p.ld + row) * K + a] =
                AR::to_p(PSM ? ps[(size_t)a * R + rr] : pacc[PSM ? 0 : r][a]);
        }
      }
    }
    if (crank == 0) {
      if (tid < K * K) p.Hpart[(size_t)q * K * K + tid] = (mode == MODE_KKT) ? 0.0 : sm.Hacc[tid];
      if (tid < NYT) {   // fixed-order combine of the column lanes' terms
        double v = sm.yt[0][tid];
        for (int jj = 1; jj < TJ; ++jj) v = (tid == YT_YMAX) ? fmax(v, sm.yt[jj][tid]) : v + sm.yt[jj][tid];
        p.Yterms[(size_t)q * NYT + tid] = v;
      }
    }
  } else {
    // ======================= NNLS warp ======================================
    for (int e = lane; e < K * K; e += 32) sm.G[e] = p.G[e];
    if (!TABLE) {
      if (lane < CACHE_N) {
        uint32_t msk = 0;
        if (mode == MODE_SWEEP && p.warm && ncols > 0) {
          const int j = c0 + (int)(((long long)lane * ncols) / CACHE_N);
          msk = p.ymask[cur][wrap_col(p.head, j, p.mcap)];
        }
        sm.samples[lane] = msk;
      }
      if (lane == 0) sm.cache.n = 0;
    }
    __syncwarp();
    NnlsSolver<K> solver;
    solver.init(sm.G, AR::EPS);
    if (!TABLE && mode == MODE_SWEEP) build_cache_warp<K>(&sm.cache, solver, sm.samples, CACHE_N);
    // k <= 6: the subset table of G is built below by this warp while the
    // compute warps contract the first tile (k = 7, 8: by the previous row pass)
    double Ascr[K * K];   // scratch of the incremental solver (k > 8, degenerate entries)
    if (TABLE) {
      // lanes <-> (column slot jj, component a); per-lane KKT accumulators
      LaneGroup<K> g;
      g.init();
      const int jj = lane / LaneGroup<K>::KP;
      const bool ca = g.a < K;
      using NV = typename Tr::NV;
      constexpr bool F32NN = Tr::F32NN;
      double grow[K];   // row a of G (FP64: the KKT terms)
#pragma unroll
      for (int c = 0; c < K; ++c) grow[c] = ca ? sm.G[g.a * K + c] : 0.0;
      if constexpr (F32NN) {
        for (int e = lane; e < K * K; e += 32) sm.Gn[e] = (NV)sm.G[e];
        __syncwarp();
      }
      NV grown[K];      // row a of G in the solve's type
#pragma unroll
      for (int c = 0; c < K; ++c) grown[c] = (NV)grow[c];
      double* acc_t = sm.lt[lane];
#pragma unroll
      for (int e = 0; e < NYT; ++e) acc_t[e] = 0.0;
      double hacc[K];   // row a of H = Y Y^T over this warp's column slots
#pragma unroll
      for (int c = 0; c < K; ++c) hacc[c] = 0.0;
      // k = 7, 8 always, k <= 6 when the row pass's tail has built it: the
      // table of G in global memory; otherwise this warp builds it below
      // (FP32 solves: always this warp's own FP32 table)
      const bool gglob = !F32NN && (K > 6 || ((p.tab_global || p.gtab_tail) && st->gtab_valid));
      const NV* gtab;
      const int* gok;
      if constexpr (F32NN) {
        gtab = sm.gtab;
        gok = sm.gok;
      } else {
        gtab = gglob ? p.Gtab : sm.gtab;
        gok = gglob ? p.Gok : sm.gok;
      }
      // warm start and passive set of the next tile, fetched one tile ahead
      // (incremental sweeps: with the column's reference contraction and y)
      constexpr bool INC = AR::INC;
      double yo_nx = 0.0, br_nx = 0.0, yr_nx = 0.0;
      uint32_t om_nx = 0;
      int ph_nx = 0;
      if (jj < min(TJ, ncols)) {
        ph_nx = wrap_col(p.head, c0 + jj, p.mcap);
        if (ca) yo_nx = p.Y[cur][(size_t)ph_nx * K + g.a];
        if (INC && ca && mode == MODE_SWEEP) {
          br_nx = p.Bref[(size_t)ph_nx * K + g.a];
          yr_nx = p.Yref[(size_t)ph_nx * K + g.a];
        }
        om_nx = p.ymask[cur][ph_nx];
      }
      // chain warm start: the last solved column's new y (component g.a)
      double chain_y = 0.0;
      bool chain_started = false;
      if constexpr (Tr::LOCAL_TAB) {
        if (mode == MODE_SWEEP && !gglob) {
          if constexpr (F32NN)
            build_subset_table_lanes_v<K, NV>(sm.Gn, (NV)solver.pivot_min, sm.gtab, sm.gok, NCW * 32, 32,
                                              [] { __syncwarp(); });
          else
            build_subset_table_lanes<K>(solver, sm.gtab, sm.gok, NCW * 32, 32, [] { __syncwarp(); });
        }
      }
      for (int t = 0; t < ntiles; ++t) {
        const int slot = t & 1;
        const int tj = min(TJ, ncols - t * TJ);
        const bool active = jj < tj;
        const bool comp = active && ca;
        const double yo = yo_nx, bref = br_nx, yref = yr_nx;
        const uint32_t old_mask = om_nx;
        const int phys = ph_nx;
        yo_nx = br_nx = yr_nx = 0.0;
        om_nx = 0;
        ph_nx = 0;
        if (t + 1 < ntiles && jj < min(TJ, ncols - (t + 1) * TJ)) {
          ph_nx = wrap_col(p.head, c0 + (t + 1) * TJ + jj, p.mcap);
          if (ca) yo_nx = p.Y[cur][(size_t)ph_nx * K + g.a];
          if (INC && ca && mode == MODE_SWEEP) {
            br_nx = p.Bref[(size_t)ph_nx * K + g.a];
            yr_nx = p.Yref[(size_t)ph_nx * K + g.a];
          }
          om_nx = p.ymask[cur][ph_nx];
        }
        if (!mbar_wait(&sm.bready[slot], (uint32_t)((t >> 1) & 1))) timed_out = true;
        // incremental sweeps: B = Bref + (X - Xref)^T m_j
        const double b = comp ? (INC ? bref + sm.Bfull[slot][jj * K + g.a] : sm.Bfull[slot][jj * K + g.a]) : 0.0;
        if (mode != MODE_PRIME) {
          // Y-half KKT terms of the incoming iterate: g = G y - b (component a)
          double gy = -b;
#pragma unroll
          for (int c = 0; c < K; ++c) gy = fmad(grow[c], g.from(yo, c), gy);
          if (comp) {
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
        }
        double yn = yo;
        if (mode == MODE_SWEEP) {
          uint32_t msk = 0;
          int stt = 0, nin = 0;
          // one warm-started solve of the columns whose lanes have `act` set,
          // from ystart; a degenerate table entry falls back to the
          // incremental solver on the group's first lane
          auto solve_cols = [&](double ystart, bool act, double& yo_out, uint32_t& msk_out, int& st_out,
                                int& nin_out) {
            NV ynv = (NV)ystart;
            int ss = lane_table_nnls<K, NV>(g, gtab, gok, grown, (NV)solver.gmax, (NV)AR::EPS, (NV)b, ynv,
                                            p.warm != 0, act, AR::REFINE, &msk_out, &nin_out);
            yo_out = (double)ynv;
            if (__any_sync(0xffffffffu, ss < 0)) {
              double bb[K], yy[K];
#pragma unroll
              for (int c = 0; c < K; ++c) {
                bb[c] = g.from(b, c);
                yy[c] = g.from(ystart, c);
              }
              uint32_t m2 = 0;
              int s2 = 0;
              if (ss < 0 && g.a == 0) s2 = solver.solve(Ascr, bb, yy, p.warm != 0, nullptr, &m2);
#pragma unroll
              for (int c = 0; c < K; ++c) {
                const double v = __shfl_sync(0xffffffffu, yy[c], g.base);
                if (ss < 0 && g.a == c) yo_out = v;
              }
              const uint32_t mm = __shfl_sync(0xffffffffu, m2, g.base);
              const int s3 = __shfl_sync(0xffffffffu, s2, g.base);
              if (ss < 0) {
                msk_out = mm;
                ss = s3;
              }
            }
            st_out = ss;
          };
          if (p.warm == 2) {
            // the paper's chain (Sec. 2): the tile's columns one after
            // another, each starting from the previous column's new solution
            // (the CTA's first column from its own previous-sweep solution)
            for (int sl = 0; sl < TJ; ++sl) {
              if (sl >= tj) break;                       // uniform: tj is the same on every lane
              const double ystart = chain_started ? chain_y : yo;
              double ys = 0.0;
              uint32_t ms = 0;
              int sts = 0, ns = 0;
              solve_cols(ystart, active && jj == sl, ys, ms, sts, ns);
              if (jj == sl) {
                yn = ys;
                msk = ms;
                stt = sts;
                nin = ns;
              }
              chain_y = __shfl_sync(0xffffffffu, ys, sl * LaneGroup<K>::KP + (ca ? g.a : 0));
              chain_started = true;
            }
          } else {
            solve_cols(yo, active, yn, msk, stt, nin);
          }
          if (comp) acc_t[YT_DY2] = fmad(yn - yo, yn - yo, acc_t[YT_DY2]);
          if (active && g.a == 0) {
            acc_t[YT_CHANGED] += (old_mask != msk) ? 1.0 : 0.0;
            acc_t[YT_NOTCONV] += (double)stt;
            acc_t[YT_ENTER] += (double)nin;
          }
          if (crank == 0 && active) {
            if (ca) p.Y[nxt][(size_t)phys * K + g.a] = yn;
            if (g.a == 0) p.ymask[nxt][phys] = msk;
            if (p.record_refs && ca) {   // references for the incremental sweeps
              p.Bref[(size_t)phys * K + g.a] = b;
              p.Yref[(size_t)phys * K + g.a] = yn;
            }
          }
        } else {
          const uint32_t msk = g.bits(comp && dpos(yo));
          if (mode == MODE_PRIME && crank == 0 && active && g.a == 0) p.ymask[cur][phys] = msk;
        }
        if (mode != MODE_KKT) {
          const double yv = comp ? yn : 0.0;
#pragma unroll
          for (int c = 0; c < K; ++c) hacc[c] = fmad(yv, g.from(yv, c), hacc[c]);
        }
        if (jj < TJ && ca) {
          sm.ybufD[slot][jj][g.a] = active ? yn : 0.0;
          // incremental sweeps accumulate M (Y - Yref)^T
          sm.ybufA[slot][jj][g.a] = AR::yval(active ? (INC && mode == MODE_SWEEP ? yn - yref : yn) : 0.0);
        }
        if (t == ntiles - 1) {
          // the per-lane H accumulators to shared memory (the KKT terms are
          // there already), before the last release: the compute warps
          // reduce both in the epilogue, off this warp's FP64 chain
#pragma unroll
          for (int c = 0; c < K; ++c) sm.lh[lane][c] = hacc[c];
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&sm.yready[slot]);
      }
    } else {
      for (int t = 0; t < ntiles; ++t) {
        const int slot = t & 1;
        const int tj = min(TJ, ncols - t * TJ);
        double yo[K], yn[K];
        uint32_t old_mask = 0;
        int phys = 0;
        constexpr bool INC = AR::INC;
        const bool inc = INC && mode == MODE_SWEEP;
        if (lane < tj) {   // warm start and passive set, fetched before B is ready
          phys = wrap_col(p.head, c0 + t * TJ + lane, p.mcap);
#pragma unroll
          for (int a = 0; a < K; ++a) yo[a] = p.Y[cur][(size_t)phys * K + a];
          old_mask = p.ymask[cur][phys];
        }
        if (!mbar_wait(&sm.bready[slot], (uint32_t)((t >> 1) & 1))) timed_out = true;
#pragma unroll
        for (int a = 0; a < K; ++a) yn[a] = 0.0;
        if (lane < tj) {
          double b[K];
#pragma unroll
          for (int a = 0; a < K; ++a)
            b[a] = sm.Bfull[slot][lane * K + a] + (inc ? p.Bref[(size_t)phys * K + a] : 0.0);
          double* yt = sm.yt[lane];
          if (mode != MODE_PRIME) {
            double neg = 0.0, comp = 0.0, bn = 0.0, by = 0.0, ygy = 0.0, ymax = 0.0, yn2 = 0.0;
#pragma unroll
            for (int a = 0; a < K; ++a) {
              const double gv = dot_masked<K>(sm.G + a * K, yo, 0xffffffffu) - b[a];
              const double mn = dminz(gv), pos = dmaxz(gv) * yo[a];
              neg = fmad(mn, mn, neg);
              comp = fmad(pos, pos, comp);
              bn = fmad(b[a], b[a], bn);
              by = fmad(b[a], yo[a], by);
              ygy = fmad(yo[a], gv + b[a], ygy);
              ymax = dmax_nn(ymax, yo[a]);
              yn2 = fmad(yo[a], yo[a], yn2);
              if (!isfinite(b[a])) set_err(st, ERR_NONFINITE);
            }
            yt[YT_NEG] += neg;
            yt[YT_COMP] += comp;
            yt[YT_BNORM2] += bn;
            yt[YT_BY] += by;
            yt[YT_YGY] += ygy;
            yt[YT_YMAX] = dmax_nn(yt[YT_YMAX], ymax);
            yt[YT_YNORM2] += yn2;
          }
          if (mode == MODE_SWEEP) {
#pragma unroll
            for (int a = 0; a < K; ++a) yn[a] = yo[a];
            uint32_t msk = 0;
            const int stt = solver.solve(Ascr, b, yn, p.warm != 0, &sm.cache, &msk);
            double d2 = 0.0;
#pragma unroll
            for (int a = 0; a < K; ++a) d2 = fmad(yn[a] - yo[a], yn[a] - yo[a], d2);
            yt[YT_DY2] += d2;
            yt[YT_CHANGED] += (old_mask != msk) ? 1.0 : 0.0;
            yt[YT_NOTCONV] += (double)stt;
            if (crank == 0) {
#pragma unroll
              for (int a = 0; a < K; ++a) p.Y[nxt][(size_t)phys * K + a] = yn[a];
              p.ymask[nxt][phys] = msk;
              if (p.record_refs) {
#pragma unroll
                for (int a = 0; a < K; ++a) {
                  p.Bref[(size_t)phys * K + a] = b[a];
                  p.Yref[(size_t)phys * K + a] = yn[a];
                }
              }
            }
          } else {
            uint32_t msk = 0;
#pragma unroll
            for (int a = 0; a < K; ++a) {
              yn[a] = yo[a];
              if (dpos(yo[a])) msk |= 1u << a;
            }
            if (mode == MODE_PRIME && crank == 0) p.ymask[cur][phys] = msk;
          }
        }
        if (lane < TJ) {
#pragma unroll
          for (int a = 0; a < K; ++a) {
            sm.ybufD[slot][lane][a] = yn[a];
            sm.ybufA[slot][lane][a] =
                AR::yval((inc && lane < tj) ? yn[a] - p.Yref[(size_t)phys * K + a] : yn[a]);
          }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&sm.yready[slot]);
      }
    }
  }
  if (timed_out) set_err(st, ERR_TIMEOUT);
  __syncthreads();
  if (tid == 0) {
    for (int s2 = 0; s2 < S; ++s2) mbar_inval(&sm.full[s2]);
    for (int b = 0; b < 2; ++b) {
      mbar_inval(&sm.bready[b]);
      mbar_inval(&sm.yready[b]);
      mbar_inval(&sm.xbar[b]);
    }
  }
  if (C > 1) cluster.sync();
}

// ---------------------------------------------------------------------------
// Statistics record of iterate t (Sec. 5.1 KKT error with r = max(graX, 0),
// s = max(graY, 0), 2-norms; f from the Grams) from the Y-half terms (this
// sweep's M pass) and the X-half terms (the row pass that produced X_t).
// ---------------------------------------------------------------------------
// Called by the 32 lanes of one warp: the six square roots and three quotients run on
// separate lanes (each FP64 warp instruction costs the same whatever the
// number of active lanes); lane 0 writes out[].  dx2 < 0: no step term.
// sqrt(x) and a / b to ~2^-23 relative: the significands in FP32, the
// binary exponents exactly (FP64 square roots and divisions are chains of
// ~20 dependent FP64 instructions on this part, and these ratios and norms
// of the statistics record need 7 digits at most).  Outside the normal FP64
// range, for non-positive or non-finite arguments, the FP64 operation.
__device__ __forceinline__ bool normal_pos(double x, int& e, double& m) {
  const long long b = __double_as_longlong(x);
  const int be = (int)((b >> 52) & 0x7ff);
  if (b <= 0 || be == 0 || be >= 2046) return false;   // <= 0, denormal, huge, inf or NaN
  e = be - 1023;
  m = __longlong_as_double((b & 0x000FFFFFFFFFFFFFll) | (1023ll << 52));   // [1, 2)
  return true;
}
__device__ __forceinline__ double scale2(double v, int e) {   // v * 2^e for a normal result
  return __longlong_as_double(__double_as_longlong(v) + ((long long)e << 52));
}
__device__ __forceinline__ double sqrt_f32(double x) {
  int e;
  double m;
  if (!normal_pos(x, e, m)) return sqrt(x);
  if (e & 1) {   // make the exponent even: m in [2, 4)
    m *= 2.0;
    e -= 1;
  }
  return scale2((double)sqrtf((float)m), e / 2);
}
__device__ __forceinline__ double div_f32(double a, double b) {
  int ea, eb;
  double ma, mb;
  if (!normal_pos(a, ea, ma) || !normal_pos(b, eb, mb)) return a / b;
  return scale2((double)__fdiv_rn((float)ma, (float)mb), ea - eb);
}

__device__ inline void combine_stats_warp(const double* yterm, const double* xterm, double msq,
                                          double dx2, int iter, int fp64, double* out) {
  const int lane = threadIdx.x & 31;
  const double neg = yterm[YT_NEG] + xterm[XT_NEG];
  const double comp = yterm[YT_COMP] + xterm[XT_COMP];
  double arg = 0.0;
  if (lane == 0) arg = neg;
  else if (lane == 1) arg = comp;
  else if (lane == 2) arg = xterm[XT_PNORM2];
  else if (lane == 3) arg = yterm[YT_BNORM2];
  else if (lane == 4) arg = dx2 >= 0.0 ? dx2 + yterm[YT_DY2] : 0.0;
  else if (lane == 5) arg = xterm[XT_XNORM2] + yterm[YT_YNORM2];
  const double sq = arg > 0.0 ? sqrt_f32(arg) : 0.0;
  const double e1 = __shfl_sync(0xffffffffu, sq, 0), e2 = __shfl_sync(0xffffffffu, sq, 1);
  const double sg = __shfl_sync(0xffffffffu, sq, 2) + __shfl_sync(0xffffffffu, sq, 3);
  const double s4 = __shfl_sync(0xffffffffu, sq, 4), s5 = __shfl_sync(0xffffffffu, sq, 5);
  const double xymax = fmax(xterm[XT_XMAX], yterm[YT_YMAX]);
  const double d2 = sg * xymax;
  const double num = lane == 0 ? e1 : (lane == 1 ? e2 : s4);
  const double den = lane == 0 ? sg : (lane == 1 ? d2 : 1.0 + s5);
  const double qt = (lane >= 2 || den > 0.0) ? (num > 0.0 ? div_f32(num, den) : 0.0) : num;
  const double r1 = __shfl_sync(0xffffffffu, qt, 0), r2 = __shfl_sync(0xffffffffu, qt, 1);
  const double step = __shfl_sync(0xffffffffu, qt, 2);
  if (lane != 0) return;
  for (int e = 0; e < NSTAT; ++e) out[e] = 0.0;
  out[ST_ITER] = iter;
  out[ST_F] = 0.5 * (msq - 2.0 * yterm[YT_BY] + yterm[YT_YGY]);
  out[ST_EABS] = fmax(e1, e2);
  out[ST_REL] = fmax(r1, r2);
  out[ST_STEP] = (dx2 >= 0.0) ? step : -1.0;
  out[ST_NEG] = e1;
  out[ST_COMP] = e2;
  out[ST_SG] = sg;
  out[ST_XYMAX] = xymax;
  out[ST_CHANGED_COLS] = yterm[YT_CHANGED];
  out[ST_NOTCONV] = yterm[YT_NOTCONV];
  out[ST_ENTER] = yterm[YT_ENTER];
  out[ST_FP64] = fp64;
  out[ST_MSQ] = msq;
  out[ST_VALID] = xterm[XT_VALID];
}

template <int K>
struct XTraits {
  static constexpr int NW = 16;          // warps
  static constexpr int T = NW * 32;
  static constexpr int RB = 32;          // rows per block (lane <-> row)
  static constexpr int NV = K * K + NXT; // Gram partial + X-half terms
  static constexpr int NVC = (NV + 31) / 32;
};

// Sum over p of src[p * stride + e] for e < nval, in a fixed order, with
// short FP64 dependency chains: G threads per value (8 by default) each add
// every G-th term, then a shuffle tree inside the G-lane group.  Called by all T
// threads of the block; writes out[e] (shared memory).  max_e: 1 = max.
template <int T, int G = 8>
__device__ void tree_sum(const double* src, int nparts, size_t stride, int nval, double* out,
                         int max_e) {
  constexpr int VPB = T / G, U = 8;   // U loads in flight per thread
  const int g = threadIdx.x & (G - 1), vi = threadIdx.x / G;
  for (int e0 = 0; e0 < nval; e0 += VPB) {
    const int e = e0 + vi;
    const bool ok = e < nval;
    const bool is_max = ok && e == max_e;
    double r = 0.0;
    for (int q0 = g; q0 < nparts; q0 += G * U) {
      double w[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int q = q0 + u * G;
        w[u] = (ok && q < nparts) ? src[(size_t)q * stride + e] : 0.0;
      }
#pragma unroll
      for (int u = 0; u < U; ++u) r = is_max ? dmax_nn(r, w[u]) : r + w[u];
    }
#pragma unroll
    for (int o = 1; o < G; o <<= 1) {
      const double w = __shfl_xor_sync(0xffffffffu, r, o);
      r = is_max ? dmax_nn(r, w) : r + w;
    }
    if (ok && g == 0) out[e] = r;
  }
}

// Two tree_sum reductions in one pass (values [0, n1) from src1, then
// [n1, n1 + n2) from src2), so that both sets of loads are in flight at
// once; every value is summed in the same order as by tree_sum.
template <int T>
__device__ void tree_sum2(const double* src1, int np1, size_t st1, int n1, double* out1, int max1,
                          const double* src2, int np2, size_t st2, int n2, double* out2, int max2) {
  constexpr int G = 8, VPB = T / G, U = 8;
  const int g = threadIdx.x & (G - 1), vi = threadIdx.x / G;
  for (int e0 = 0; e0 < n1 + n2; e0 += VPB) {
    const int e = e0 + vi;
    const bool ok = e < n1 + n2, first = e < n1;
    const double* src = first ? src1 : src2;
    const int np = first ? np1 : np2, ee = first ? e : e - n1;
    const size_t stride = first ? st1 : st2;
    const bool is_max = ok && ee == (first ? max1 : max2);
    double r = 0.0;
    for (int q0 = g; q0 < (ok ? np : 0); q0 += G * U) {
      double w[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int q = q0 + u * G;
        w[u] = q < np ? src[(size_t)q * stride + ee] : 0.0;
      }
#pragma unroll
      for (int u = 0; u < U; ++u) r = is_max ? dmax_nn(r, w[u]) : r + w[u];
    }
#pragma unroll
    for (int o = 1; o < G; o <<= 1) {
      const double w = __shfl_xor_sync(0xffffffffu, r, o);
      r = is_max ? dmax_nn(r, w) : r + w;
    }
    if (ok && g == 0) (first ? out1 : out2)[ee] = r;
  }
}

// Row pass of an incremental sweep or of the compensated sweep that records
// the references (entry e of row-major X): the FP32 change of the new X
// against the reference X for the next incremental sweep; when recording,
// the reference X (the sweep's input X, whose contractions the M pass just
// recorded) and the reference P (this sweep's P, from the recorded Y).
__device__ __forceinline__ void store_increment_refs(const Problem& p, int nxt, size_t e, double xo, double xn,
                                                     double pr) {
  const double xr = p.record_refs ? xo : p.Xref[e];
  p.Xd32[nxt][e] = __double2float_rn(xn - xr);
  if (p.record_refs) {
    p.Xref[e] = xo;
    p.Pref[e] = pr;
  }
}

// Dynamic shared memory of the row pass: the working arrays, then the
// subset table of H (k <= 8).
template <typename TA, int K>
struct XSmem {
  using Tr = XTraits<K>;
  static constexpr bool TABLE = K <= 8;
  // NNLS warps: k <= 8, lane groups of KP lanes; k = 16, every warp (two rows of 16 lanes)
  static constexpr int NWN = TABLE ? Tr::RB / LaneGroup<K>::CPW : Tr::NW;
  // warps that build the subset table of H: enough lane groups for its
  // largest level (C(k, k/2) subsets), at most half the block
  static constexpr int binom_mid() {
    int v = 1;
    for (int i = 1; i <= K / 2; ++i) v = v * (K - K / 2 + i) / i;
    return v;
  }
  static constexpr int WT_NEED = (binom_mid() * LaneGroup<K>::KP + 31) / 32;
  // k <= 5: the table by independent Gauss-Jordan inversions, every subset
  // in one round (build_subset_table_gj); larger k: level by level
  static constexpr bool GJ = K <= 5;
  static constexpr int WT_GJ = (((1 << K) - 1) * LaneGroup<K>::KP + 31) / 32;
  static constexpr int WT = !TABLE ? 0 : GJ ? WT_GJ
                                            : (WT_NEED < 1 ? 1 : (WT_NEED > Tr::NW / 2 ? Tr::NW / 2 : WT_NEED));
  // value type of the row solves: FP64 in every pass (see YTraits::F32NN)
  static constexpr bool F32NN = false;
  using SV = typename std::conditional<F32NN, float, double>::type;
  // k = 16: value type of the 16-lane row solves (FP64 in every pass: an
  // FP32 solve with its 2^-23 tolerance leaves out variables worth percents
  // of a row where H is ill conditioned)
  using V16 = double;
  // Lawson-Hanson tolerance constant of the FP64 row solves: 2^-52, but 2^-23
  // at rank 16 with FP32 partials (the tensor-core pass: its P carries ~1e-5,
  // and entering decisions below that level would follow the rounding of P);
  // incremental sweeps use 2^-44, as the compensated pass
  static constexpr double EPS =
      (std::is_same<TA, float>::value && K > 8) ? 1.1920928955078125e-07 : 2.220446049250313e-16;
  struct Small {
    double H[K * K];
    double Gs[K * K];
    SV Hn[K * K];                      // H in the solve's type
    TA psum[Tr::NW][Tr::RB][K + 1];   // padded: a lane's K values start on another bank
    double fin[Tr::NV];
    double yfin[NYT];
    double gram_w[NWN][K * K];
    V16 Hp[K][K + 1];                  // k = 16: H, padded rows, in the solves' type
    float HpF[K][K + 1];               // k = 16: H in FP32 (the tensor-core pass's predictor solves)
    double term_w[NWN][16];
    unsigned ticket;
  };
  static constexpr size_t SMALL = (sizeof(Small) + 127) & ~size_t(127);
  static constexpr size_t TAB = TABLE ? (size_t(1) << K) * K * K * sizeof(SV) : 0;
  static constexpr size_t OK = TABLE ? (size_t(1) << K) * sizeof(int) : 0;
  __host__ __device__ static constexpr size_t bytes() { return SMALL + TAB + OK + 16; }
};

// Row pass: rows [32 b, 32 b + 32) of X.  The 16 warps split the cluster
// partials of P = M Y^T (lane <-> row, summed in the partials' own type) and
// build the subset table of H; k <= 8: 32 / CPW warps solve the 32 row NNLS
// problems lane-parallel (lane <-> (row, component)) and form the X-half
// terms and the Gram partial (k = 16: every warp, one row per 16-lane group); the last
// block to finish combines the blocks, forms G = X^T X (and its subset table
// for k = 7, 8), and the statistics of the iterate.
//
// blk: the row block; xsm_raw: XSmem<TA, K>::bytes() of shared memory.
// tail_done (may be null): the block that runs the last-block tail stores
// tail_value there (release) once the tail's results are visible.
template <typename TA, int K>
__device__ __forceinline__ void xpass_body(const Problem& p, int mode, int Q, int nxblk, int blk,
                                           unsigned char* xsm_raw, unsigned* tail_done,
                                           unsigned tail_value) {
  using Tr = XTraits<K>;
  using Xs = XSmem<TA, K>;
  constexpr int T = Tr::T, NW = Tr::NW, RB = Tr::RB, NV = Tr::NV;
  constexpr bool TABLE = Xs::TABLE;
  typename Xs::Small& xs = *reinterpret_cast<typename Xs::Small*>(xsm_raw);
  // tab_global: H and its subset table come from the batch's H stage
  using SV = typename Xs::SV;   // value type of the row solves
  constexpr bool F32NN = Xs::F32NN;
  const bool hglob = TABLE && p.tab_global && mode == MODE_SWEEP;
  SV* tab = hglob ? reinterpret_cast<SV*>(p.Htab) : reinterpret_cast<SV*>(xsm_raw + Xs::SMALL);
  int* tok = hglob ? p.Hok : reinterpret_cast<int*>(xsm_raw + Xs::SMALL + Xs::TAB);
  double* H = xs.H;
  double* Gs = xs.Gs;
  auto& psum = xs.psum;
  double* fin = xs.fin;
  double* yfin = xs.yfin;
  unsigned& ticket = xs.ticket;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  DevState* st = p.st;
  if (st->done) return;
  const int iter = st->iter;
  const int cur = iter & 1, nxt = cur ^ 1;
  const int row0 = blk * RB;
  const int row = row0 + lane;
  const bool active = row < p.n;

  if (hglob) {
    for (int e = tid; e < K * K; e += T) H[e] = p.Hg[e];
  } else {
    // as many threads per value as the block has for K * K values (one load each for ~Q / 32 partials)
    tree_sum<T, (K * K * 32 <= T) ? 32 : ((K * K * 16 <= T) ? 16 : 8)>(p.Hpart, Q, (size_t)K * K, K * K, H, -1);
  }
  // the first wt warps build the subset table of H while the others sum the
  // cluster partials of P
  const int wt = (TABLE && !hglob && mode == MODE_SWEEP) ? Xs::WT : 0;
  const int npw = NW - wt;
  if (wt) __syncthreads();   // H
  if (warp < wt) {
    if constexpr (TABLE) {
      NnlsSolver<K> ts;
      ts.init(H, 2.220446049250313e-16);
      if constexpr (F32NN) {
        for (int e = tid; e < K * K; e += wt * 32) xs.Hn[e] = (SV)H[e];
        named_sync(2, wt * 32);
        build_subset_table_lanes_v<K, SV>(xs.Hn, (SV)ts.pivot_min, tab, tok, 0, wt * 32,
                                          [wt] { named_sync(2, wt * 32); });
      } else if constexpr (Xs::GJ) {
        build_subset_table_gj<K>(H, ts.pivot_min, tab, tok, 0, wt * 32);
      } else {
        build_subset_table_lanes<K>(ts, tab, tok, 0, wt * 32, [wt] { named_sync(2, wt * 32); });
      }
    }
  } else {
    using PO = PartOps<TA>;
    const TA* Pp = static_cast<const TA*>(p.Ppart);
    const int pw = warp - wt;
    TA acc[K];
#pragma unroll
    for (int a = 0; a < K; ++a) acc[a] = PO::zero();
    if (active)
      for (int q0 = pw; q0 < Q; q0 += npw * 4) {   // four partials in flight per thread
        TA w[4][K];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int qq = q0 + u * npw;
#pragma unroll
          for (int a = 0; a < K; ++a) w[u][a] = qq < Q ? Pp[((size_t)qq * p.ld + row) * K + a] : PO::zero();
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int a = 0; a < K; ++a) acc[a] = PO::add(acc[a], w[u][a]);
      }
#pragma unroll
    for (int a = 0; a < K; ++a) psum[pw][lane][a] = acc[a];
  }
  __syncthreads();
  NnlsSolver<K> solver;
  solver.init(H, 2.220446049250313e-16);

  if constexpr (TABLE) {
    // lanes <-> (row slot jj, component a): warps 0 .. NWN-1 hold the 32 rows
    constexpr int KP = LaneGroup<K>::KP, CPW = LaneGroup<K>::CPW, NWN = RB / CPW;
    auto& gram_w = xs.gram_w;
    auto& term_w = xs.term_w;
    if (warp < NWN) {
      LaneGroup<K> g;
      g.init();
      const int jj = lane / KP;
      const int lrow = warp * CPW + jj, grow_i = row0 + lrow;
      const bool ract = grow_i < p.n;
      const bool ca = g.a < K, comp = ract && ca;
      double hrow[K];
#pragma unroll
      for (int c = 0; c < K; ++c) hrow[c] = ca ? H[g.a * K + c] : 0.0;
      SV hrown[K];
#pragma unroll
      for (int c = 0; c < K; ++c) hrown[c] = (SV)hrow[c];
      double pr = 0.0, xo = 0.0;
      uint32_t old_mask = 0;
      if (comp) {
        TA ts = psum[0][lrow][g.a];
        for (int w = 1; w < npw; ++w) ts = PartOps<TA>::add(ts, psum[w][lrow][g.a]);
        pr = PartOps<TA>::to_double(ts);
        // incremental sweeps: P = Pref + M (Y - Yref)^T
        if (p.inc && mode == MODE_SWEEP) pr += p.Pref[(size_t)grow_i * K + g.a];
        xo = p.X[cur][(size_t)grow_i * K + g.a];
      }
      if (ract) old_mask = p.xmask[cur][grow_i];
      double xn = xo;
      uint32_t msk = 0;
      int stt = 0;
      if (mode == MODE_SWEEP) {
        SV xnv = (SV)xn;
        stt = lane_table_nnls<K, SV>(g, tab, tok, hrown, (SV)solver.gmax,
                                     (SV)(p.inc ? 5.684341886080802e-14 : Xs::EPS), (SV)pr,
                                     xnv, p.warm != 0, ract, true, &msk);
        xn = (double)xnv;
        if (__any_sync(0xffffffffu, stt < 0)) {
          double bb[K], xx[K];
#pragma unroll
          for (int c = 0; c < K; ++c) {
            bb[c] = g.from(pr, c);
            xx[c] = g.from(xo, c);
          }
          uint32_t m2 = 0;
          int s2 = 0;
          if (stt < 0 && g.a == 0) {
            double Ascr[K * K];
            s2 = solver.solve(Ascr, bb, xx, p.warm != 0, nullptr, &m2);
          }
#pragma unroll
          for (int c = 0; c < K; ++c) {
            const double v = __shfl_sync(0xffffffffu, xx[c], g.base);
            if (stt < 0 && g.a == c) xn = v;
          }
          const uint32_t mm = __shfl_sync(0xffffffffu, m2, g.base);
          const int ss = __shfl_sync(0xffffffffu, s2, g.base);
          if (stt < 0) {
            msk = mm;
            stt = ss;
          }
        }
      } else {
        msk = g.bits(comp && dpos(xo));
      }
      // X-half KKT terms of the iterate leaving this sweep: graX = H x - P
      double gx = -pr;
      double xc[K];
#pragma unroll
      for (int c = 0; c < K; ++c) {
        xc[c] = g.from(xn, c);
        gx = fmad(hrow[c], xc[c], gx);
      }
      double tv[16];
#pragma unroll
      for (int e = 0; e < 16; ++e) tv[e] = 0.0;
      if (comp) {
        const double mn = dminz(gx), pos = dmaxz(gx) * xn;
        tv[XT_NEG] = mn * mn;
        tv[XT_COMP] = pos * pos;
        tv[XT_PNORM2] = pr * pr;
        tv[XT_XMAX] = xn;
        tv[XT_XNORM2] = xn * xn;
        tv[XT_DX2] = (xn - xo) * (xn - xo);
        tv[XT_XP] = xn * pr;
        if (!isfinite(pr)) set_err(st, ERR_NONFINITE);
      }
      if (ract && g.a == 0) {
        tv[XT_CHANGED] = (mode == MODE_SWEEP && old_mask != msk) ? 1.0 : 0.0;
        tv[XT_NOTCONV] = (double)stt;
      }
      // Gram partial: row a of x x^T summed over the warp's rows
      double gr[K];
#pragma unroll
      for (int c = 0; c < K; ++c) {
        double v = comp ? xn * xc[c] : 0.0;
#pragma unroll
        for (int o = KP; o < 32; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        gr[c] = v;
      }
      if (lane < KP && ca) {
#pragma unroll
        for (int c = 0; c < K; ++c) gram_w[warp][c * K + g.a] = gr[c];   // G is symmetric: conflict-free order
      }
      const double mx = warp_max(tv[XT_XMAX]);
      tv[XT_XMAX] = 0.0;
      const double tr = warp_reduce_scatter<16, double>(tv);
      if (lane < 16) term_w[warp][lane] = (lane == XT_XMAX) ? mx : tr;
      if (mode == MODE_SWEEP) {
        if (comp) {
          const size_t e = (size_t)grow_i * K + g.a;
          const float hi = __double2float_rn(xn);
          p.X[nxt][e] = xn;
          p.X32[nxt][e] = hi;
          p.X32lo[nxt][e] = __double2float_rn(xn - (double)hi);
          if (p.inc || p.record_refs) store_increment_refs(p, nxt, e, xo, xn, pr);
        }
        if (ract && g.a == 0) p.xmask[nxt][grow_i] = msk;
      } else {
        if (comp) {
          const float hi = __double2float_rn(xo);
          p.X32[cur][(size_t)grow_i * K + g.a] = hi;
          p.X32lo[cur][(size_t)grow_i * K + g.a] = __double2float_rn(xo - (double)hi);
        }
        if (ract && g.a == 0) p.xmask[cur][grow_i] = msk;
      }
    }
    __syncthreads();
    // block partial in fixed order over the warps
    for (int e = tid; e < NV; e += T) {
      double r = 0.0;
      if (e < K * K) {
        for (int w = 0; w < NWN; ++w) r += gram_w[w][e];
      } else {
        const int te = e - K * K;
        for (int w = 0; w < NWN; ++w) r = (te == XT_XMAX) ? dmax_nn(r, term_w[w][te]) : r + term_w[w][te];
      }
      p.Xpart[(size_t)blk * NV + e] = r;
    }
    __threadfence();
  } else {
    // k = 16: lane groups of 16 (lane a <-> component a), one row per group,
    // rows 2 w and 2 w + 1 on warp w; warm-started Lawson-Hanson on the group
    using V16 = typename Xs::V16;
    auto& gram_w = xs.gram_w;
    auto& term_w = xs.term_w;
    for (int e = tid; e < K * K; e += T) {
      xs.Hp[e / K][e % K] = (V16)H[e];
      xs.HpF[e / K][e % K] = (float)H[e];
    }
    __syncthreads();
    const int half = lane >> 4, a = lane & 15;
    const int lrow = warp * 2 + half, grow_i = row0 + lrow;
    const bool ract = grow_i < p.n;   // uniform on the 16 lanes of a row
    const int gbase = lane & 16;
    const unsigned ggm = 0xFFFFu << gbase;
    // the row's right-hand side P_i (+ P_ref in incremental sweeps)
    auto prow = [&](int r) -> double {
      TA ts = psum[0][r][a];
      for (int w = 1; w < npw; ++w) ts = PartOps<TA>::add(ts, psum[w][r][a]);
      double v = PartOps<TA>::to_double(ts);
      if (p.inc && mode == MODE_SWEEP) v += p.Pref[(size_t)(row0 + r) * K + a];
      return v;
    };
    double pr = 0.0, xo = 0.0;
    uint32_t old_mask = 0;
    if (ract) {
      pr = prow(lrow);
      xo = p.X[cur][(size_t)grow_i * K + a];
      old_mask = p.xmask[cur][grow_i];
    }
    double xn = xo;
    uint32_t msk = 0;
    int stt = 0;
    if (ract && mode == MODE_SWEEP) {
      bool done = false;
      bool warm = p.warm != 0;
      if (std::is_same<TA, float>::value) {
        // FP32 partials: the tensor-core pass and the incremental sweeps.  An
        // FP32 solve predicts the passive set (an FP64 solve pays a cold
        // inverse of H_PP per row at ~1/60 of the FP32 rate), FP64-residual
        // refinement gives x, and an FP64 optimality test accepts it;
        // otherwise the FP64 solve continues from the refined x
        LaneNnls16<float> nf;
        // the FP32 solve's tolerance constant: 2^-23 in the tensor-core pass
        // (its P carries ~1e-5), 2^-27 in the incremental sweeps (above the
        // FP32 rounding, close to the FP64 decisions)
        nf.init(xs.HpF, p.inc ? 7.450580596923828e-09f : 1.1920928955078125e-07f);
        double hmax = 0.0;
#pragma unroll
        for (int c = 0; c < K; ++c) hmax = dmax_nn(hmax, dabs(H[c * K + c]));
        done = p.inc ? predict_refine16(nf, H + a * K, hmax, pr, xn, &msk, &stt, warm, 5.684341886080802e-14,
                                        1.4210854715202004e-14, 4, true)
                     : predict_refine16(nf, H + a * K, hmax, pr, xn, &msk, &stt, warm, Xs::EPS,
                                        9.094947017729282e-13, 2, false);
        warm = true;   // a fallback starts from the refined x
      }
      if (!done) {
        LaneNnls16<V16> nn;
        nn.init(xs.Hp, (V16)(p.inc ? 5.684341886080802e-14 : Xs::EPS));
        V16 xv = (V16)xn;
        stt = nn.solve((V16)pr, xv, warm, &msk);
        xn = (double)xv;
      }
    } else if (ract) {
      msk = (__ballot_sync(ggm, dpos(xo)) >> gbase) & 0xFFFFu;
    }
    // X-half KKT terms of the iterate leaving this sweep: graX = H x - P;
    // Gram partial: row a of x x^T
    // components with x_c == 0 add exact zeros: skipped by branches uniform
    // on the group (gx, the row's Gram terms) and on the warp (their sum over
    // the two rows)
    const uint32_t S = (__ballot_sync(ggm, vnz(xn)) >> gbase) & 0xFFFFu;
    double gx = -pr;
    double gr[K];
#pragma unroll
    for (int c = 0; c < K; ++c) {
      gr[c] = 0.0;
      if ((S >> c) & 1u) {
        const double xc = __shfl_sync(ggm, xn, gbase + c);
        gx = fmad(H[a * K + c], xc, gx);
        gr[c] = ract ? xn * xc : 0.0;
      }
    }
    __syncwarp();
    const uint32_t S2 = S | __shfl_xor_sync(0xffffffffu, S, 16);
#pragma unroll
    for (int c = 0; c < K; ++c)
      if ((S2 >> c) & 1u) gr[c] += __shfl_xor_sync(0xffffffffu, gr[c], 16);
    if (lane < 16) {
#pragma unroll
      for (int c = 0; c < K; ++c) gram_w[warp][c * K + a] = gr[c];   // G is symmetric: conflict-free order
    }
    double tv[16];
#pragma unroll
    for (int e = 0; e < 16; ++e) tv[e] = 0.0;
    if (ract) {
      const double mn = dminz(gx), pos = dmaxz(gx) * xn;
      tv[XT_NEG] = mn * mn;
      tv[XT_COMP] = pos * pos;
      tv[XT_PNORM2] = pr * pr;
      tv[XT_XMAX] = xn;
      tv[XT_XNORM2] = xn * xn;
      tv[XT_DX2] = (xn - xo) * (xn - xo);
      tv[XT_XP] = xn * pr;
      if (!isfinite(pr)) set_err(st, ERR_NONFINITE);
      if (a == 0) {
        tv[XT_CHANGED] = (mode == MODE_SWEEP && old_mask != msk) ? 1.0 : 0.0;
        tv[XT_NOTCONV] = (double)stt;
      }
    }
    const double mx = warp_max(tv[XT_XMAX]);
    tv[XT_XMAX] = 0.0;
    const double tr = warp_reduce_scatter<16, double>(tv);
    if (lane < 16) term_w[warp][lane] = (lane == XT_XMAX) ? mx : tr;
    if (ract) {
      const int xb = mode == MODE_SWEEP ? nxt : cur;
      const double xv = mode == MODE_SWEEP ? xn : xo;
      const float hi = __double2float_rn(xv);
      if (mode == MODE_SWEEP) {
        p.X[nxt][(size_t)grow_i * K + a] = xn;
        if (p.inc || p.record_refs) store_increment_refs(p, nxt, (size_t)grow_i * K + a, xo, xn, pr);
      }
      p.X32[xb][(size_t)grow_i * K + a] = hi;
      p.X32lo[xb][(size_t)grow_i * K + a] = __double2float_rn(xv - (double)hi);
      if (a == 0) p.xmask[xb][grow_i] = msk;
    }
    __syncthreads();
    // block partial in fixed order over the warps
    for (int e = tid; e < NV; e += T) {
      double r = 0.0;
      if (e < K * K) {
        for (int w = 0; w < NW; ++w) r += gram_w[w][e];
      } else {
        const int te = e - K * K;
        for (int w = 0; w < NW; ++w) r = (te == XT_XMAX) ? dmax_nn(r, term_w[w][te]) : r + term_w[w][te];
      }
      p.Xpart[(size_t)blk * NV + e] = r;
    }
    __threadfence();
  }
  // last block to finish: G for the next sweep, terms and statistics
  __syncthreads();
  const double* xsrc = p.Xpart;
  int nxsrc = nxblk;
  if (K == 16 && p.xgt && !tail_done) {
    // many blocks of 32 rows: the last block of each group of XGROUP sums its
    // group in block order, and the last group's finisher the group partials
    // in group order (one block summing every block's 272 values in FP64 took
    // ~17 us at n = 8192)
    const int g = blk / XGROUP, b0 = g * XGROUP, b1 = min(nxblk, b0 + XGROUP);
    if (tid == 0) ticket = atomicAdd(&p.xgt[g], 1u);
    __syncthreads();
    if (ticket != (unsigned)(b1 - b0 - 1)) return;
    __threadfence();
    double* grp = p.Xpart + (size_t)nxblk * NV;
    for (int e = tid; e < NV; e += T) {
      const bool is_max = e == K * K + XT_XMAX;
      double r = __ldcg(p.Xpart + (size_t)b0 * NV + e);
      for (int b = b0 + 1; b < b1; ++b) {
        const double w = __ldcg(p.Xpart + (size_t)b * NV + e);
        r = is_max ? dmax_nn(r, w) : r + w;
      }
      grp[(size_t)g * NV + e] = r;
    }
    if (tid == 0) p.xgt[g] = 0u;
    __threadfence();
    __syncthreads();
    xsrc = grp;
    nxsrc = (nxblk + XGROUP - 1) / XGROUP;
  }
  if (tid == 0) ticket = atomicAdd(&st->xblocks_done, 1u);
  __syncthreads();
  if (ticket != (unsigned)(nxsrc - 1)) return;
  __threadfence();
  tree_sum2<T>(xsrc, nxsrc, NV, NV, fin, K * K + XT_XMAX, p.Yterms, Q, NYT, NYT, yfin, YT_YMAX);
  __syncthreads();
  if (tid < K * K) {
    p.G[tid] = fin[tid];
    Gs[tid] = fin[tid];
  }
  __syncthreads();
  // subset table of the new G for the next M pass in global memory: always
  // for k = 7, 8; for k <= 6 with tab_global or gtab_tail (otherwise the M
  // pass builds it).  Warps 1..15 build it while warp 0 forms the statistics.
  const bool gbuilt = TABLE && (K > 6 || p.tab_global || p.gtab_tail);
  double rec[NSTAT];
  if (warp == 0) {
    // the statistics and the record of the iterate (warp 0) while warps 1..15
    // build the table of G: the record does not wait for the table (the next
    // kernel, or the release of the batch's tail flag below, follows both)
    if (mode != MODE_PRIME)
      // statistics of iterate t: Y half from this sweep's M pass, X half from
      // the sweep that produced X_t
      combine_stats_warp(yfin, st->xiter[cur], st->msq, fin[K * K + XT_DX2], iter, p.fp64_pass, rec);
    if (lane == 0) {
      st->gtab_valid = gbuilt ? 1 : 0;
      double xt[NXT];
      for (int e = 0; e < NXT; ++e) xt[e] = fin[K * K + e];
      xt[XT_VALID] = 1.0;
      if (mode == MODE_PRIME) {
        for (int e = 0; e < NXT; ++e) st->xiter[cur][e] = xt[e];
      } else {
        rec[ST_CHANGED_ROWS] = fin[K * K + XT_CHANGED];
        rec[ST_NOTCONV] += fin[K * K + XT_NOTCONV];
        const bool kkt_ok = rec[ST_VALID] > 0.0 && ((p.kkt_target > 0.0 && rec[ST_REL] <= p.kkt_target) ||
                                                    (p.kkt_abs_target > 0.0 && rec[ST_EABS] <= p.kkt_abs_target));
        const bool step_ok = p.stol > 0.0 && rec[ST_STEP] >= 0.0 && rec[ST_STEP] <= p.stol;
        if (kkt_ok) {
          st->done = 1;
          st->stop_reason = 1;
        } else {
          st->iter = iter + 1;
          if (step_ok) {
            st->done = 1;
            st->stop_reason = 2;
          }
        }
        for (int e = 0; e < NSTAT; ++e) st->stats[iter % STAT_CAP][e] = rec[e];
        for (int e = 0; e < NXT; ++e) st->xiter[nxt][e] = xt[e];
        if (p.fp64_pass) ++st->fp64_sweeps;
        if (p.auto_mixed && st->pass_var != VAR_DF && rec[ST_VALID] > 0.0) {
          const double rel = rec[ST_REL];
          if (st->best_rel <= 0.0 || rel < 0.98 * st->best_rel) {   // <= 0: none yet
            st->best_rel = rel;
            st->since_best = 0;
          } else {
            ++st->since_best;
          }
          if (rel <= p.mixed_switch || st->since_best >= p.stall_sweeps) st->pass_var = VAR_DF;
        }
      }
      st->xblocks_done = 0;
    }
  } else {
    if constexpr (TABLE) {
      if (gbuilt) {
        NnlsSolver<K> gs;
        gs.init(Gs, 2.220446049250313e-16);
        // level by level: the warps without a subset of a level skip its
        // arithmetic, so the FP64 pipe stays free for the statistics on warp 0
        build_subset_table_lanes<K>(gs, p.Gtab, p.Gok, 32, T - 32, [] { named_sync(3, T - 32); });
      }
    }
  }
  if (tail_done) {
    __syncthreads();
    if (tid == 0) {
      __threadfence();
      st_release_u32(tail_done, tail_value);
    }
  }
}

// H stage of problem p after its M pass (k <= 8): H = Y Y^T from the Q
// cluster partials (the same fixed-order tree as the row pass), and its
// subset table, into the problem's global buffers; every row block of the
// sweep then reads them instead of forming them itself.  All 512 threads of
// the batch item that completes the problem's M pass.  (The one-problem
// sweep does not use it: its row blocks form the table while their other
// warps sum the P partials, which hides it, whereas a stage at the end of
// the M pass adds its FP64 chains to the sweep's critical path.)
// The table is in the value type of the sweep's row solves (NV: FP32 for the
// FP32 pass), stored in the problem's table buffer.
template <int K, typename NV>
__device__ void h_stage(const Problem& p, int Q, unsigned char* smem_raw) {
  double* H = reinterpret_cast<double*>(smem_raw);
  NV* Hn = reinterpret_cast<NV*>(smem_raw + 2048);
  tree_sum<512>(p.Hpart, Q, (size_t)K * K, K * K, H, -1);
  __syncthreads();
  for (int e = threadIdx.x; e < K * K; e += 512) {
    p.Hg[e] = H[e];
    Hn[e] = (NV)H[e];
  }
  __syncthreads();
  NnlsSolver<K> solver;
  solver.init(H, 2.220446049250313e-16);
  build_subset_table_lanes_v<K, NV>(Hn, (NV)solver.pivot_min, reinterpret_cast<NV*>(p.Htab), p.Hok, 0, 512,
                                    [] { __syncthreads(); });
}

template <typename TM, typename AR, int K>
__global__ void __launch_bounds__(512, 1)
    ypass_kernel(Problem p, int mode, int S, int C, int R, int Q) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  if (p.st->done) return;                     // uniform: written by an earlier launch
  ypass_body<TM, AR, K>(p, mode, S, C, R, Q, (int)blockIdx.x / C, smem_raw);
}

template <typename TA, int K>
__global__ void __launch_bounds__(XTraits<K>::T)
    xpass_kernel(Problem p, int mode, int Q, int nxblk) {
  extern __shared__ __align__(128) unsigned char xsm_raw[];
  xpass_body<TA, K>(p, mode, Q, nxblk, (int)blockIdx.x, xsm_raw, nullptr, 0u);
}

}  // namespace nmfgb

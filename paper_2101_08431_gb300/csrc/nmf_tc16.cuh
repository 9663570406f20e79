// Rank-16 fused M pass on the 5th-generation tensor cores (the FP32-class
// pass of the mixed form at k = 16): for every column j of M,
//   b_j = X^T M_{:,j},  y_j = NNLS(G, b_j)          (Y half, Sec. 2 "qp")
// and, from the same staged tile of M, the X-update accumulation
//   P += M_{:,j} y_j^T,  H += y_j y_j^T             (Sec. 2, C = Y^T).
//
// Precision: M (FP32 in HBM), X and Y are split into BF16 pairs
// v = hi + lo (hi = bf16(v), lo = bf16(v - hi)); both contractions are
// (M_hi + M_lo)(V_hi + V_lo) as BF16 x BF16 products with FP32 accumulation
// in tensor memory.  The column solves run in FP32 (this pass's B is good
// to ~1e-5, far above FP32 rounding of the solve); G, H and the KKT terms
// are FP64.
//
// Partition.  A cluster of C CTAs covers all rows of M: CTA r owns the rows
// [r R, r R + R) (R a multiple of 128).  Cluster q owns a contiguous range
// of columns, processed in tiles of 16.  Per tile and CTA:
//   converter warps  load the tile's rows of M (16-byte loads), split them
//                    into BF16 hi/lo and write the core-matrix layout of a
//                    shared-memory slot;
//   MMA thread       B-MMA: D_B(64 x 32) = [X_hi; X_lo]^T-slab (A, K-major)
//                    x [M_hi | M_lo] (B, K-major), over the CTA's rows;
//   B epilogue       reads D_B (rows 0-15: X_hi, 16-31: X_lo), adds the
//                    four partial products and pushes column j's partial
//                    to the CTA that owns column j (rank j mod C);
//   solve groups     four 16-lane groups (warps 1 and 3) sum the C partials
//                    of their columns in rank order, solve each column with a
//                    warm-started Lawson-Hanson and send y (FP32) to every CTA
//                    of the cluster, then form the KKT terms and H;
//   Y builder        splits the tile's y into the BF16 operand of the P-MMA;
//   MMA thread       P-MMA: D_P(128 x 16 per 128-row chunk) +=
//                    [M_hi, M_lo] (A, M-major) x [Y_hi, Y_lo] (B, K-major);
//                    its completion frees the slot.
// A ring of NS slots holds each converted tile from its B-MMA to its P-MMA,
// so the stream of M continues while the columns of earlier tiles are being
// solved; M is read from HBM exactly once.  The B-MMA uses M = 64 rows of
// which 32 carry X: rows 32-63 read the next core matrices of the slab (whose
// 512-byte zero pad keeps the last K-step's reads in bounds) and are
// discarded.
//
// Every wait is bounded; on a timeout the CTA raises ERR_TIMEOUT, stops its
// loops, drains its MMAs and frees its tensor memory before returning.
#pragma once

#include <cuda_bf16.h>

#include "nmf_nnls.cuh"
#include "nmf_sweep.cuh"
#include "nmf_tc.cuh"
#include "nmf_tc16.h"
#include "nmf_lane16.cuh"

namespace nmfgb {


namespace tc16 {

constexpr int K = 16;
constexpr int TJ = 16;         // columns per tile
constexpr int NT = 512;        // threads per CTA
constexpr int W_MMA = 0, W_NN = 1, W_YB = 2, W_NN2 = 3, W_BE0 = 4, W_BE1 = 5, W_CV0 = 6, NCV = 10;
constexpr int NG = 4;          // column-solve groups (16 lanes each: warps W_NN, W_NN2)
constexpr int NSG_MAX = 24;    // ring entries of a group's received B partials
constexpr int XROWS = 32;      // ring entries x sources of a group (NSG * C)
constexpr int NSMAX = 6;
constexpr int ROW_BYTES = 64;  // per row of M in a slot: 16 columns x (hi, lo) BF16; per row of X: 16 x (hi, lo)
constexpr int AX_PAD = 512;    // the B-MMA's discarded rows read up to 512 bytes past the slab

struct Small {
  uint64_t conv_full[NSMAX];   // slot converted (converter warps -> MMA)
  uint64_t bmma_done[NSMAX];   // B-MMA complete (MMA commit -> B epilogue)
  uint64_t xbarg[NG][NSG_MAX]; // B partials of a group's column received (cluster -> NNLS)
  uint64_t yready[NSMAX];      // y of the tile received (cluster -> Y builder)
  uint64_t yop_ready[NSMAX];   // P-MMA operand built (Y builder -> MMA)
  uint64_t slot_free[NSMAX];   // P-MMA complete (MMA commit -> converters)
  uint64_t pdone;              // every MMA of the pass complete
  uint32_t tmem_base;
  int abort_flag;
  double Gp[K][K + 1];         // G, rows padded against bank conflicts (KKT terms)
  float Gpf[K][K + 1];         // G in the solves' type
  double Hw[2][K * K];         // H over the owned columns, per solve warp
  double Ytw[2][NYT];          // Y-half terms, per solve warp
  uint64_t bs_full[2], bs_free[2];   // X_lo half of the B partial handed between the two epilogue warps
  float bsum[2][TJ][K + 1];    // X_lo half of the B partial (by tile parity)
  float bloc[TJ][K];           // this CTA's B partial, [column][component]
  __align__(16) float xchg[NG][XROWS][K];  // received partials, [group][entry * C + source][component]
  __align__(16) float yraw[NSMAX][TJ][K];   // y of each tile column (FP32)
  __align__(128) unsigned char yop[NSMAX][1024];   // P-MMA B operand: Y_hi (512 B), Y_lo (512 B)
};

__host__ __device__ constexpr size_t small_bytes() { return (sizeof(Small) + 1023) / 1024 * 1024; }
__host__ __device__ constexpr size_t ax_bytes(int R) { return ((size_t)R * ROW_BYTES + AX_PAD + 1023) / 1024 * 1024; }
__host__ __device__ constexpr size_t slot_bytes(int R) { return (size_t)R * ROW_BYTES; }

// byte offsets in the core-matrix layouts (no swizzle)
// X slab: K-block kb (8 rows) holds 4 core matrices: hi c0-7, hi c8-15, lo c0-7, lo c8-15
__device__ __forceinline__ int ax_off(int i, int gc) {
  return (i >> 3) * 512 + (gc >> 3) * 128 + (gc & 7) * 16 + (i & 7) * 2;
}
// M slot: row block I holds hi j0-7, hi j8-15, lo j0-7, lo j8-15
__device__ __forceinline__ int sl_off(int I, int h, int j) { return (I * 4 + h * 2 + (j >> 3)) * 128 + (j & 7) * 16; }
// Y operand (K = tile column j, N = component c), K-major
__device__ __forceinline__ int yop_off(int j, int c) { return ((c >> 3) * 2 + (j >> 3)) * 128 + (c & 7) * 16 + (j & 7) * 2; }

__device__ __forceinline__ uint16_t bf16_bits(float f) {
  return __bfloat16_as_ushort(__float2bfloat16_rn(f));
}
__device__ __forceinline__ float bf16_val(uint16_t u) { return __uint_as_float((uint32_t)u << 16); }
// hi/lo split of two FP32 values, packed two BF16 per word
__device__ __forceinline__ void split2(float a, float b, uint32_t& hi, uint32_t& lo) {
  const uint16_t ha = bf16_bits(a), hb = bf16_bits(b);
  const uint16_t la = bf16_bits(a - bf16_val(ha)), lb = bf16_bits(b - bf16_val(hb));
  hi = (uint32_t)ha | ((uint32_t)hb << 16);
  lo = (uint32_t)la | ((uint32_t)lb << 16);
}

// ---------------------------------------------------------------------------
// The kernel
// ---------------------------------------------------------------------------
constexpr unsigned long long WAIT_NS = 2000000000ull;   // bound of every wait: 2 s of wall time

__device__ __forceinline__ unsigned long long gtime() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ bool flag_set(int* flag) { return *reinterpret_cast<volatile int*>(flag) != 0; }
__device__ __forceinline__ bool aborted(Small& sm) { return flag_set(&sm.abort_flag); }
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
__device__ __forceinline__ bool bwait(Small& sm, uint64_t* bar, uint32_t parity) {
  return bwait_flag<false>(&sm.abort_flag, bar, parity);
}
__device__ __forceinline__ bool bwait_cluster(Small& sm, uint64_t* bar, uint32_t parity) {
  return bwait_flag<true>(&sm.abort_flag, bar, parity);
}

__device__ __forceinline__ void st_remote_f32(float* local_addr, int rank, float v) {
  uint32_t ra;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(smem_u32(local_addr)), "r"(rank));
  asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(ra), "f"(v) : "memory");
}
__device__ __forceinline__ void st_remote_v4(float* local_addr, int rank, float4 v) {
  uint32_t ra;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(smem_u32(local_addr)), "r"(rank));
  asm volatile("st.shared::cluster.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(ra), "f"(v.x), "f"(v.y), "f"(v.z),
               "f"(v.w)
               : "memory");
}
__device__ __forceinline__ void fence_acq_rel_cluster() { asm volatile("fence.acq_rel.cluster;" ::: "memory"); }
__device__ __forceinline__ double ld_remote_f64(const double* local_addr, int rank) {
  uint32_t ra;
  double v;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(smem_u32(local_addr)), "r"(rank));
  asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(ra) : "memory");
  return v;
}

__global__ void __launch_bounds__(NT, 1) ypass_tc16_kernel(Problem p, int mode, Tc16Plan L) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  Small& sm = *reinterpret_cast<Small*>(smem_raw);
  unsigned char* ax = smem_raw + small_bytes();
  unsigned char* slots = ax + ax_bytes(L.R);
  cg::cluster_group cluster = cg::this_cluster();
  const int C = L.C, NS = L.NS, R = L.R, Q = L.Q;
  const int crank = (int)cluster.block_rank(), q = (int)blockIdx.x / C;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  DevState* st = p.st;
  if (st->done) return;   // uniform: written by an earlier launch
  const int cur = st->iter & 1, nxt = cur ^ 1;
  const int c0 = (int)(((long long)q * p.m) / Q);
  const int c1 = (int)(((long long)(q + 1) * p.m) / Q);
  const int ncols = c1 - c0;
  const int ntiles = (ncols + TJ - 1) / TJ;
  const int r0 = crank * R;
  const int rows_c = max(0, min(R, p.ld - r0));   // multiple of 32
  const int nown = TJ / C;                        // columns of a tile owned by this CTA
  // column solve items w = tile * nown + owned column, group w % NG; each
  // group receives its items' partials in a ring of NSG entries, deep enough
  // that the sources of item w + NG * NSG can only push after item w is solved
  const int NSG = max(2, (NS * nown + NG - 1) / NG);
  const size_t SB = slot_bytes(R);
  const float* M = static_cast<const float*>(p.M);

  // ---- set-up: barriers, G, the BF16 X slab, tensor memory
  if (tid == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(&sm.conv_full[s], NCV);
      mbar_init(&sm.bmma_done[s], 1);
      mbar_init(&sm.yready[s], TJ);   // one arrival per column of the tile
      mbar_init(&sm.yop_ready[s], 1);
      mbar_init(&sm.slot_free[s], 1);
    }
    mbar_init(&sm.pdone, 1);
    for (int g = 0; g < NG; ++g)
      for (int e = 0; e < NSG; ++e) mbar_init(&sm.xbarg[g][e], (uint32_t)C);
    for (int b = 0; b < 2; ++b) {
      mbar_init(&sm.bs_full[b], 1);
      mbar_init(&sm.bs_free[b], 1);
    }
    sm.abort_flag = 0;
    fence_mbar_init();
  }
  for (int e = tid; e < K * K; e += NT) {
    sm.Gp[e / K][e % K] = p.G[e];
    sm.Gpf[e / K][e % K] = (float)p.G[e];
    sm.Hw[0][e] = sm.Hw[1][e] = 0.0;
  }
  for (int e = tid; e < NYT; e += NT) sm.Ytw[0][e] = sm.Ytw[1][e] = 0.0;
  for (int e = tid; e < R * K; e += NT) {
    const int i = e / K, c = e % K, row = r0 + i;
    const float x = (i < rows_c && row < p.n) ? (float)p.X[cur][(size_t)row * K + c] : 0.f;
    const uint16_t h = bf16_bits(x);
    const double xd = (i < rows_c && row < p.n) ? p.X[cur][(size_t)row * K + c] : 0.0;
    const uint16_t l = bf16_bits((float)(xd - (double)bf16_val(h)));
    *reinterpret_cast<uint16_t*>(ax + ax_off(i, c)) = h;
    *reinterpret_cast<uint16_t*>(ax + ax_off(i, 16 + c)) = l;
  }
  for (int e = tid; e < AX_PAD / 4; e += NT) reinterpret_cast<uint32_t*>(ax + (size_t)R * ROW_BYTES)[e] = 0u;
  if (warp == W_MMA) {
    tc::alloc(&sm.tmem_base, (uint32_t)L.tmem_cols);
    tc::relinquish();
  }
  tc::fence_proxy_async();
  tc::fence_before_sync();
  cluster.sync();   // every CTA's barriers exist before any remote arrival
  tc::fence_after_sync();
  const uint32_t tmem = sm.tmem_base;
  const uint32_t tm_P = tmem + (uint32_t)NS * 32;   // D_P chunks after the NS B accumulators
  const int nch = (rows_c + 127) / 128;
  bool timed_out = false;

  if (warp == W_MMA) {
    // ======================= MMA issue (one thread) =========================
    if (lane == 0) {
      const uint32_t idB = tc::idesc_bf16(64, 32, false, false);
      const uint32_t idP = tc::idesc_bf16(128, 16, true, false);
      const uint32_t axa = smem_u32(ax), sla = smem_u32(slots), ya = smem_u32(&sm.yop[0][0]);
      const int nks = rows_c / 16;
      int nb = 0, np = 0;
      unsigned idle = 0;
      unsigned long long t_idle = gtime();
      while (np < ntiles) {
        bool prog = false;
        if (nb < ntiles && nb - np < NS) {
          const int s = nb % NS;
          if (mbar_try_wait(&sm.conv_full[s], (uint32_t)((nb / NS) & 1))) {
            tc::fence_after_sync();
            const uint32_t d = tmem + (uint32_t)s * 32;
            for (int ks = 0; ks < nks; ++ks)
              tc::mma_bf16(d, tc::sdesc(axa + ks * 1024, 512, 128),
                           tc::sdesc(sla + (uint32_t)(s * SB) + ks * 1024, 512, 128), idB, ks > 0);
            tc::commit(&sm.bmma_done[s]);
            ++nb;
            prog = true;
          }
        }
        if (np < nb) {
          const int s = np % NS;
          if (mbar_try_wait(&sm.yop_ready[s], (uint32_t)((np / NS) & 1))) {
            tc::fence_after_sync();
            for (int ch = 0; ch < nch; ++ch)
#pragma unroll
              for (int hy = 0; hy < 4; ++hy) {
                const int h = hy >> 1, yh = hy & 1;
                tc::mma_bf16(tm_P + (uint32_t)ch * 16,
                             tc::sdesc(sla + (uint32_t)(s * SB) + ch * 16 * 512 + h * 256, 128, 512),
                             tc::sdesc(ya + s * 1024 + yh * 512, 128, 256), idP, np > 0 || hy > 0);
              }
            tc::commit(&sm.slot_free[s]);
            ++np;
            prog = true;
          }
        }
        if (prog) {
          idle = 0;
          t_idle = gtime();
        } else if ((++idle & 63) == 0 && (aborted(sm) || gtime() - t_idle > WAIT_NS)) {
          timed_out = true;
          atomicExch(&sm.abort_flag, 1);
          break;
        }
      }
      tc::commit(&sm.pdone);   // arrives once every MMA issued above has completed
    }
    __syncwarp();
  } else if (warp >= W_CV0) {
    // ======================= converter warps ================================
    const int cw = warp - W_CV0;
    const int nI = rows_c / 8;                  // 8-row blocks of this CTA
    const int nitems = (nI + 3) / 4 * 2;        // (4 row blocks x 8 columns) per item
    const int iq = lane >> 3, j8 = lane & 7;
    for (int t = 0; t < ntiles; ++t) {
      const int s = t % NS;
      if (t >= NS && !bwait(sm, &sm.slot_free[s], (uint32_t)(((t / NS) - 1) & 1))) {
        timed_out = true;
        break;
      }
      if (aborted(sm)) break;
      tc::fence_proxy_async();   // the tensor core's reads of this slot precede the rewrite
      unsigned char* slot = slots + s * SB;
      for (int it0 = cw; it0 < nitems; it0 += 4 * NCV) {
        float4 v[4][2];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int it = it0 + u * NCV;
          const int I = (it >> 1) * 4 + iq, j = (it & 1) * 8 + j8, col = t * TJ + j;
          v[u][0] = v[u][1] = make_float4(0.f, 0.f, 0.f, 0.f);
          if (it < nitems && I < nI && col < ncols) {
            const int phys = wrap_col(p.head, c0 + col, p.mcap);
            const float4* src = reinterpret_cast<const float4*>(M + (size_t)phys * p.ld + r0 + I * 8);
            v[u][0] = __ldg(src);
            v[u][1] = __ldg(src + 1);
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int it = it0 + u * NCV;
          const int I = (it >> 1) * 4 + iq, j = (it & 1) * 8 + j8;
          if (it < nitems && I < nI) {
            uint4 hi, lo;
            split2(v[u][0].x, v[u][0].y, hi.x, lo.x);
            split2(v[u][0].z, v[u][0].w, hi.y, lo.y);
            split2(v[u][1].x, v[u][1].y, hi.z, lo.z);
            split2(v[u][1].z, v[u][1].w, hi.w, lo.w);
            *reinterpret_cast<uint4*>(slot + sl_off(I, 0, j)) = hi;
            *reinterpret_cast<uint4*>(slot + sl_off(I, 1, j)) = lo;
          }
        }
      }
      tc::fence_proxy_async();
      __syncwarp();
      if (lane == 0) mbar_arrive(&sm.conv_full[s]);
    }
  } else if (warp == W_BE0 || warp == W_BE1) {
    // ======================= B epilogue =====================================
    const uint32_t lanebase = (uint32_t)(32 * (warp & 3)) << 16;
    for (int t = 0; t < ntiles; ++t) {
      const int s = t % NS;
      if (!bwait(sm, &sm.bmma_done[s], (uint32_t)((t / NS) & 1))) {
        timed_out = true;
        break;
      }
      tc::fence_after_sync();
      float v0[16], v1[16];
      tc::ld16(tmem + lanebase + (uint32_t)s * 32, v0);        // A_X x M_hi
      tc::ld16(tmem + lanebase + (uint32_t)s * 32 + 16, v1);   // A_X x M_lo
      tc::fence_before_sync();
      const bool have = rows_c > 0;
      const int pb = t & 1;
      if (warp == W_BE1) {
        if (t >= 2 && !bwait(sm, &sm.bs_free[pb], (uint32_t)(((t >> 1) - 1) & 1))) {
          timed_out = true;
          break;
        }
        if (lane < K) {
#pragma unroll
          for (int j = 0; j < TJ; ++j) sm.bsum[pb][j][lane] = have ? v0[j] + v1[j] : 0.f;
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&sm.bs_full[pb]);
      } else {
        if (!bwait(sm, &sm.bs_full[pb], (uint32_t)((t >> 1) & 1))) {
          timed_out = true;
          break;
        }
        if (lane < K) {
#pragma unroll
          for (int j = 0; j < TJ; ++j) sm.bloc[j][lane] = (have ? v0[j] + v1[j] : 0.f) + sm.bsum[pb][j][lane];
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&sm.bs_free[pb]);
        if (lane < TJ) {
          const int owner = lane % C, jl = lane / C;
          const int w = t * nown + jl, g = w % NG, gs = (w / NG) % NSG;
          float* dst = &sm.xchg[g][gs * C + crank][0];
#pragma unroll
          for (int c = 0; c < K; c += 4)
            st_remote_v4(dst + c, owner,
                         make_float4(sm.bloc[lane][c], sm.bloc[lane][c + 1], sm.bloc[lane][c + 2], sm.bloc[lane][c + 3]));
          mbar_arrive_remote(&sm.xbarg[g][gs], (uint32_t)owner);
        }
        __syncwarp();
      }
    }
  } else if (warp == W_NN || warp == W_NN2) {
    // ======================= column solves ==================================
    // FP32 Lawson-Hanson (this pass's B is accurate to ~1e-5, far above FP32
    // rounding of the solve); the KKT terms of the incoming iterate and H in
    // FP64, after y has been sent
    const int half = lane >> 4, a = lane & 15, wi = warp == W_NN2 ? 1 : 0;
    const int gid = 2 * wi + half;
    LaneNnls16<float> nn;
    // the FP32 solve's own tolerance constant, 2^-23 (a finer one would
    // follow the rounding of this FP32 arithmetic and of B)
    nn.init(sm.Gpf, 1.1920928955078125e-07f);
    double acc_t[NYT];
#pragma unroll
    for (int e = 0; e < NYT; ++e) acc_t[e] = 0.0;
    // triangle of H = sum y y^T: lane a accumulates H[a][(a + d) % 16], d = 0..8
    double hacc[9];
#pragma unroll
    for (int d = 0; d < 9; ++d) hacc[d] = 0.0;
    const int nitems = ntiles * nown;
    for (int w = gid; w < nitems; w += NG) {
      const int t = w / nown, jl = w % nown;
      const int jj = crank + jl * C, col = t * TJ + jj;   // tile column, column of the range
      const bool active = col < ncols;
      const int phys = active ? wrap_col(p.head, c0 + col, p.mcap) : 0;
      const double yo = active ? p.Y[cur][(size_t)phys * K + a] : 0.0;   // in flight during the wait
      const uint32_t om = active ? p.ymask[cur][phys] : 0u;
      const int gi = w / NG, gs = gi % NSG;
      if (!bwait_cluster(sm, &sm.xbarg[gid][gs], (uint32_t)((gi / NSG) & 1))) {
        timed_out = true;
        break;
      }
      // the C partials in rank order, four FP32 chains (the partials are FP32
      // tensor-core sums; this sum adds no error beyond theirs)
      float b4[4] = {0.f, 0.f, 0.f, 0.f};
      for (int src = 0; src < C; ++src) b4[src & 3] += sm.xchg[gid][gs * C + src][a];
      const double bd = (double)((b4[0] + b4[1]) + (b4[2] + b4[3]));
      double yn = yo;
      uint32_t msk = 0;
      int stt = 0;
      if (mode == MODE_SWEEP) {
        float y32 = (float)yo;
        stt = nn.solve((float)bd, y32, p.warm != 0, &msk);
        yn = (double)y32;
      }
      if (!active) yn = 0.0;
      // y to every CTA of the cluster: each lane stores its component
      // everywhere and fences once; then lane r alone signals CTA r
      const int s = t % NS;
      const float ys = (float)yn;
      for (int r = 0; r < C; ++r) st_remote_f32(&sm.yraw[s][jj][a], r, ys);
      fence_acq_rel_cluster();
      __syncwarp(nn.gm);
      if (a < C) mbar_arrive_remote(&sm.yready[s], (uint32_t)a);
      if (!active) continue;
      if (mode != MODE_PRIME) {
        // Y-half KKT terms of the incoming iterate: g = G yo - b (component a)
        double gy = -bd;
#pragma unroll
        for (int c = 0; c < K; ++c) gy = fmad(sm.Gp[a][c], __shfl_sync(nn.gm, yo, nn.base + c), gy);
        const double mn = dminz(gy), pos = dmaxz(gy) * yo;
        acc_t[YT_NEG] = fmad(mn, mn, acc_t[YT_NEG]);
        acc_t[YT_COMP] = fmad(pos, pos, acc_t[YT_COMP]);
        acc_t[YT_BNORM2] = fmad(bd, bd, acc_t[YT_BNORM2]);
        acc_t[YT_BY] = fmad(bd, yo, acc_t[YT_BY]);
        acc_t[YT_YGY] = fmad(yo, gy + bd, acc_t[YT_YGY]);
        acc_t[YT_YMAX] = dmax_nn(acc_t[YT_YMAX], yo);
        acc_t[YT_YNORM2] = fmad(yo, yo, acc_t[YT_YNORM2]);
        if (!isfinite(bd)) set_err(st, ERR_NONFINITE);
      }
      if (mode == MODE_SWEEP) {
        acc_t[YT_DY2] = fmad(yn - yo, yn - yo, acc_t[YT_DY2]);
        if (a == 0) {
          acc_t[YT_CHANGED] += (om != msk) ? 1.0 : 0.0;
          acc_t[YT_NOTCONV] += (double)stt;
        }
        p.Y[nxt][(size_t)phys * K + a] = yn;
        if (a == 0) p.ymask[nxt][phys] = msk;
      } else if (mode == MODE_PRIME) {
        const uint32_t pm = (__ballot_sync(nn.gm, dpos(yo)) >> nn.base) & 0xFFFFu;
        if (a == 0) p.ymask[cur][phys] = pm;
      }
      if (mode != MODE_KKT) {
#pragma unroll
        for (int d = 0; d < 9; ++d) {
          const double yc = __shfl_sync(nn.gm, yn, nn.base + ((a + d) & 15));
          hacc[d] = fmad(yn, yc, hacc[d]);
        }
      }
      if (aborted(sm)) break;
    }
    // this warp's H (fixed order: the two halves, then the triangle entries)
    __syncwarp();
#pragma unroll
    for (int d = 0; d < 9; ++d) hacc[d] += __shfl_xor_sync(0xffffffffu, hacc[d], 16);
    if (half == 0) {
#pragma unroll
      for (int d = 0; d < 9; ++d) {
        const int c = (a + d) & 15;
        if (d < 8 || a < 8) {
          sm.Hw[wi][a * K + c] = hacc[d];
          sm.Hw[wi][c * K + a] = hacc[d];
        }
      }
    }
#pragma unroll
    for (int e = 0; e < NYT; ++e) {
      const double v = (e == YT_YMAX) ? warp_max(acc_t[e]) : warp_sum(acc_t[e]);
      if (lane == 0) sm.Ytw[wi][e] = v;
    }
  } else if (warp == W_YB) {
    // ======================= P-MMA operand builder ==========================
    for (int t = 0; t < ntiles; ++t) {
      const int s = t % NS;
      if (!bwait_cluster(sm, &sm.yready[s], (uint32_t)((t / NS) & 1))) {
        timed_out = true;
        break;
      }
      for (int e = lane; e < TJ * K; e += 32) {
        const int j = e / K, c = e % K;
        const float y = sm.yraw[s][j][c];
        const uint16_t h = bf16_bits(y);
        const uint16_t l = bf16_bits(y - bf16_val(h));
        *reinterpret_cast<uint16_t*>(&sm.yop[s][yop_off(j, c)]) = h;
        *reinterpret_cast<uint16_t*>(&sm.yop[s][512 + yop_off(j, c)]) = l;
      }
      tc::fence_proxy_async();
      __syncwarp();
      if (lane == 0) mbar_arrive(&sm.yop_ready[s]);
    }
  }

  // ---- epilogue: P partial of this CTA's rows (warps 4-7 cover the 4 lane quarters)
  if (warp >= 4 && warp < 8) {
    const bool ok = bwait(sm, &sm.pdone, 0u);
    if (!ok) timed_out = true;
    tc::fence_after_sync();
    float* Pp = static_cast<float*>(p.Ppart);
    for (int ch = 0; ch < nch; ++ch) {
      float v[16];
      tc::ld16(tm_P + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)ch * 16, v);
      const int rl = ch * 128 + 32 * (warp & 3) + lane, row = r0 + rl;
      if (mode != MODE_KKT && rl < rows_c && row < p.n) {
#pragma unroll
        for (int c = 0; c < K; ++c) Pp[((size_t)q * p.ld + row) * K + c] = (ntiles > 0 && ok) ? v[c] : 0.f;
      }
    }
    tc::fence_before_sync();
  }
  if (timed_out) set_err(st, ERR_TIMEOUT);
  __syncthreads();
  cluster.sync();   // every CTA's H and terms are final
  if (crank == 0) {
    if (tid < K * K) {
      double h = 0.0;
      for (int r = 0; r < C; ++r) h += ld_remote_f64(&sm.Hw[0][tid], r) + ld_remote_f64(&sm.Hw[1][tid], r);
      p.Hpart[(size_t)q * K * K + tid] = (mode == MODE_KKT) ? 0.0 : h;
    } else if (tid >= 256 && tid < 256 + NYT) {
      const int e = tid - 256;
      double v = 0.0;
      for (int r = 0; r < C; ++r)
        for (int u = 0; u < 2; ++u) {
          const double w = ld_remote_f64(&sm.Ytw[u][e], r);
          v = (e == YT_YMAX) ? dmax_nn(v, w) : v + w;
        }
      p.Yterms[(size_t)q * NYT + e] = v;
    }
  }
  cluster.sync();   // remote reads done before any CTA leaves
  if (warp == W_MMA) tc::dealloc(tmem, (uint32_t)L.tmem_cols);
  if (tid == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_inval(&sm.conv_full[s]);
      mbar_inval(&sm.bmma_done[s]);
      mbar_inval(&sm.yready[s]);
      mbar_inval(&sm.yop_ready[s]);
      mbar_inval(&sm.slot_free[s]);
    }
    mbar_inval(&sm.pdone);
    for (int g = 0; g < NG; ++g)
      for (int e = 0; e < NSG; ++e) mbar_inval(&sm.xbarg[g][e]);
    for (int b = 0; b < 2; ++b) {
      mbar_inval(&sm.bs_full[b]);
      mbar_inval(&sm.bs_free[b]);
    }
  }
}

}  // namespace tc16


}  // namespace nmfgb

// Rank-16 M pass in three streaming launches (the FP32-class pass of the
// mixed form at k = 16):
//   bgemm   B = X^T M                 split-BF16 tcgen05 MMAs; each CTA streams
//                                     128-column tiles of M over a range of rows
//   solve   y_j = NNLS(G, b_j)        every column on a 16-lane group (Sec. 2,
//           eq. "qp"); the KKT terms of the incoming iterate, H = Y Y^T and
//           the BF16 split of the new Y
//   pgemm   P = M Y^T                 split-BF16 tcgen05 MMAs; each CTA streams
//                                     128-row blocks of M over a range of columns
// M is read twice per sweep instead of once: the single-read form couples
// every 16-column tile to a round trip through a 16-CTA cluster (all row
// partials of B to the column's owner, y back to every CTA) and is paced by
// that latency at ~0.13 of HBM bandwidth; two independent streams run far
// closer to the copy rate.
//
// Precision (as the single-read form): v = hi + lo with hi = bf16(v),
// lo = bf16(v - hi) for M, X and Y; each contraction sums all four products
// hi*hi, hi*lo, lo*hi, lo*lo in FP32 in tensor memory (D += A_hi B + A_lo B
// with B = [V_hi | V_lo]); the column solves run in FP32.
//
// Shared-memory operands use the no-swizzle core-matrix layout (8 x 16-byte
// rows per 128-byte core matrix, nmf_tc.cuh).  A stage of the TMA ring first
// receives FP32 slabs of M (32 rows x the tile's columns, one 2-D tensor
// copy each, 128-byte swizzle so that the converter warps read without bank
// conflicts); the converters read their rows into registers, meet at a named
// barrier and write the BF16 hi/lo operand over the same bytes.  The other
// operand (the split of X or Y, precomputed in global memory in the
// core-matrix layout) is bulk-copied beside it.  Tiles never wrap: the first
// MIRROR columns of the ring are mirrored after its last one, and the tensor
// map covers mcap + MIRROR columns.
//
// Every wait is bounded (2 s of wall time); a role that gives up raises the
// CTA's abort flag, the converters leave together (a barrier with an AND
// reduction), and the CTA waits (bounded) for its copies and MMAs in flight
// and frees its tensor memory before it returns with ERR_TIMEOUT set.
#pragma once

#include "nmf_tc16.cuh"

namespace nmfgb {
namespace tc16s {

using tc16::bf16_bits;
using tc16::bf16_val;
using tc16::gtime;
using tc16::split2;
using tc16::WAIT_NS;

constexpr int K = 16;
// GEMM CTAs: warps 0-3 epilogue (TMEM lane quarters 0-3), 4 producer, 5 MMA
// issue, 6-9 converters; two CTAs per SM (two independent rings)
constexpr int NT = 320;            // threads of the GEMM kernels
constexpr int W_EPI = 0, W_PROD = 4, W_MMA = 5, W_CV = 6, NCV = 4;
constexpr int CV_ITEMS = 1024 / (NCV * 32);   // (column, 8-row group) items per converter thread per chunk
constexpr int NSMAX = 6;
constexpr int CTL_BYTES = 1024;
constexpr int SLAB_ROWS = 32;      // rows of one tensor copy (128 bytes of FP32: the swizzle span)

// B-GEMM stage: 128 columns x up to 64 rows of M (two slabs of 16 KB)
constexpr int BG_COLS = 128, BG_ROWS = 64;
constexpr int BG_SLAB = SLAB_ROWS * 4 * BG_COLS;   // 16384
constexpr int BG_XOFF = 2 * BG_SLAB;               // X operand (64 rows x 32 BF16)
constexpr int BG_STAGE = BG_XOFF + BG_ROWS * 64;   // 36864
constexpr int BG_ALO = BG_COLS * BG_ROWS * 2;      // A_lo after A_hi

// P-GEMM stage: 128 rows x 64 columns of M (four slabs of 8 KB)
constexpr int PG_ROWS = 128, PG_COLS = 64;
constexpr int PG_SLAB = SLAB_ROWS * 4 * PG_COLS;   // 8192
constexpr int PG_YOFF = 4 * PG_SLAB;               // Y operand (64 columns x 32 BF16)
constexpr int PG_STAGE = PG_YOFF + PG_COLS * 64;   // 36864
constexpr int PG_ALO = PG_ROWS * PG_COLS * 2;

constexpr int RED = K * K + NYT;   // per-block partials of the solve kernel: H, Y terms
constexpr int SOLVE_T = 256;       // threads of the solve kernel (16 column groups)
constexpr int RGROUP = 16;         // block partials summed per group before the groups are summed

struct Ctl {
  uint64_t full[NSMAX];    // stage filled (tensor and bulk copies)
  uint64_t conv[NSMAX];    // stage converted (converter warps)
  uint64_t freed[NSMAX];   // stage's MMAs complete (commit)
  uint64_t acc_full[2];    // accumulator complete (commit)
  uint64_t acc_free[2];    // accumulator read (epilogue warps)
  uint64_t drain;          // every MMA of the CTA complete
  uint32_t tmem_base;
  int abort_flag;
};
static_assert(sizeof(Ctl) <= CTL_BYTES, "control block");
static_assert(CV_ITEMS == 8, "converter maps: 4 warps x 8 items x 32 lanes = 128 columns x 8 row groups");

// byte offset of (row or column index i, operand column n in 0..31) in the
// split operands of X (i = row) and Y (i = window column): 8 indices x 32
// operand columns per 512-byte block, K-major core matrices
__host__ __device__ __forceinline__ int xs_off(int i, int n) {
  return (i >> 3) * 512 + (n >> 3) * 128 + (n & 7) * 16 + (i & 7) * 2;
}
// byte offset of the 16-byte chunk c (rows 4c .. 4c+3) of column j in a slab
// written with the 128-byte swizzle (1024-byte aligned slab)
__host__ __device__ __forceinline__ int swz(int j, int c) { return j * 128 + ((c ^ (j & 7)) << 4); }

// 2-D tensor copy global -> shared (the TMA engine): the box of the map at
// element coordinates (x = row, y = column), completion in bytes on bar
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ bool timed_wait(uint64_t* bar, uint32_t parity, unsigned long long limit_ns) {
  const unsigned long long t0 = gtime();
  for (unsigned i = 0;; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 63) == 63 && gtime() - t0 > limit_ns) return false;
  }
}
// wait of one lane, result broadcast to the warp
__device__ __forceinline__ bool warp_wait(Ctl& sm, uint64_t* bar, uint32_t parity) {
  bool ok = true;
  if ((threadIdx.x & 31) == 0) ok = tc16::bwait_flag<false>(&sm.abort_flag, bar, parity);
  return __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
}
// barrier over `count` threads with an AND of v
__device__ __forceinline__ bool named_and(int id, int count, bool v) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 q, %1, 0;\n\t"
      "bar.red.and.pred p, %2, %3, q;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(r)
      : "r"(v ? 1u : 0u), "r"(id), "r"(count)
      : "memory");
  return r != 0;
}

__device__ __forceinline__ void ctl_init(Ctl& sm, int NS) {
  for (int s = 0; s < NS; ++s) {
    mbar_init(&sm.full[s], 1);
    mbar_init(&sm.conv[s], NCV);
    mbar_init(&sm.freed[s], 1);
  }
  for (int b = 0; b < 2; ++b) {
    mbar_init(&sm.acc_full[b], 1);
    mbar_init(&sm.acc_free[b], 4);
  }
  mbar_init(&sm.drain, 1);
  sm.abort_flag = 0;
  fence_mbar_init();
}
__device__ __forceinline__ void ctl_inval(Ctl& sm, int NS) {
  for (int s = 0; s < NS; ++s) {
    mbar_inval(&sm.full[s]);
    mbar_inval(&sm.conv[s]);
    mbar_inval(&sm.freed[s]);
  }
  for (int b = 0; b < 2; ++b) {
    mbar_inval(&sm.acc_full[b]);
    mbar_inval(&sm.acc_free[b]);
  }
  mbar_inval(&sm.drain);
}

// The copies a producer issued into stages that nobody consumed (after a
// timeout) still land: wait for the last min(NS, issued) fills (bounded).
__device__ __forceinline__ void drain_fills(Ctl& sm, int NS, int issued) {
  for (int g = issued - NS; g < issued; ++g)
    if (g >= 0) timed_wait(&sm.full[g % NS], (uint32_t)((g / NS) & 1), WAIT_NS);
}

// Sum over the grid of the solve kernels' block partials (RED doubles per
// block at red + block * RED, written by this block before the call), in a
// fixed order whatever the order in which blocks finish: the last block of
// each group of RGROUP consecutive blocks (ticket 1 + group) sums its group
// in block order into a group partial, the last group to finish (ticket 0)
// sums the group partials in group order.  Returns the totals (RED doubles)
// in the one block that finishes, nullptr in every other block; each thread
// of the finishing block owns the entries e = tid (mod blockDim.x) it wrote.
// The tickets reset themselves.  Against one last block summing every block,
// the tail on one SM is ~RGROUP + grid / RGROUP FP64 adds per entry instead
// of grid adds (each FP64 warp instruction holds a sub-partition's unit for
// tens of cycles on this part).
__device__ __forceinline__ const double* reduce_blocks(const Bufs& bf, unsigned* s_last) {
  const int tid = threadIdx.x, nb = (int)gridDim.x;
  const int g = (int)blockIdx.x / RGROUP, ng = (nb + RGROUP - 1) / RGROUP;
  const int b0 = g * RGROUP, b1 = min(nb, b0 + RGROUP);
  double* grp = bf.red + (size_t)nb * RED;   // ng group partials, then the totals
  __threadfence();
  __syncthreads();
  if (tid == 0) *s_last = (atomicAdd(&bf.ticket[1 + g], 1u) == (unsigned)(b1 - b0 - 1)) ? 1u : 0u;
  __syncthreads();
  if (!*s_last) return nullptr;
  __threadfence();
  for (int e = tid; e < RED; e += blockDim.x) {
    double v = __ldcg(bf.red + (size_t)b0 * RED + e);
    for (int b = b0 + 1; b < b1; ++b) {
      const double w = __ldcg(bf.red + (size_t)b * RED + e);
      v = (e == K * K + YT_YMAX) ? dmax_nn(v, w) : v + w;
    }
    grp[(size_t)g * RED + e] = v;
  }
  if (tid == 0) bf.ticket[1 + g] = 0u;
  __threadfence();
  __syncthreads();
  if (tid == 0) *s_last = (atomicAdd(&bf.ticket[0], 1u) == (unsigned)(ng - 1)) ? 1u : 0u;
  __syncthreads();
  if (!*s_last) return nullptr;
  __threadfence();
  double* tot = grp + (size_t)ng * RED;
  for (int e = tid; e < RED; e += blockDim.x) {
    double v = __ldcg(grp + e);
    for (int q = 1; q < ng; ++q) {
      const double w = __ldcg(grp + (size_t)q * RED + e);
      v = (e == K * K + YT_YMAX) ? dmax_nn(v, w) : v + w;
    }
    tot[e] = v;
  }
  if (tid == 0) bf.ticket[0] = 0u;
  return tot;
}

// Knuth's two-sum: s + e == a + b exactly (round to nearest, no reassociation)
__host__ __device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bp = s - a;
  e = (a - (s - bp)) + (b - bp);
}
// float-float accumulation (s, c) += (x, y): the rounding error of each FP32
// add is carried in c, so sums of a few hundred terms keep FP64-class accuracy
// with FP32 instructions only
__host__ __device__ __forceinline__ void ff_add(float& s, float& c, float x, float y) {
  float t, e;
  two_sum(s, x, t, e);
  s = t;
  c += e + y;
}

// ---------------------------------------------------------------------------
// split of X into the B-GEMM's operand: [X_hi | X_lo] per row, rows >= n zero
// ---------------------------------------------------------------------------
__global__ void xsplit_kernel(Problem p, Bufs bf) {
  if (p.st->done) return;
  const int cur = p.st->iter & 1;
  const int total = p.ld * K;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const int i = e >> 4, c = e & 15;
    const double x = i < p.n ? p.X[cur][(size_t)i * K + c] : 0.0;
    const uint16_t h = bf16_bits((float)x);
    const uint16_t l = bf16_bits((float)(x - (double)bf16_val(h)));
    *reinterpret_cast<uint16_t*>(bf.Xs + xs_off(i, c)) = h;
    *reinterpret_cast<uint16_t*>(bf.Xs + xs_off(i, K + c)) = l;
  }
}

// ---------------------------------------------------------------------------
// B-GEMM: B_j = X^T M_{:,j}.  Unit u = (tile u / SB of 128 window columns,
// row split u % SB); D (128 columns x 32) = sum over the split's rows of
// (M_hi + M_lo)^T [X_hi | X_lo]; B_j = D[j][0:16] + D[j][16:32] goes to
// Bpart[split][j].
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ void bg_unit(const Problem& p, int SB, int u, int& tile, int& split, int& r0,
                                                 int& r1) {
  const int ngran = p.ld / 32;
  tile = u / SB;
  split = u % SB;
  r0 = (int)(((long long)split * ngran) / SB) * 32;
  r1 = (int)(((long long)(split + 1) * ngran) / SB) * 32;
}

__global__ void __launch_bounds__(NT, 2) bgemm_kernel(const __grid_constant__ CUtensorMap tmap, Problem p, Bufs bf,
                                                      Plan L) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  Ctl& sm = *reinterpret_cast<Ctl*>(smem_raw);
  unsigned char* stages = smem_raw + CTL_BYTES;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  DevState* st = p.st;
  if (st->done) return;   // uniform: written by an earlier launch
  if (smem_u32(smem_raw) & 1023u) {   // the swizzled slabs need 1024-byte alignment
    if (tid == 0) set_err(st, ERR_CONFIG);
    return;
  }
  const int NS = L.NSB, SB = L.SB;
  const int ncols = p.m;
  const int nunits = ((ncols + BG_COLS - 1) / BG_COLS) * SB;
  if (tid == 0) ctl_init(sm, NS);
  if (warp == W_MMA) {
    tc::alloc(&sm.tmem_base, 64);
    tc::relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = sm.tmem_base;
  bool timed_out = false;
  int issued = 0;

  if (warp == W_PROD) {
    // ======================= tensor copies ==================================
    int gc = 0;
    for (int u = blockIdx.x; u < nunits && !timed_out; u += gridDim.x) {
      int tile, split, r0, r1;
      bg_unit(p, SB, u, tile, split, r0, r1);
      const int p0 = wrap_col(p.head, tile * BG_COLS, p.mcap);   // + up to 127 mirrored columns
      for (int rc = r0; rc < r1; rc += BG_ROWS, ++gc) {
        const int rows = min(BG_ROWS, r1 - rc);
        const int s = gc % NS;
        if (gc >= NS && !warp_wait(sm, &sm.freed[s], (uint32_t)(((gc / NS) - 1) & 1))) {
          timed_out = true;
          break;
        }
        unsigned char* stg = stages + (size_t)s * BG_STAGE;
        if (lane == 0) {
          const int nslab = rows / SLAB_ROWS;
          mbar_arrive_expect_tx(&sm.full[s], (uint32_t)(nslab * BG_SLAB + rows * 64));
          for (int h = 0; h < nslab; ++h) tma_load_2d(stg + h * BG_SLAB, &tmap, rc + h * SLAB_ROWS, p0, &sm.full[s]);
          bulk_g2s(stg + BG_XOFF, bf.Xs + (size_t)rc * 64, (uint32_t)(rows * 64), &sm.full[s]);
        }
        __syncwarp();
        issued = gc + 1;
      }
    }
  } else if (warp == W_MMA) {
    // ======================= MMA issue (one thread) =========================
    if (lane == 0) {
      const uint32_t idB = tc::idesc_bf16(128, 32, false, false);
      const uint32_t sa = smem_u32(stages);
      int gc = 0, ul = 0;
      for (int u = blockIdx.x; u < nunits && !timed_out; u += gridDim.x, ++ul) {
        int tile, split, r0, r1;
        bg_unit(p, SB, u, tile, split, r0, r1);
        const int buf = ul & 1;
        if (ul >= 2 &&
            !tc16::bwait_flag<false>(&sm.abort_flag, &sm.acc_free[buf], (uint32_t)(((ul >> 1) - 1) & 1))) {
          timed_out = true;
          break;
        }
        tc::fence_after_sync();
        const uint32_t d = tmem + (uint32_t)buf * 32;
        bool first = true;
        for (int rc = r0; rc < r1; rc += BG_ROWS, ++gc) {
          const int rows = min(BG_ROWS, r1 - rc);
          const int s = gc % NS;
          if (!tc16::bwait_flag<false>(&sm.abort_flag, &sm.conv[s], (uint32_t)((gc / NS) & 1))) {
            timed_out = true;
            break;
          }
          tc::fence_after_sync();
          const uint32_t a = sa + (uint32_t)(s * BG_STAGE);
          for (int ks = 0; ks < rows / 16; ++ks) {
            const uint64_t bd = tc::sdesc(a + BG_XOFF + ks * 1024, 512, 128);
            tc::mma_bf16(d, tc::sdesc(a + ks * 4096, 2048, 128), bd, idB, !first);
            tc::mma_bf16(d, tc::sdesc(a + BG_ALO + ks * 4096, 2048, 128), bd, idB, true);
            first = false;
          }
          tc::commit(&sm.freed[s]);
        }
        if (timed_out) break;
        tc::commit(&sm.acc_full[buf]);
      }
      tc::commit(&sm.drain);   // arrives once every MMA issued above has completed
    }
    __syncwarp();
  } else if (warp >= W_EPI && warp < W_EPI + 4) {
    // ======================= epilogue: D -> B partials ======================
    const int e = warp - W_EPI;
    int ul = 0;
    for (int u = blockIdx.x; u < nunits; u += gridDim.x, ++ul) {
      int tile, split, r0, r1;
      bg_unit(p, SB, u, tile, split, r0, r1);
      const int buf = ul & 1;
      if (!warp_wait(sm, &sm.acc_full[buf], (uint32_t)((ul >> 1) & 1))) {
        timed_out = true;
        break;
      }
      tc::fence_after_sync();
      float v0[16], v1[16];
      const uint32_t ta = tmem + ((uint32_t)(32 * e) << 16) + (uint32_t)buf * 32;
      tc::ld16(ta, v0);
      tc::ld16(ta + 16, v1);
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) mbar_arrive(&sm.acc_free[buf]);
      const int col = tile * BG_COLS + 32 * e + lane;
      if (col < ncols) {
        const bool have = r1 > r0;
        float4* dst = reinterpret_cast<float4*>(bf.Bpart + ((size_t)split * p.mcap + col) * K);
#pragma unroll
        for (int q = 0; q < 4; ++q)
          dst[q] = have ? make_float4(v0[4 * q] + v1[4 * q], v0[4 * q + 1] + v1[4 * q + 1],
                                      v0[4 * q + 2] + v1[4 * q + 2], v0[4 * q + 3] + v1[4 * q + 3])
                        : make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
  } else if (warp >= W_CV) {
    // ======================= converters: FP32 -> BF16 hi/lo, in place =======
    const int w = warp - W_CV, jl = lane & 7, gq = lane >> 3;
    int gc = 0;
    bool go = true;
    for (int u = blockIdx.x; u < nunits && go; u += gridDim.x) {
      int tile, split, r0, r1;
      bg_unit(p, SB, u, tile, split, r0, r1);
      for (int rc = r0; rc < r1; rc += BG_ROWS, ++gc) {
        const int rows = min(BG_ROWS, r1 - rc);
        const int s = gc % NS;
        const bool ok = warp_wait(sm, &sm.full[s], (uint32_t)((gc / NS) & 1));
        unsigned char* stg = stages + (size_t)s * BG_STAGE;
        const int ng = rows / 8;
        float4 v[CV_ITEMS][2];
#pragma unroll
        for (int uu = 0; uu < CV_ITEMS; ++uu) {
          const int j = 8 * (w + NCV * (uu & 3)) + jl, g = gq + 4 * (uu >> 2);
          v[uu][0] = v[uu][1] = make_float4(0.f, 0.f, 0.f, 0.f);
          if (ok && g < ng) {   // rows 8g .. 8g+7: slab g / 4, chunks 2 (g % 4) and 2 (g % 4) + 1
            const unsigned char* sl = stg + (g >> 2) * BG_SLAB;
            v[uu][0] = *reinterpret_cast<const float4*>(sl + swz(j, 2 * (g & 3)));
            v[uu][1] = *reinterpret_cast<const float4*>(sl + swz(j, 2 * (g & 3) + 1));
          }
        }
        if (!named_and(1, NCV * 32, ok)) {   // every converter leaves at the same stage
          timed_out = true;
          go = false;
          break;
        }
#pragma unroll
        for (int uu = 0; uu < CV_ITEMS; ++uu) {
          const int j = 8 * (w + NCV * (uu & 3)) + jl, g = gq + 4 * (uu >> 2);
          if (g < ng) {
            uint4 hi, lo;
            split2(v[uu][0].x, v[uu][0].y, hi.x, lo.x);
            split2(v[uu][0].z, v[uu][0].w, hi.y, lo.y);
            split2(v[uu][1].x, v[uu][1].y, hi.z, lo.z);
            split2(v[uu][1].z, v[uu][1].w, hi.w, lo.w);
            const int o = g * 2048 + (j >> 3) * 128 + (j & 7) * 16;
            *reinterpret_cast<uint4*>(stg + o) = hi;
            *reinterpret_cast<uint4*>(stg + BG_ALO + o) = lo;
          }
        }
        tc::fence_proxy_async();
        __syncwarp();
        if (lane == 0) mbar_arrive(&sm.conv[s]);
      }
    }
  }

  if (timed_out) {
    atomicExch(&sm.abort_flag, 1);
    set_err(st, ERR_TIMEOUT);
  }
  if (warp == W_PROD && lane == 0) drain_fills(sm, NS, issued);
  __syncthreads();
  if (warp == W_MMA) {
    if (lane == 0) timed_wait(&sm.drain, 0u, WAIT_NS);
    __syncwarp();
    tc::fence_after_sync();
    tc::dealloc(tmem, 64);
  }
  if (tid == 0) ctl_inval(sm, NS);
}

// ---------------------------------------------------------------------------
// P-GEMM: P = M Y^T.  Unit u = (row block u / SP of 128 rows, column split
// u % SP over 64-column granules of the window); D (128 rows x 32) = sum
// over the split's columns of (M_hi + M_lo) [Y_hi | Y_lo];
// P_i = D[i][0:16] + D[i][16:32] goes to Ppart[split][row].
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ void pg_unit(const Problem& p, int SP, int u, int& rb, int& split, int& g0,
                                                 int& g1) {
  const int ncg = (p.m + PG_COLS - 1) / PG_COLS;
  rb = u / SP;
  split = u % SP;
  g0 = (int)(((long long)split * ncg) / SP);
  g1 = (int)(((long long)(split + 1) * ncg) / SP);
}

__global__ void __launch_bounds__(NT, 2) pgemm_kernel(const __grid_constant__ CUtensorMap tmap, Problem p, Bufs bf,
                                                      Plan L) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  Ctl& sm = *reinterpret_cast<Ctl*>(smem_raw);
  unsigned char* stages = smem_raw + CTL_BYTES;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  DevState* st = p.st;
  if (st->done) return;
  if (smem_u32(smem_raw) & 1023u) {
    if (tid == 0) set_err(st, ERR_CONFIG);
    return;
  }
  const int NS = L.NSP, SP = L.SP;
  const int ncols = p.m;
  const int nrb = (p.ld + PG_ROWS - 1) / PG_ROWS;
  const int nunits = nrb * SP;
  if (tid == 0) ctl_init(sm, NS);
  if (warp == W_MMA) {
    tc::alloc(&sm.tmem_base, 64);
    tc::relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = sm.tmem_base;
  bool timed_out = false;
  int issued = 0;

  if (warp == W_PROD) {
    int gc = 0;
    for (int u = blockIdx.x; u < nunits && !timed_out; u += gridDim.x) {
      int rb, split, g0, g1;
      pg_unit(p, SP, u, rb, split, g0, g1);
      const int r0 = rb * PG_ROWS, rows = min(PG_ROWS, p.ld - r0), nslab = rows / SLAB_ROWS;
      for (int g = g0; g < g1; ++g, ++gc) {
        const int s = gc % NS;
        if (gc >= NS && !warp_wait(sm, &sm.freed[s], (uint32_t)(((gc / NS) - 1) & 1))) {
          timed_out = true;
          break;
        }
        unsigned char* stg = stages + (size_t)s * PG_STAGE;
        if (lane == 0) {
          const int p0 = wrap_col(p.head, g * PG_COLS, p.mcap);
          mbar_arrive_expect_tx(&sm.full[s], (uint32_t)(nslab * PG_SLAB + PG_COLS * 64));
          for (int h = 0; h < nslab; ++h) tma_load_2d(stg + h * PG_SLAB, &tmap, r0 + h * SLAB_ROWS, p0, &sm.full[s]);
          bulk_g2s(stg + PG_YOFF, bf.Ys + (size_t)g * PG_COLS * 64, (uint32_t)(PG_COLS * 64), &sm.full[s]);
        }
        __syncwarp();
        issued = gc + 1;
      }
    }
  } else if (warp == W_MMA) {
    if (lane == 0) {
      const uint32_t idP = tc::idesc_bf16(128, 32, true, false);
      const uint32_t sa = smem_u32(stages);
      int gc = 0, ul = 0;
      for (int u = blockIdx.x; u < nunits && !timed_out; u += gridDim.x, ++ul) {
        int rb, split, g0, g1;
        pg_unit(p, SP, u, rb, split, g0, g1);
        const int buf = ul & 1;
        if (ul >= 2 &&
            !tc16::bwait_flag<false>(&sm.abort_flag, &sm.acc_free[buf], (uint32_t)(((ul >> 1) - 1) & 1))) {
          timed_out = true;
          break;
        }
        tc::fence_after_sync();
        const uint32_t d = tmem + (uint32_t)buf * 32;
        bool first = true;
        for (int g = g0; g < g1; ++g, ++gc) {
          const int s = gc % NS;
          if (!tc16::bwait_flag<false>(&sm.abort_flag, &sm.conv[s], (uint32_t)((gc / NS) & 1))) {
            timed_out = true;
            break;
          }
          tc::fence_after_sync();
          const uint32_t a = sa + (uint32_t)(s * PG_STAGE);
#pragma unroll
          for (int ks = 0; ks < PG_COLS / 16; ++ks) {
            const uint64_t bd = tc::sdesc(a + PG_YOFF + ks * 1024, 512, 128);
            tc::mma_bf16(d, tc::sdesc(a + ks * 4096, 128, 256), bd, idP, !first);
            tc::mma_bf16(d, tc::sdesc(a + PG_ALO + ks * 4096, 128, 256), bd, idP, true);
            first = false;
          }
          tc::commit(&sm.freed[s]);
        }
        if (timed_out) break;
        tc::commit(&sm.acc_full[buf]);
      }
      tc::commit(&sm.drain);
    }
    __syncwarp();
  } else if (warp >= W_EPI && warp < W_EPI + 4) {
    const int e = warp - W_EPI;
    float* Pp = static_cast<float*>(p.Ppart);
    int ul = 0;
    for (int u = blockIdx.x; u < nunits; u += gridDim.x, ++ul) {
      int rb, split, g0, g1;
      pg_unit(p, SP, u, rb, split, g0, g1);
      const int buf = ul & 1;
      if (!warp_wait(sm, &sm.acc_full[buf], (uint32_t)((ul >> 1) & 1))) {
        timed_out = true;
        break;
      }
      tc::fence_after_sync();
      float v0[16], v1[16];
      const uint32_t ta = tmem + ((uint32_t)(32 * e) << 16) + (uint32_t)buf * 32;
      tc::ld16(ta, v0);
      tc::ld16(ta + 16, v1);
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) mbar_arrive(&sm.acc_free[buf]);
      const int row = rb * PG_ROWS + 32 * e + lane;
      if (row < p.ld) {
        const bool have = g1 > g0;
        float4* dst = reinterpret_cast<float4*>(Pp + ((size_t)split * p.ld + row) * K);
#pragma unroll
        for (int q = 0; q < 4; ++q)
          dst[q] = have ? make_float4(v0[4 * q] + v1[4 * q], v0[4 * q + 1] + v1[4 * q + 1],
                                      v0[4 * q + 2] + v1[4 * q + 2], v0[4 * q + 3] + v1[4 * q + 3])
                        : make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
  } else if (warp >= W_CV) {
    const int w = warp - W_CV, jl = lane & 7, gq = lane >> 3;
    int gc = 0;
    bool go = true;
    for (int u = blockIdx.x; u < nunits && go; u += gridDim.x) {
      int rb, split, g0, g1;
      pg_unit(p, SP, u, rb, split, g0, g1);
      const int rows = min(PG_ROWS, p.ld - rb * PG_ROWS), ng = rows / 8;
      for (int g = g0; g < g1; ++g, ++gc) {
        const int nv = min(PG_COLS, ncols - g * PG_COLS);
        const int s = gc % NS;
        const bool ok = warp_wait(sm, &sm.full[s], (uint32_t)((gc / NS) & 1));
        unsigned char* stg = stages + (size_t)s * PG_STAGE;
        float4 v[CV_ITEMS][2];
#pragma unroll
        for (int uu = 0; uu < CV_ITEMS; ++uu) {
          const int j = 8 * (w + NCV * (uu & 1)) + jl;   // column of the chunk (K index)
          const int g8 = gq + 4 * (uu >> 1);              // 8-row group (M index)
          v[uu][0] = v[uu][1] = make_float4(0.f, 0.f, 0.f, 0.f);
          if (ok && j < nv && g8 < ng) {   // rows 8 g8 .. 8 g8 + 7: slab g8 / 4
            const unsigned char* sl = stg + (g8 >> 2) * PG_SLAB;
            v[uu][0] = *reinterpret_cast<const float4*>(sl + swz(j, 2 * (g8 & 3)));
            v[uu][1] = *reinterpret_cast<const float4*>(sl + swz(j, 2 * (g8 & 3) + 1));
          }
        }
        if (!named_and(1, NCV * 32, ok)) {
          timed_out = true;
          go = false;
          break;
        }
#pragma unroll
        for (int uu = 0; uu < CV_ITEMS; ++uu) {
          const int j = 8 * (w + NCV * (uu & 1)) + jl;
          const int g8 = gq + 4 * (uu >> 1);
          uint4 hi, lo;   // columns beyond the window and rows beyond ld are written as zero
          split2(v[uu][0].x, v[uu][0].y, hi.x, lo.x);
          split2(v[uu][0].z, v[uu][0].w, hi.y, lo.y);
          split2(v[uu][1].x, v[uu][1].y, hi.z, lo.z);
          split2(v[uu][1].z, v[uu][1].w, hi.w, lo.w);
          const int o = (j >> 4) * 4096 + g8 * 256 + ((j >> 3) & 1) * 128 + (j & 7) * 16;
          *reinterpret_cast<uint4*>(stg + o) = hi;
          *reinterpret_cast<uint4*>(stg + PG_ALO + o) = lo;
        }
        tc::fence_proxy_async();
        __syncwarp();
        if (lane == 0) mbar_arrive(&sm.conv[s]);
      }
    }
  }

  if (timed_out) {
    atomicExch(&sm.abort_flag, 1);
    set_err(st, ERR_TIMEOUT);
  }
  if (warp == W_PROD && lane == 0) drain_fills(sm, NS, issued);
  __syncthreads();
  if (warp == W_MMA) {
    if (lane == 0) timed_wait(&sm.drain, 0u, WAIT_NS);
    __syncwarp();
    tc::fence_after_sync();
    tc::dealloc(tmem, 64);
  }
  if (tid == 0) ctl_inval(sm, NS);
}

// ---------------------------------------------------------------------------
// Column order for the solves: the window's columns stably sorted by their
// current passive set (16-bit mask), so that a 16-lane group's consecutive
// columns share their passive set and its carried inverse of G_PP is reused
// (the factorization reuse of Sec. 2, over columns grouped by passive set
// instead of neighbouring ones).  One CTA: the keys are gathered, then two
// LSD radix passes of 8 bits; each warp sorts a contiguous segment, lanes
// rank equal digits with a match, so equal keys keep their window order.
// ---------------------------------------------------------------------------
constexpr int SORT_T = 1024;

__global__ void __launch_bounds__(SORT_T) sort_cols_kernel(Problem p, Bufs bf) {
  __shared__ unsigned hist[SORT_T / 32][256];
  __shared__ unsigned dtot[256];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (p.st->done) return;
  const int cur = p.st->iter & 1;
  const int m = p.m;
  for (int i = tid; i < m; i += SORT_T) bf.keys[i] = (int)(p.ymask[cur][wrap_col(p.head, i, p.mcap)] & 0xFFFFu);
  __syncthreads();
  const int seg = (m + SORT_T / 32 - 1) / (SORT_T / 32);
  const int s0 = min(m, warp * seg), s1 = min(m, s0 + seg);
  const unsigned lt = (1u << lane) - 1u;
  for (int pass = 0; pass < 2; ++pass) {
    const int* src = pass == 0 ? nullptr : bf.perm_tmp;
    int* dst = pass == 0 ? bf.perm_tmp : bf.perm;
    const int shift = 8 * pass;
    for (int e = tid; e < (SORT_T / 32) * 256; e += SORT_T) hist[e >> 8][e & 255] = 0u;
    __syncthreads();
    for (int base = s0; base < s1; base += 32) {   // digit counts of the warp's segment
      const int i = base + lane;
      const bool v = i < s1;
      const int col = v ? (src ? src[i] : i) : 0;
      const unsigned d = v ? ((unsigned)bf.keys[col] >> shift) & 255u : 256u + lane;
      const unsigned peers = __match_any_sync(0xffffffffu, d);
      if (v && (peers & lt) == 0) hist[warp][d] += (unsigned)__popc(peers);
      __syncwarp();
    }
    __syncthreads();
    if (tid < 256) {   // offsets: digit-major, then warp order
      unsigned t = 0;
      for (int w = 0; w < SORT_T / 32; ++w) {
        const unsigned c = hist[w][tid];
        hist[w][tid] = t;
        t += c;
      }
      dtot[tid] = t;
    }
    __syncthreads();
    if (tid == 0) {
      unsigned t = 0;
      for (int d = 0; d < 256; ++d) {
        const unsigned c = dtot[d];
        dtot[d] = t;
        t += c;
      }
    }
    __syncthreads();
    for (int base = s0; base < s1; base += 32) {   // stable scatter
      const int i = base + lane;
      const bool v = i < s1;
      const int col = v ? (src ? src[i] : i) : 0;
      const unsigned d = v ? ((unsigned)bf.keys[col] >> shift) & 255u : 256u + lane;
      const unsigned peers = __match_any_sync(0xffffffffu, d);
      if (v) dst[dtot[d] + hist[warp][d] + (unsigned)__popc(peers & lt)] = col;
      __syncwarp();
      if (v && (peers & lt) == 0) hist[warp][d] += (unsigned)__popc(peers);
      __syncwarp();
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Column solves: every 16-lane group takes a contiguous range of window
// columns (the carried inverse of the group is reused where neighbours share
// their passive set; the FP32 rebuild is cheap enough that sorting the
// columns by passive set, as the FP64 refinement solves do, does not pay
// here), b_j = sum of the SB partials
// (fixed order); the KKT terms of the incoming iterate and H = Y Y^T; the
// BF16 split of the new y for the P-GEMM (zero for the padding columns of the
// last 64-column granule).  This pass's b carries ~1e-5 relative error, so
// its per-column arithmetic is FP32; the per-lane sums over a group's few
// columns are FP32, the sums across lanes and groups float-float (FP32
// instructions carrying each add's rounding error), those across blocks FP64
// (reduce_blocks, fixed order) into Hpart[0], Yterms[0]; entries 1 .. Q-1 are
// written as zero, so that the row pass's sum over Q partials (those of P)
// returns them.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(SOLVE_T, 3) solve_kernel(Problem p, Bufs bf, Plan L, int mode) {
  __shared__ float Gf[K][K + 1];
  __shared__ float wfs[SOLVE_T / 16][RED];   // per 16-lane group: H entries and term sums
  __shared__ float wfc[SOLVE_T / 16][NYT];   // the terms' float-float carries
  __shared__ unsigned last;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  DevState* st = p.st;
  if (st->done) return;
  const int cur = st->iter & 1, nxt = cur ^ 1;
  for (int e = tid; e < K * K; e += SOLVE_T) Gf[e / K][e % K] = (float)p.G[e];
  __syncthreads();
  LaneNnls16<float> nn;
  // the FP32 solve's own tolerance constant, 2^-23 (a finer one would follow
  // the rounding of this FP32 arithmetic and of B)
  nn.init(Gf, 1.1920928955078125e-07f);
  const int a = nn.a;
  const int ncols = p.m, ncolp = (ncols + PG_COLS - 1) / PG_COLS * PG_COLS;
  const int gid = blockIdx.x * (SOLVE_T / 16) + (tid >> 4);
  const int cbeg = min(ncolp, gid * L.cpgF), cend = min(ncolp, cbeg + L.cpgF);
  float acc_t[NYT];
#pragma unroll
  for (int e = 0; e < NYT; ++e) acc_t[e] = 0.f;
  float hacc[9];   // lane a: H[a][(a + d) % 16], d = 0..8
#pragma unroll
  for (int d = 0; d < 9; ++d) hacc[d] = 0.f;
  for (int col = cbeg; col < cend; ++col) {
    if (col >= ncols) {
      if (mode != MODE_KKT) {
        *reinterpret_cast<uint16_t*>(bf.Ys + xs_off(col, a)) = 0;
        *reinterpret_cast<uint16_t*>(bf.Ys + xs_off(col, K + a)) = 0;
      }
      continue;
    }
    const int phys = wrap_col(p.head, col, p.mcap);
    const float yo = (float)p.Y[cur][(size_t)phys * K + a];
    const uint32_t om = p.ymask[cur][phys];
    float b = 0.f;
    if (mode != MODE_PRIME) {
      float b4[4] = {0.f, 0.f, 0.f, 0.f};
      for (int s = 0; s < L.SB; ++s) b4[s & 3] += bf.Bpart[((size_t)s * p.mcap + col) * K + a];
      b = (b4[0] + b4[1]) + (b4[2] + b4[3]);
    }
    float yn = yo;
    uint32_t msk = 0;
    int stt = 0;
    if (mode == MODE_SWEEP) stt = nn.solve(b, yn, p.warm != 0, &msk);
    if (mode != MODE_PRIME) {
      // Y-half KKT terms of the incoming iterate: g = G yo - b (component a)
      const float gy = nn.gdot(yo) - b;
      const float mn = fminf(gy, 0.f), pos = fmaxf(gy, 0.f) * yo;
      acc_t[YT_NEG] = fmaf(mn, mn, acc_t[YT_NEG]);
      acc_t[YT_COMP] = fmaf(pos, pos, acc_t[YT_COMP]);
      acc_t[YT_BNORM2] = fmaf(b, b, acc_t[YT_BNORM2]);
      acc_t[YT_BY] = fmaf(b, yo, acc_t[YT_BY]);
      acc_t[YT_YGY] = fmaf(yo, gy + b, acc_t[YT_YGY]);
      acc_t[YT_YMAX] = fmaxf(acc_t[YT_YMAX], yo);
      acc_t[YT_YNORM2] = fmaf(yo, yo, acc_t[YT_YNORM2]);
      if (!isfinite(b)) set_err(st, ERR_NONFINITE);
    }
    if (mode == MODE_SWEEP) {
      acc_t[YT_DY2] = fmaf(yn - yo, yn - yo, acc_t[YT_DY2]);
      if (a == 0) {
        acc_t[YT_CHANGED] += (om != msk) ? 1.f : 0.f;
        acc_t[YT_NOTCONV] += (float)stt;
      }
      p.Y[nxt][(size_t)phys * K + a] = (double)yn;
      if (a == 0) p.ymask[nxt][phys] = msk;
    } else if (mode == MODE_PRIME) {
      const uint32_t pm = (__ballot_sync(nn.gm, yo > 0.f) >> nn.base) & 0xFFFFu;
      if (a == 0) p.ymask[cur][phys] = pm;
    }
    if (mode != MODE_KKT) {
#pragma unroll
      for (int d = 0; d < 9; ++d) hacc[d] = fmaf(yn, __shfl_sync(nn.gm, yn, nn.base + ((a + d) & 15)), hacc[d]);
      const uint16_t h = bf16_bits(yn);
      const uint16_t l = bf16_bits(yn - bf16_val(h));
      *reinterpret_cast<uint16_t*>(bf.Ys + xs_off(col, a)) = h;
      *reinterpret_cast<uint16_t*>(bf.Ys + xs_off(col, K + a)) = l;
    }
  }
  // group partials: H entries as the group's FP32 sums, the terms summed over
  // the group's lanes as float-float pairs; then per block, each entry over
  // the 16 groups in group order, float-float, to one double per entry
  const int grp = tid >> 4;
#pragma unroll
  for (int d = 0; d < 9; ++d) {
    const int c = (a + d) & 15;
    if (d < 8 || a < 8) {
      wfs[grp][a * K + c] = hacc[d];
      wfs[grp][c * K + a] = hacc[d];
    }
  }
#pragma unroll
  for (int e = 0; e < NYT; ++e) {
    float sv = acc_t[e], cv = 0.f;
#pragma unroll
    for (int o = 8; o >= 1; o >>= 1) {
      const float os = __shfl_xor_sync(nn.gm, sv, o), oc = __shfl_xor_sync(nn.gm, cv, o);
      if (e == YT_YMAX) sv = fmaxf(sv, os);
      else ff_add(sv, cv, os, oc);
    }
    if (a == 0) {
      wfs[grp][K * K + e] = sv;
      wfc[grp][e] = (e == YT_YMAX) ? 0.f : cv;
    }
  }
  __syncthreads();
  double* myred = bf.red + (size_t)blockIdx.x * RED;
  for (int e = tid; e < RED; e += SOLVE_T) {
    float sv = wfs[0][e], cv = e >= K * K ? wfc[0][e - K * K] : 0.f;
    for (int g = 1; g < SOLVE_T / 16; ++g) {
      if (e == K * K + YT_YMAX) sv = fmaxf(sv, wfs[g][e]);
      else ff_add(sv, cv, wfs[g][e], e >= K * K ? wfc[g][e - K * K] : 0.f);
    }
    myred[e] = (double)sv + (double)cv;
  }
  const double* tot = reduce_blocks(bf, &last);
  if (!tot) return;
  const int Q = L.SP;
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

}  // namespace tc16s
}  // namespace nmfgb

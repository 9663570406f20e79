// Host side of the rank-16 tensor-core M passes: launch plans and launches.
#include <algorithm>

#include <cudaTypedefs.h>

#include "nmf.h"
#include "nmf_tc16r.cuh"

namespace nmfgb {

namespace tc16s {

size_t bpart_bytes(int mcap) { return (size_t)8 * (size_t)mcap * K * sizeof(float); }
size_t xs_bytes(int ld) { return (size_t)ld * 64; }
size_t ys_bytes(int mcap) { return (size_t)((mcap + PG_COLS - 1) / PG_COLS) * PG_COLS * 64; }
size_t perm_bytes(int mcap) { return (size_t)mcap * sizeof(int); }
// block partials of up to 3 nsm blocks, their group partials, the totals
size_t red_bytes(int nsm) {
  const size_t nb = (size_t)3 * (size_t)std::max(1, nsm);
  return (nb + (nb + RGROUP - 1) / RGROUP + 1) * RED * sizeof(double);
}
size_t ticket_count(int nsm) { return 1 + ((size_t)3 * (size_t)std::max(1, nsm) + RGROUP - 1) / RGROUP; }

namespace {

// splits s in 1..smax minimising the time of `units1 * s` equal units on
// `slots` CTAs relative to one unit per CTA (waves / s), plus a small charge
// per split for the partials it writes
int best_splits(int units1, int smax, int slots) {
  int best = 1;
  double bc = 1e30;
  for (int s = 1; s <= std::max(1, smax); ++s) {
    const long long u = (long long)units1 * s;
    const double c = (double)((u + slots - 1) / slots) / s + 0.01 * s;
    if (c < bc - 1e-12) {
      bc = c;
      best = s;
    }
  }
  return best;
}

}  // namespace

void set_attr() {
  static bool done[64] = {false};
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64 || done[dev]) return;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  bool ok = cudaFuncSetAttribute(bgemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin) == cudaSuccess;
  ok &= cudaFuncSetAttribute(pgemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin) == cudaSuccess;
  if (ok) done[dev] = true;
  else cudaGetLastError();
}

bool encode_maps(void* M, int ld, int mcap, Maps* out) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
      cudaGetLastError();
      return false;
    }
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  const cuuint64_t dims[2] = {(cuuint64_t)ld, (cuuint64_t)mcap + MIRROR};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * sizeof(float)};
  const cuuint32_t es[2] = {1, 1};
  const cuuint32_t boxb[2] = {SLAB_ROWS, BG_COLS}, boxp[2] = {SLAB_ROWS, PG_COLS};
  bool ok = encode(&out->b, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, M, dims, strides, boxb, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
  ok = ok && encode(&out->p, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, M, dims, strides, boxp, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
  return ok;
}

bool plan(int ld, int m, int nsm, int smem_optin, Plan* out) {
  if (ld < 32 || ld % 32 != 0 || m < 1 || nsm < 1) return false;
  Plan L{};
  // two CTAs per SM: each holds at most half of the SM's shared memory (the
  // opt-in limit plus the 1 KB the SM reserves per CTA)
  const int half = (smem_optin + 1024) / 2 - 1024;
  const int slots = 2 * nsm;
  L.NSB = std::min(NSMAX, (half - CTL_BYTES) / BG_STAGE);
  L.NSP = std::min(NSMAX, (half - CTL_BYTES) / PG_STAGE);
  if (L.NSB < 2 || L.NSP < 2) return false;
  L.smemB = (size_t)CTL_BYTES + (size_t)L.NSB * BG_STAGE;
  L.smemP = (size_t)CTL_BYTES + (size_t)L.NSP * PG_STAGE;
  const int ngran = ld / 32;
  const int ntile = (m + BG_COLS - 1) / BG_COLS;
  // every row split keeps at least 64 rows (two 32-row granules)
  L.SB = best_splits(ntile, std::min(8, std::max(1, ngran / 2)), slots);
  L.gridB = std::min(ntile * L.SB, slots);
  const int nrb = (ld + PG_ROWS - 1) / PG_ROWS;
  const int ncg = (m + PG_COLS - 1) / PG_COLS;
  L.SP = best_splits(nrb, std::min(16, ncg), slots);
  L.gridP = std::min(nrb * L.SP, slots);
  // column solves: a group's columns run in sequence, each from the inverse
  // of G_PP carried from its left neighbour (neighbouring columns share most
  // of their passive set), so a group takes several columns, at most 16.
  const int ncolp = ncg * PG_COLS;
  const auto groups = [&](int per_sm, int& cpg, int& grid) {
    cpg = std::max(1, std::min(16, (ncolp + per_sm * nsm * (SOLVE_T / 16) - 1) / (per_sm * nsm * (SOLVE_T / 16))));
    const int ngroups = (ncolp + cpg - 1) / cpg;
    grid = (ngroups + SOLVE_T / 16 - 1) / (SOLVE_T / 16);
  };
  // FP64 refinement solves (solve64_kernel: FP64-pipe bound, runs of equal
  // passive sets after the sort) one block per SM; the FP32 solves two: their
  // chains of shuffles are latency-bound, and twice the groups with half the
  // columns each measured 8 % faster at m = 16384 (three per SM: the same)
  groups(1, L.cpg, L.gridS);
  groups(2, L.cpgF, L.gridF);
  if (L.gridS > 3 * nsm || L.gridF > 3 * nsm) return false;
  *out = L;
  return true;
}

cudaError_t launch(const Problem& p, int mode, const Plan& L, const Bufs& B, const Maps& T, cudaStream_t s,
                   int* nl) {
  set_attr();
  int n = 0;
  if (mode != MODE_PRIME) {
    const int tot = p.ld * K;
    xsplit_kernel<<<std::min((tot + 255) / 256, 1024), 256, 0, s>>>(p, B);
    bgemm_kernel<<<L.gridB, NT, L.smemB, s>>>(T.b, p, B, L);
    n += 2;
  }
  solve_kernel<<<L.gridF, SOLVE_T, 0, s>>>(p, B, L, mode);
  ++n;
  if (mode != MODE_KKT) {
    pgemm_kernel<<<L.gridP, NT, L.smemP, s>>>(T.p, p, B, L);
    ++n;
  }
  if (nl) *nl = n;
  return cudaGetLastError();
}

}  // namespace tc16s

namespace tc16r {

size_t bdf_bytes(int ld, int mcap) { return (size_t)((ld + BR - 1) / BR) * (size_t)mcap * K * sizeof(double); }

bool plan(int ld, int m, int nsm, RefPlan* out) {
  if (ld < 32 || ld % 32 != 0 || m < 1 || nsm < 1) return false;
  RefPlan R{};
  // two CTAs per SM for both kernels
  R.nrbB = (ld + BR - 1) / BR;
  R.slicesB = std::max(1, std::min(m, (2 * nsm + R.nrbB - 1) / R.nrbB));
  R.gridB = R.nrbB * R.slicesB;
  R.nrbP = (ld + TP - 1) / TP;
  R.SPd = std::max(1, std::min(std::min(m, nsm), (2 * nsm) / R.nrbP));
  R.gridP = R.nrbP * R.SPd;
  *out = R;
  return true;
}

namespace {
void set_attr_ref() {
  static bool done[64] = {false};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64 || done[dev]) return;
  if (cudaFuncSetAttribute(dfb_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dfb_smem()) == cudaSuccess)
    done[dev] = true;
  else
    cudaGetLastError();
}
}  // namespace

cudaError_t launch(const Problem& p, int mode, int pass, const RefPlan& R, const tc16s::Plan& L,
                   const tc16s::Bufs& B, const tc16s::Maps& T, double* Bdf, cudaStream_t s, int* nl, int* Q) {
  set_attr_ref();
  tc16s::set_attr();
  int n = 0;
  if (pass == REF_PASS) {
    *Q = R.SPd;
    if (mode != MODE_PRIME) {
      dfb_kernel<<<R.gridB, TB, dfb_smem(), s>>>(p, Bdf, R);
      ++n;
    }
    tc16s::sort_cols_kernel<<<1, tc16s::SORT_T, 0, s>>>(p, B);
    solve64_kernel<<<L.gridS, SOLVE_T, 0, s>>>(p, B, Bdf, R, L.cpg, R.nrbB, R.SPd, REF, mode);
    n += 2;
    if (mode != MODE_KKT) {
      dfp_kernel<<<R.gridP, TP, 0, s>>>(p, R, mode);
      ++n;
    }
  } else {
    *Q = L.SP;
    const int tot = p.ld * K;
    xdsplit_kernel<<<std::min((tot + 255) / 256, 1024), 256, 0, s>>>(p, B);
    tc16s::bgemm_kernel<<<L.gridB, tc16s::NT, L.smemB, s>>>(T.b, p, B, L);
    tc16s::sort_cols_kernel<<<1, tc16s::SORT_T, 0, s>>>(p, B);
    solve64_kernel<<<L.gridS, SOLVE_T, 0, s>>>(p, B, Bdf, R, L.cpg, L.SB, L.SP, INC, mode);
    tc16s::pgemm_kernel<<<L.gridP, tc16s::NT, L.smemP, s>>>(T.p, p, B, L);
    n += 5;
  }
  if (nl) *nl = n;
  return cudaGetLastError();
}

}  // namespace tc16r

namespace {

// One warp waits, through the rank-16 pass's own bounded wait, on an mbarrier
// that nothing arrives on; out[0] = 1 when the wait gave up, out[1] = the
// abort flag it raised for the other roles.
__global__ void tc16_wait_selftest_kernel(unsigned long long limit_ns, int* out) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    abort_flag = 0;
    fence_mbar_init();
  }
  __syncthreads();
  const bool ok = tc16::bwait_flag<false>(&abort_flag, &bar, 0u, limit_ns);
  __syncthreads();
  if (threadIdx.x == 0) {
    out[0] = ok ? 0 : 1;
    out[1] = abort_flag;
    mbar_inval(&bar);
  }
}

}  // namespace

}  // namespace nmfgb

extern "C" nmf_status nmf_selftest_tc16_wait(int64_t limit_ms, void* cuda_stream) {
  if (limit_ms < 1 || limit_ms > 10000) return NMF_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  int* d = nullptr;
  int h[2] = {0, 0};
  if (cudaMalloc(&d, 2 * sizeof(int)) != cudaSuccess) return NMF_ENOMEM;
  nmf_status out = NMF_ECUDA;
  if (cudaMemsetAsync(d, 0, 2 * sizeof(int), s) == cudaSuccess) {
    nmfgb::tc16_wait_selftest_kernel<<<1, 32, 0, s>>>((unsigned long long)limit_ms * 1000000ull, d);
    if (cudaGetLastError() == cudaSuccess &&
        cudaMemcpyAsync(h, d, 2 * sizeof(int), cudaMemcpyDeviceToHost, s) == cudaSuccess &&
        cudaStreamSynchronize(s) == cudaSuccess)
      out = (h[0] == 1 && h[1] == 1) ? NMF_ETIMEOUT : NMF_OK;
  }
  cudaFree(d);
  return out;
}

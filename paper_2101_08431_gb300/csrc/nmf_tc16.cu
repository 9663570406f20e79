// Host side of the rank-16 tensor-core M pass: launch plan and launch.
#include "nmf.h"
#include "nmf_tc16.cuh"

namespace nmfgb {

namespace {

void tc16_set_attr() {
  static bool done[64] = {false};
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64 || done[dev]) return;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  bool ok = cudaFuncSetAttribute(tc16::ypass_tc16_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin) ==
            cudaSuccess;
  ok &= cudaFuncSetAttribute(tc16::ypass_tc16_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
        cudaSuccess;
  if (ok) done[dev] = true;
  else cudaGetLastError();
}

cudaLaunchConfig_t tc16_config(const Tc16Plan& L, cudaLaunchAttribute* at) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(L.Q * L.C), 1, 1);
  cfg.blockDim = dim3(tc16::NT, 1, 1);
  cfg.dynamicSmemBytes = L.smem;
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)L.C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cfg;
}

int pow2ceil(int v) {
  int p = 1;
  while (p < v) p <<= 1;
  return p;
}

}  // namespace

bool tc16_shape(int ld, int C, int smem_optin, Tc16Plan* out) {
  using namespace tc16;
  if (ld < 1 || C < 1 || C > 16 || (C & (C - 1)) != 0) return false;
  const size_t small = small_bytes();
  const int R = (ld + C - 1) / C;
  const int Rr = (R + 127) / 128 * 128;
  const long long room = (long long)smem_optin - (long long)small - (long long)ax_bytes(Rr);
  if (room <= 0) return false;
  int NS = (int)(room / (long long)slot_bytes(Rr));
  if (NS > NSMAX) NS = NSMAX;
  if (NS < 2) return false;
  const int tcols = pow2ceil(std::max(32, NS * 32 + (Rr / 128) * 16));
  if (tcols > 512) return false;
  Tc16Plan L{};
  L.C = C;
  L.R = Rr;
  L.NS = NS;
  L.Q = 0;
  L.tmem_cols = tcols;
  L.smem = small + ax_bytes(Rr) + (size_t)NS * slot_bytes(Rr);
  *out = L;
  return true;
}

bool tc16_plan(int ld, int m, int nsm, int smem_optin, Tc16Plan* out) {
  using namespace tc16;
  tc16_set_attr();
  Tc16Plan best{};
  bool have = false;
  for (int C = 1; C <= 16; C <<= 1) {
    Tc16Plan L{};
    if (!tc16_shape(ld, C, smem_optin, &L)) continue;
    cudaLaunchAttribute at[1];
    L.Q = 1;
    cudaLaunchConfig_t cfg = tc16_config(L, at);
    int fit = 0;
    if (cudaOccupancyMaxActiveClusters(&fit, (const void*)ypass_tc16_kernel, &cfg) != cudaSuccess) {
      cudaGetLastError();
      fit = 0;
    }
    if (fit <= 0) continue;
    const int tiles = std::max(1, (m + TJ - 1) / TJ);
    L.Q = std::max(1, std::min(fit, tiles));
    (void)nsm;
    best = L;
    have = true;
    if (L.NS >= 4) break;   // the smallest cluster with a ring of four tiles
  }
  if (have) *out = best;
  return have;
}

cudaError_t tc16_launch(const Problem& p, int mode, const Tc16Plan& L, cudaStream_t s) {
  tc16_set_attr();
  cudaLaunchAttribute at[1];
  cudaLaunchConfig_t cfg = tc16_config(L, at);
  cfg.stream = s;
  return cudaLaunchKernelEx(&cfg, tc16::ypass_tc16_kernel, p, mode, L);
}

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

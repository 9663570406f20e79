// Launch plumbing shared by the kernel-instantiation units and the C ABI.
#pragma once

#include "nmf_sweep.cuh"

namespace nmfgb {

struct YPlan {
  int C, R, Q, S;
  size_t smem;
};

struct KernelSet {
  cudaError_t (*ypass)(const Problem&, int mode, const YPlan&, cudaStream_t);
  int (*max_clusters)(int C, size_t smem);   // co-resident clusters of the M pass
  cudaError_t (*xpass)(const Problem&, int mode, int Q, int nxblk, cudaStream_t);
  int TJ, RPT;
  int rows;                                  // rows one CTA of the M pass can own
  size_t small_bytes;
  int tm_size;
  int pacc_row_bytes;                        // shared-memory P accumulators per owned row
};

bool get_kernels_f32(int k, KernelSet* out);
bool get_kernels_ref(int k, KernelSet* out);
bool get_kernels_f64(int k, KernelSet* out);
bool get_kernels_df(int k, KernelSet* out);
bool get_kernels_inc(int k, KernelSet* out);

template <typename TM, typename AR, int K>
cudaError_t launch_y(const Problem& p, int mode, const YPlan& L, cudaStream_t s) {
  auto kern = ypass_kernel<TM, AR, K>;
  static bool attr_done[64] = {false};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64 && !attr_done[dev]) {
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
    if (e != cudaSuccess) return e;
    cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    attr_done[dev] = true;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(L.Q * L.C, 1, 1);
  cfg.blockDim = dim3(YTraits<TM, AR, K>::T, 1, 1);
  cfg.dynamicSmemBytes = L.smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = L.C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, p, mode, L.S, L.C, L.R, L.Q);
}

// How many clusters of C CTAs with `smem` bytes each the device can hold at
// once (the M pass is persistent: a second wave would double its time).
template <typename TM, typename AR, int K>
int max_clusters_y(int C, size_t smem) {
  auto kern = ypass_kernel<TM, AR, K>;
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C, 1, 1);
  cfg.blockDim = dim3(YTraits<TM, AR, K>::T, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, (const void*)kern, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

template <typename TA, int K>
cudaError_t launch_x(const Problem& p, int mode, int Q, int nxblk, cudaStream_t s) {
  auto kern = xpass_kernel<TA, K>;
  constexpr size_t dyn = XSmem<TA, K>::bytes();
  static bool attr_done[64] = {false};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64 && !attr_done[dev]) {
    if (dyn > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
      if (e != cudaSuccess) return e;
    }
    // the same shared-memory carve-out as the M pass, so that the SMs need
    // not be reconfigured between the two kernels of a sweep
    cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    attr_done[dev] = true;
  }
  kern<<<nxblk, XTraits<K>::T, dyn, s>>>(p, mode, Q, nxblk);
  return cudaGetLastError();
}

// TM: element type of M, AR: accumulation policy, PT: element type of the
// P partials (read by the row pass)
#define NMF_FILL(TM, AR, PT, K)                              \
  case K:                                                    \
    out->ypass = launch_y<TM, AR, K>;                        \
    out->max_clusters = max_clusters_y<TM, AR, K>;           \
    out->xpass = launch_x<PT, K>;                            \
    out->TJ = YTraits<TM, AR, K>::TJ;                        \
    out->RPT = YTraits<TM, AR, K>::RPT;                      \
    out->rows = YTraits<TM, AR, K>::ROWS;                    \
    out->small_bytes = YSmem<TM, AR, K>::small_bytes();      \
    out->tm_size = (int)sizeof(TM);                          \
    out->pacc_row_bytes = YTraits<TM, AR, K>::PACC_ROW_BYTES; \
    return true;

#define NMF_FILL_ALL(TM, AR, PT)                                                                  \
  switch (k) {                                                                                    \
    NMF_FILL(TM, AR, PT, 1) NMF_FILL(TM, AR, PT, 2) NMF_FILL(TM, AR, PT, 3)                       \
    NMF_FILL(TM, AR, PT, 4) NMF_FILL(TM, AR, PT, 5) NMF_FILL(TM, AR, PT, 6)                       \
    NMF_FILL(TM, AR, PT, 7) NMF_FILL(TM, AR, PT, 8) NMF_FILL(TM, AR, PT, 16)                      \
    default: return false;                                                                        \
  }

}  // namespace nmfgb

// Launch plumbing shared by the kernel-instantiation units and the C ABI.
#pragma once

#include "nmf_sweep.cuh"

namespace nmfgb {

// Arithmetic of one M pass.
enum Variant {
  VAR_F32 = 0,   // FP32 M, FP32 contraction (mixed precision, bulk sweeps)
  VAR_REF = 1,   // FP32 M, FP64 contraction (mixed precision, refinement sweeps)
  VAR_F64 = 2,   // FP64 M, FP64 contraction (the plain FP64 form)
  NVAR = 3
};

struct YPlan {
  int C, R, Q, S;
  size_t smem;
};

struct KernelSet {
  cudaError_t (*ypass)(const Problem&, int mode, const YPlan&, cudaStream_t);
  int (*max_clusters)(int C, size_t smem);   // co-resident clusters of the M pass
  cudaError_t (*xpass)(const Problem&, int mode, int Q, int nxblk, cudaStream_t);
  int TJ, RPT;
  size_t small_bytes;
  int tm_size;
};

bool get_kernels_f32(int k, KernelSet* out);
bool get_kernels_ref(int k, KernelSet* out);
bool get_kernels_f64(int k, KernelSet* out);

template <typename TM, typename TA, int K>
cudaError_t launch_y(const Problem& p, int mode, const YPlan& L, cudaStream_t s) {
  auto kern = ypass_kernel<TM, TA, K>;
  static bool attr_done[64] = {false};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64 && !attr_done[dev]) {
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
    if (e != cudaSuccess) return e;
    attr_done[dev] = true;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(L.Q * L.C, 1, 1);
  cfg.blockDim = dim3(YTraits<TM, TA, K>::T, 1, 1);
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
template <typename TM, typename TA, int K>
int max_clusters_y(int C, size_t smem) {
  auto kern = ypass_kernel<TM, TA, K>;
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C, 1, 1);
  cfg.blockDim = dim3(YTraits<TM, TA, K>::T, 1, 1);
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
  xpass_kernel<TA, K><<<nxblk, XTraits<K>::T, 0, s>>>(p, mode, Q, nxblk, nullptr);
  return cudaGetLastError();
}

#define NMF_FILL(TM, TA, K)                                  \
  case K:                                                    \
    out->ypass = launch_y<TM, TA, K>;                        \
    out->max_clusters = max_clusters_y<TM, TA, K>;           \
    out->xpass = launch_x<TA, K>;                            \
    out->TJ = YTraits<TM, TA, K>::TJ;                        \
    out->RPT = YTraits<TM, TA, K>::RPT;                      \
    out->small_bytes = YSmem<TM, TA, K>::small_bytes();      \
    out->tm_size = (int)sizeof(TM);                          \
    return true;

#define NMF_FILL_ALL(TM, TA)                                                              \
  switch (k) {                                                                            \
    NMF_FILL(TM, TA, 1) NMF_FILL(TM, TA, 2) NMF_FILL(TM, TA, 3) NMF_FILL(TM, TA, 4)       \
    NMF_FILL(TM, TA, 5) NMF_FILL(TM, TA, 6) NMF_FILL(TM, TA, 7) NMF_FILL(TM, TA, 8)       \
    NMF_FILL(TM, TA, 16)                                                                  \
    default: return false;                                                                \
  }

}  // namespace nmfgb

// Measured FMA throughput of this GPU, the denominators of the ALU rooflines
// (the FP64 form's M pass, the SIMT passes): kernels of independent FMA chains
// on every SM, timed with CUDA events on the caller's stream.
#include <cstdint>

#include "nmf.h"
#include "nmf_common.cuh"

namespace {

constexpr int CHAINS = 8;           // independent FMA chains per thread
constexpr int PEAK_THREADS = 256;   // threads per block; 2 blocks per SM

// x <- x a + b on CHAINS independent chains for `iters` steps; |a| < 1 keeps
// the values bounded.  The final store is guarded by a test the values never
// meet, so that the chains are not removed and nothing is written.
template <typename T>
__global__ void __launch_bounds__(PEAK_THREADS) fma_chain_kernel(T* sink, int iters, T a, T b) {
  T x[CHAINS];
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) x[c] = fma(x[c], a, b);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) s += x[c];
  if (s == (T)-1.0) sink[threadIdx.x] = s;
}

template <typename T>
bool time_fma(cudaStream_t s, int nsm, int iters, double* tflops) {
  T* sink = nullptr;
  if (cudaMalloc(&sink, PEAK_THREADS * sizeof(T)) != cudaSuccess) return false;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  bool ok = cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess;
  const int grid = 2 * nsm;
  float ms = 0.f;
  if (ok) {
    fma_chain_kernel<T><<<grid, PEAK_THREADS, 0, s>>>(sink, iters / 8, (T)0.999999, (T)1e-7);   // warm-up
    cudaEventRecord(e0, s);
    fma_chain_kernel<T><<<grid, PEAK_THREADS, 0, s>>>(sink, iters, (T)0.999999, (T)1e-7);
    cudaEventRecord(e1, s);
    ok = cudaGetLastError() == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
         cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms > 0.f;
  }
  if (ok) *tflops = 2.0 * CHAINS * (double)iters * grid * PEAK_THREADS / (ms * 1e-3) / 1e12;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(sink);
  return ok;
}

}  // namespace

extern "C" nmf_status nmf_measure_fma_peaks(double* out, void* cuda_stream) {
  if (!out) return NMF_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1)
    return NMF_ECUDA;
  // ~5 GFLOP of FP64 and ~80 GFLOP of FP32: a few ms each at this part's rates
  if (!time_fma<double>(s, nsm, 4096, &out[0])) return NMF_ECUDA;
  if (!time_fma<float>(s, nsm, 131072, &out[1])) return NMF_ECUDA;
  return NMF_OK;
}

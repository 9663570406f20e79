// nmf_sweep_noalloc: one ANLS sweep on caller-owned device memory that
// allocates nothing.  Every piece of working memory the sweep needs (the
// partial products of the M pass, the block partials of the row pass, the
// device control block, the next iterate) lives in one file-scope
// __device__ array of NOALLOC_SCRATCH_BYTES.  The caller passes M, X and Y;
// X and Y are updated in place.
#include <cstdint>
#include <cstring>
#include <mutex>

#include "nmf.h"
#include "nmf_launch.cuh"

using namespace nmfgb;

namespace {

constexpr int NA_NMAX = 2048;        // rows
constexpr int NA_MMAX = 4096;        // columns
constexpr int NA_KMAX = 8;           // rank
constexpr int NA_QMAX = 32;          // clusters of the M pass
constexpr size_t NOALLOC_SCRATCH_BYTES = size_t(5) << 20;

// The scratch.  Every GPU that loads the library holds it until the process
// exits.  Host code must not use the name as an address (it is a host-side
// stand-in); the set-up below obtains the device address.
__device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

std::mutex g_setup_mu;
void* g_scratch_dev[64] = {};        // device address of the array, per device

nmf_status scratch_for_current_device(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return NMF_ECUDA;
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_scratch_dev[dev]) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) {
      cudaGetLastError();
      return NMF_ECUDA;
    }
    g_scratch_dev[dev] = ptr;
  }
  *out = g_scratch_dev[dev];
  return NMF_OK;
}

// ||M_{:,j}||^2 per column (FP64) and their sum into the control block.
__global__ void na_colsq_kernel(const float* M, long long ld, int n, double* colsq) {
  __shared__ double red[32];
  const float* col = M + (size_t)blockIdx.x * ld;
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc = fmad((double)col[i], (double)col[i], acc);
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    colsq[blockIdx.x] = t;
  }
}

__global__ void na_msq_kernel(const double* colsq, int m, DevState* st) {
  __shared__ double red[256];
  double t = 0.0;
  for (int j = threadIdx.x; j < m; j += blockDim.x) t += colsq[j];
  red[threadIdx.x] = t;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) st->msq = red[0];
}

// Last step of a call: the statistics record of the incoming iterate (slot
// 15: the control block's error bits, 0 when the sweep completed cleanly) and,
// only when no error bit is set, the next iterate over the caller's X and Y.
// With an error bit set X and Y keep the incoming iterate.
__global__ void na_finish_kernel(const DevState* st, const double* Xn, double* X, long long nx, const double* Yn,
                                 double* Y, long long ny, double* stats_dev) {
  const unsigned err = st->err;
  const long long i0 = blockIdx.x * (long long)blockDim.x + threadIdx.x, step = (long long)gridDim.x * blockDim.x;
  if (stats_dev && i0 < NSTAT) stats_dev[i0] = (i0 == NSTAT - 1) ? (double)err : st->stats[0][i0];
  if (err) return;
  for (long long i = i0; i < nx; i += step) X[i] = Xn[i];
  for (long long i = i0; i < ny; i += step) Y[i] = Yn[i];
}

size_t take(size_t& off, size_t bytes) {
  const size_t at = off;
  off += (bytes + 255) & ~size_t(255);
  return at;
}

}  // namespace

extern "C" nmf_status nmf_sweep_noalloc(const float* M, int64_t n, int64_t m, int64_t ldm, int32_t k,
                                        double* X, double* Y, double* stats_dev, void* cuda_stream) {
  if (!M || !X || !Y || n < 1 || m < 1 || k < 1) return NMF_EINVAL;
  if (n > NA_NMAX || m > NA_MMAX || k > NA_KMAX) return NMF_ECAPACITY;
  if (ldm != ((n + 31) / 32) * 32) return NMF_EINVAL;
  // the M pass stages column segments with bulk copies, which need a 16-byte
  // aligned source (ldm * 4 bytes is a multiple of 128); X, Y and the record
  // are read and written as doubles.  Checked here, before any device work.
  if (reinterpret_cast<uintptr_t>(M) % 16 != 0 || reinterpret_cast<uintptr_t>(X) % 8 != 0 ||
      reinterpret_cast<uintptr_t>(Y) % 8 != 0 || reinterpret_cast<uintptr_t>(stats_dev) % 8 != 0)
    return NMF_EINVAL;
  cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
  void* base = nullptr;
  nmf_status s = scratch_for_current_device(&base);
  if (s != NMF_OK) return s;
  KernelSet ks;
  if (!get_kernels_ref(k, &ks)) return NMF_EINVAL;
  int dev = 0, nsm = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);

  // launch plan of the M pass: at most NA_QMAX clusters
  const int ld = (int)ldm;
  int C = 1, R = 0;
  for (C = 1; C <= 8; C <<= 1) {
    R = ((ld + C - 1) / C + 31) / 32 * 32;
    if (R <= ks.rows) break;
  }
  if (C > 8) return NMF_ECAPACITY;
  YPlan L;
  L.C = C;
  L.R = R;
  L.Q = (int)std::min<int64_t>(std::min(NA_QMAX, std::max(1, nsm / C)), m);
  const int cpc = (int)((m + L.Q - 1) / L.Q);
  const int ntiles = (cpc + ks.TJ - 1) / ks.TJ;
  const size_t stage = (size_t)ks.TJ * R * sizeof(float);
  const size_t pacc = (size_t)R * ks.pacc_row_bytes;
  long long S = ((long long)optin - (long long)ks.small_bytes - (long long)pacc) / (long long)stage;
  S = std::min<long long>(std::min<long long>(S, 8), ntiles);
  if (S < (ntiles > 1 ? 2 : 1)) return NMF_ECAPACITY;
  L.S = (int)S;
  L.smem = ks.small_bytes + (size_t)S * stage + pacc;

  // carve the scratch
  unsigned char* b = static_cast<unsigned char*>(base);
  size_t off = 0;
  DevState* st = reinterpret_cast<DevState*>(b + take(off, sizeof(DevState)));
  double* G = reinterpret_cast<double*>(b + take(off, sizeof(double) * NA_KMAX * NA_KMAX));
  double* Gtab = reinterpret_cast<double*>(b + take(off, sizeof(double) * (1 << NA_KMAX) * NA_KMAX * NA_KMAX));
  int* Gok = reinterpret_cast<int*>(b + take(off, sizeof(int) * (1 << NA_KMAX)));
  double* colsq = reinterpret_cast<double*>(b + take(off, sizeof(double) * NA_MMAX));
  double* Xn = reinterpret_cast<double*>(b + take(off, sizeof(double) * NA_NMAX * NA_KMAX));
  float* X32a = reinterpret_cast<float*>(b + take(off, sizeof(float) * NA_NMAX * NA_KMAX));
  float* X32b = reinterpret_cast<float*>(b + take(off, sizeof(float) * NA_NMAX * NA_KMAX));
  float* X32la = reinterpret_cast<float*>(b + take(off, sizeof(float) * NA_NMAX * NA_KMAX));
  float* X32lb = reinterpret_cast<float*>(b + take(off, sizeof(float) * NA_NMAX * NA_KMAX));
  double* Yn = reinterpret_cast<double*>(b + take(off, sizeof(double) * NA_MMAX * NA_KMAX));
  uint32_t* ym0 = reinterpret_cast<uint32_t*>(b + take(off, sizeof(uint32_t) * NA_MMAX));
  uint32_t* ym1 = reinterpret_cast<uint32_t*>(b + take(off, sizeof(uint32_t) * NA_MMAX));
  uint32_t* xm0 = reinterpret_cast<uint32_t*>(b + take(off, sizeof(uint32_t) * NA_NMAX));
  uint32_t* xm1 = reinterpret_cast<uint32_t*>(b + take(off, sizeof(uint32_t) * NA_NMAX));
  double* Ppart = reinterpret_cast<double*>(b + take(off, sizeof(double) * NA_QMAX * NA_NMAX * NA_KMAX));
  double* Hpart = reinterpret_cast<double*>(b + take(off, sizeof(double) * NA_QMAX * NA_KMAX * NA_KMAX));
  double* Yterms = reinterpret_cast<double*>(b + take(off, sizeof(double) * NA_QMAX * NYT));
  const int nxblk = (int)((n + XTraits<1>::RB - 1) / XTraits<1>::RB);
  double* Xpart = reinterpret_cast<double*>(
      b + take(off, sizeof(double) * (NA_NMAX / XTraits<1>::RB) * (NA_KMAX * NA_KMAX + NXT)));
  if (off > NOALLOC_SCRATCH_BYTES) return NMF_ECAPACITY;

  Problem p{};
  p.n = (int)n;
  p.m = (int)m;
  p.k = k;
  p.ld = ld;
  p.mcap = (int)m;
  p.head = 0;
  p.M = M;
  p.X[0] = X;
  p.X[1] = Xn;
  p.X32[0] = X32a;
  p.X32[1] = X32b;
  p.X32lo[0] = X32la;
  p.X32lo[1] = X32lb;
  p.Y[0] = Y;
  p.Y[1] = Yn;
  p.ymask[0] = ym0;
  p.ymask[1] = ym1;
  p.xmask[0] = xm0;
  p.xmask[1] = xm1;
  p.G = G;
  p.Gtab = Gtab;
  p.Gok = Gok;
  p.colsq = colsq;
  p.Ppart = Ppart;
  p.Hpart = Hpart;
  p.Yterms = Yterms;
  p.Xpart = Xpart;
  p.st = st;
  p.kkt_target = 0.0;
  p.stol = 0.0;
  p.warm = 1;
  p.fp64_pass = 1;

  // the array keeps the previous call's contents: the control block (iterate
  // index, stop flag, error bits, last-block counter, terms) starts at zero
  if (cudaMemsetAsync(st, 0, sizeof(DevState), stream) != cudaSuccess) return NMF_ECUDA;
  na_colsq_kernel<<<(unsigned)m, 256, 0, stream>>>(M, ldm, (int)n, colsq);
  na_msq_kernel<<<1, 256, 0, stream>>>(colsq, (int)m, st);
  if (cudaGetLastError() != cudaSuccess) return NMF_ECUDA;
  // priming pair (G = X^T X, passive sets, X-half terms of the incoming
  // iterate), then the sweep itself; the result lands in the buffers of index 1
  if (ks.ypass(p, MODE_PRIME, L, stream) != cudaSuccess) return NMF_ECUDA;
  if (ks.xpass(p, MODE_PRIME, L.Q, nxblk, stream) != cudaSuccess) return NMF_ECUDA;
  if (ks.ypass(p, MODE_SWEEP, L, stream) != cudaSuccess) return NMF_ECUDA;
  if (ks.xpass(p, MODE_SWEEP, L.Q, nxblk, stream) != cudaSuccess) return NMF_ECUDA;
  na_finish_kernel<<<32, 256, 0, stream>>>(st, Xn, X, (long long)n * k, Yn, Y, (long long)m * k, stats_dev);
  if (cudaGetLastError() != cudaSuccess) return NMF_ECUDA;
  return NMF_OK;
}

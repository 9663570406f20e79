// Batched persistent form of the ANLS sweep: many independent problems in
// one launch per (k, cluster size) class.  Clusters claim work items from a
// global counter in list order:
//
//   sweep s: [M-pass items (problem j, column group q)] for every problem,
//            then [row-pass items (problem j, row-block group g)]
//
// and run the same bodies as the one-problem kernels.  Per-problem
// dependencies are global counters: an M-pass item of sweep s waits until
// the problem's tail of sweep s-1 has published its results (t_done >= s);
// a row-pass item waits until every M-pass CTA of its sweep has finished and
// (k <= 8) the H stage run by the last of them has published H and its
// subset table (a_done >= (s+1) (Q C + 1)).  Items are claimed in list order and depend only on
// items earlier in the list, which are held by running clusters, so every
// wait ends; each wait is bounded all the same (ERR_TIMEOUT, and the
// problem is stopped so that nothing waits on it).  A problem whose tail
// stops it (KKT target or step tolerance) drops out: its later items are
// claimed and skipped.
#pragma once

#include "nmf_launch.cuh"

namespace nmfgb {

// One problem of a batched launch (device memory).
struct BatchProb {
  Problem pv[2];   // the problem as the FP32 pass (0) and the compensated pass (1) see it
  int S[2];        // stages of each variant's M pass
  int R;           // rows per CTA of the M pass
  int Q;           // column groups: M-pass items per sweep
  int nxblk;       // row blocks of the row pass
  int nxg;         // row-pass items per sweep, ceil(nxblk / C)
};

struct BatchArgs {
  const BatchProb* probs;
  int nprob;
  const int* aoff;       // [nprob + 1]: prefix sums of Q
  const int* boff;       // [nprob + 1]: prefix sums of nxg
  int nsweeps;           // sweeps covered by the launch
  unsigned* counter;     // next item to claim (zero at launch)
  unsigned* a_done;      // [nprob]: M-pass CTAs finished in this launch (zero at launch)
  unsigned* t_done;      // [nprob]: sweeps whose tail finished in this launch (zero at launch)
  int force_var;         // -1: each problem's own schedule; 0: FP32 pass; 1: compensated pass
  unsigned smem_budget;  // dynamic shared bytes the bodies may use (the claim words follow)
};

// Largest j with off[j] <= r (off[0] = 0 <= r < off[n]).
__device__ __forceinline__ int batch_find(const int* off, int n, int r) {
  int lo = 0, hi = n;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (off[mid] <= r) lo = mid;
    else hi = mid;
  }
  return lo;
}

constexpr long long BATCH_SPIN_LIMIT = 1ll << 23;   // polls of ~256 ns: about 2 s

// Thread 0: wait until *ctr >= target or the problem has stopped.  On
// timeout the problem is marked stopped with ERR_TIMEOUT.
__device__ __forceinline__ void batch_wait(const unsigned* ctr, unsigned target, DevState* st,
                                           long long limit = BATCH_SPIN_LIMIT) {
  for (long long i = 0; i < limit; ++i) {
    if (ld_acquire_u32(ctr) >= target) return;
    if (*reinterpret_cast<volatile int*>(&st->done)) return;
    __nanosleep(256);
  }
  set_err(st, ERR_TIMEOUT);
  atomicExch(&st->done, 1);
  __threadfence();
}

template <int K>
__global__ void __launch_bounds__(512, 1) batch_kernel(BatchArgs a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned* s_item = reinterpret_cast<unsigned*>(smem_raw + a.smem_budget);   // two claim words, a flag
  constexpr unsigned HS = K <= 8 ? 1u : 0u;   // H-stage increments of a_done per sweep
  cg::cluster_group cluster = cg::this_cluster();
  const int C = (int)cluster.num_blocks();
  const int crank = (int)cluster.block_rank();
  const int A = a.aoff[a.nprob], B = a.boff[a.nprob], I = A + B;
  const unsigned total = (unsigned)I * (unsigned)a.nsweeps;
  for (unsigned round = 0;; ++round) {
    // the leader claims; the claim word alternates so that a fast leader
    // never overwrites a word a peer has not read yet
    unsigned* word = s_item + (round & 1);
    if (crank == 0 && threadIdx.x == 0) {
      const unsigned it = atomicAdd(a.counter, 1u);
      for (int r = 0; r < C; ++r) *cluster.map_shared_rank(word, r) = it;
    }
    cluster.sync();
    const unsigned it = *word;
    if (it >= total) break;
    const int s = (int)(it / (unsigned)I);
    int r = (int)(it % (unsigned)I);
    if (r < A) {
      // ---- M pass of column group q of problem j
      const int j = batch_find(a.aoff, a.nprob, r);
      const BatchProb& bp = a.probs[j];
      DevState* st = bp.pv[0].st;
      const int q = r - a.aoff[j];
      if (threadIdx.x == 0) batch_wait(&a.t_done[j], (unsigned)s, st);
      __syncthreads();
      if (!*reinterpret_cast<volatile int*>(&st->done)) {
        const int var = a.force_var >= 0 ? a.force_var : (st->pass_var == VAR_DF ? 1 : 0);
        if (var == 0)
          ypass_body<float, ArF32, K>(bp.pv[0], MODE_SWEEP, bp.S[0], C, bp.R, bp.Q, q, smem_raw);
        else
          ypass_body<float, ArDF, K>(bp.pv[1], MODE_SWEEP, bp.S[1], C, bp.R, bp.Q, q, smem_raw);
        __syncthreads();
        // the CTA that completes the sweep's M pass of the problem runs its H stage
        const unsigned per = (unsigned)(bp.Q * C) + HS;
        if (threadIdx.x == 0) {
          __threadfence();
          const unsigned old = atomicAdd(&a.a_done[j], 1u);
          s_item[2] = (HS && old + 1u == (unsigned)(s + 1) * per - HS) ? 1u : 0u;
        }
        __syncthreads();
        if constexpr (HS != 0) {
          if (s_item[2]) {
            if (var == 0) h_stage<K, typename XSmem<float, K>::SV>(bp.pv[0], bp.Q, smem_raw);
            else h_stage<K, double>(bp.pv[0], bp.Q, smem_raw);
            __syncthreads();
            if (threadIdx.x == 0) {
              __threadfence();
              atomicAdd(&a.a_done[j], 1u);
            }
          }
        }
      }
    } else {
      // ---- row pass of row block (g C + rank) of problem j
      r -= A;
      const int j = batch_find(a.boff, a.nprob, r);
      const BatchProb& bp = a.probs[j];
      DevState* st = bp.pv[0].st;
      const int blk = (r - a.boff[j]) * C + crank;
      if (threadIdx.x == 0) batch_wait(&a.a_done[j], (unsigned)(s + 1) * ((unsigned)(bp.Q * C) + HS), st);
      __syncthreads();
      if (blk < bp.nxblk && !*reinterpret_cast<volatile int*>(&st->done)) {
        // the variant of this sweep (the tail that may change it runs after
        // every row block of the sweep has read it)
        const int var = a.force_var >= 0 ? a.force_var : (st->pass_var == VAR_DF ? 1 : 0);
        if (var == 0)
          xpass_body<float, K>(bp.pv[0], MODE_SWEEP, bp.Q, bp.nxblk, blk, smem_raw, &a.t_done[j],
                               (unsigned)(s + 1));
        else
          xpass_body<DF, K>(bp.pv[1], MODE_SWEEP, bp.Q, bp.nxblk, blk, smem_raw, &a.t_done[j],
                            (unsigned)(s + 1));
      }
    }
    __syncthreads();
  }
}

// Launch of the batch kernel of rank k (dispatched to nmf_batch_k*.cu).
cudaError_t launch_batch(int k, const BatchArgs& a, int C, int nclusters, cudaStream_t s);
// Co-resident clusters of the batch kernel of rank k (also sets its
// shared-memory attribute, so that launches under graph capture need none).
int batch_max_clusters(int k, int C);
// Dynamic shared memory of a batch launch: the bodies' budget and the claim words.
size_t batch_smem_bytes(unsigned budget);

template <int K>
void batch_set_attr() {
  static bool done[64] = {false};
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64 || done[dev]) return;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (cudaFuncSetAttribute(batch_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin) == cudaSuccess)
    done[dev] = true;
}

template <int K>
cudaError_t launch_batch_t(const BatchArgs& a, int C, int nclusters, cudaStream_t s) {
  batch_set_attr<K>();
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(nclusters * C), 1, 1);
  cfg.blockDim = dim3(512, 1, 1);
  cfg.dynamicSmemBytes = batch_smem_bytes(a.smem_budget);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, batch_kernel<K>, a);
}

template <int K>
int batch_max_clusters_t(int C) {
  batch_set_attr<K>();
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)C, 1, 1);
  cfg.blockDim = dim3(512, 1, 1);
  cfg.dynamicSmemBytes = (size_t)optin;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, (const void*)batch_kernel<K>, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

}  // namespace nmfgb

// Batch kernels of rank 1..4.
#include "nmf_batch.cuh"

namespace nmfgb {

cudaError_t launch_batch_lo(int k, const BatchArgs& a, int C, int nclusters, cudaStream_t s) {
  switch (k) {
    case 1: return launch_batch_t<1>(a, C, nclusters, s);
    case 2: return launch_batch_t<2>(a, C, nclusters, s);
    case 3: return launch_batch_t<3>(a, C, nclusters, s);
    case 4: return launch_batch_t<4>(a, C, nclusters, s);
    default: return cudaErrorInvalidValue;
  }
}

int batch_max_clusters_lo(int k, int C) {
  switch (k) {
    case 1: return batch_max_clusters_t<1>(C);
    case 2: return batch_max_clusters_t<2>(C);
    case 3: return batch_max_clusters_t<3>(C);
    case 4: return batch_max_clusters_t<4>(C);
    default: return 0;
  }
}

}  // namespace nmfgb

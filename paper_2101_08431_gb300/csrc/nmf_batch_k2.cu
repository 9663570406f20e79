// Batch kernels of rank 5..8 and 16.
#include "nmf_batch.cuh"

namespace nmfgb {

cudaError_t launch_batch_hi(int k, const BatchArgs& a, int C, int nclusters, cudaStream_t s) {
  switch (k) {
    case 5: return launch_batch_t<5>(a, C, nclusters, s);
    case 6: return launch_batch_t<6>(a, C, nclusters, s);
    case 7: return launch_batch_t<7>(a, C, nclusters, s);
    case 8: return launch_batch_t<8>(a, C, nclusters, s);
    case 16: return launch_batch_t<16>(a, C, nclusters, s);
    default: return cudaErrorInvalidValue;
  }
}

int batch_max_clusters_hi(int k, int C) {
  switch (k) {
    case 5: return batch_max_clusters_t<5>(C);
    case 6: return batch_max_clusters_t<6>(C);
    case 7: return batch_max_clusters_t<7>(C);
    case 8: return batch_max_clusters_t<8>(C);
    case 16: return batch_max_clusters_t<16>(C);
    default: return 0;
  }
}

}  // namespace nmfgb

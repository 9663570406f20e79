// Kernel instantiations of the M pass with M stored as double and the
// contraction accumulated in double, for ranks 1..8 and 16.
#include "nmf_launch.cuh"

namespace nmfgb {
bool get_kernels_f64(int k, KernelSet* out) { NMF_FILL_ALL(double, double) }
}  // namespace nmfgb

// Kernel instantiations of the M pass and the row pass with M stored as double, FP64 accumulation,
// for ranks 1..8 and 16.
#include "nmf_launch.cuh"

namespace nmfgb {
bool get_kernels_f64(int k, KernelSet* out) { NMF_FILL_ALL(double, ArF64, double) }
}  // namespace nmfgb

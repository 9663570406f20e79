// Kernel instantiations of the M pass and the row pass with M stored as float, FP64 accumulation,
// for ranks 1..8 and 16.
#include "nmf_launch.cuh"

namespace nmfgb {
bool get_kernels_ref(int k, KernelSet* out) { NMF_FILL_ALL(float, ArF64, double) }
}  // namespace nmfgb

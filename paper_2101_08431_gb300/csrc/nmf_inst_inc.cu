// Kernel instantiations of the M pass and the row pass with M stored as float, incremental contraction (FP32
// change of X and Y against references recorded by a compensated sweep), for ranks 1..8 and 16.
#include "nmf_launch.cuh"

namespace nmfgb {
bool get_kernels_inc(int k, KernelSet* out) { NMF_FILL_ALL(float, ArInc, float) }
}  // namespace nmfgb

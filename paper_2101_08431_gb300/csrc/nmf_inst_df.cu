// Kernel instantiations of the M pass and the row pass with M stored as float, compensated FP32 (double-float) accumulation,
// for ranks 1..8 and 16.
#include "nmf_launch.cuh"

namespace nmfgb {
bool get_kernels_df(int k, KernelSet* out) { NMF_FILL_ALL(float, ArDF, DF) }
}  // namespace nmfgb

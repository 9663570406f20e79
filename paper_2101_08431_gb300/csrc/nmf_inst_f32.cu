// Kernel instantiations of the M pass with M stored as float and the
// contraction accumulated in float, for ranks 1..8 and 16.
#include "nmf_launch.cuh"

namespace nmfgb {
bool get_kernels_f32(int k, KernelSet* out) { NMF_FILL_ALL(float, float) }
}  // namespace nmfgb

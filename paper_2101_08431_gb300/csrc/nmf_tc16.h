// Launch interface of the rank-16 tensor-core M pass (host side).
#pragma once

#include <cstddef>

#include <cuda_runtime.h>

#include "nmf_common.cuh"

namespace nmfgb {

struct Tc16Plan {
  int C;           // cluster size (CTAs per column range)
  int R;           // rows per CTA (multiple of 128)
  int NS;          // slots of the tile ring
  int Q;           // clusters
  int tmem_cols;   // tensor-memory columns allocated per CTA
  size_t smem;     // dynamic shared memory per CTA
};

// Plan for ld rows and m resident columns: the smallest cluster whose ring
// holds four tiles (else the largest ring that fits), as many clusters as are
// co-resident (at most one per tile).  False if no configuration fits.
// Shape of the pass for ld rows and cluster size C (a power of two <= 16):
// rows per CTA, ring slots, tensor-memory columns and shared memory, Q = 0.
// Host arithmetic only (no CUDA call); false if it does not fit.
bool tc16_shape(int ld, int C, int smem_optin, Tc16Plan* out);
bool tc16_plan(int ld, int m, int nsm, int smem_optin, Tc16Plan* out);
cudaError_t tc16_launch(const Problem& p, int mode, const Tc16Plan& L, cudaStream_t s);

}  // namespace nmfgb

// Launch interface of the rank-16 tensor-core M pass (host side).
#pragma once

#include <cstddef>

#include <cuda.h>
#include <cuda_runtime.h>

#include "nmf_common.cuh"

namespace nmfgb {


// The rank-16 pass in three streaming launches (nmf_tc16s.cuh).
namespace tc16s {

// Columns of the ring mirrored after its last column (M holds mcap + MIRROR
// columns; column mcap + j repeats column j for j < MIRROR), so that a tile
// of up to MIRROR consecutive window columns is one box of the tensor map.
constexpr int MIRROR = 128;

// Buffers of the pass (device memory of the handle).
struct Bufs {
  float* Bpart;               // [SB][mcap][16]: B partials, window column order
  unsigned char* Xs;          // split of X: ld/8 blocks of 512 bytes
  unsigned char* Ys;          // split of Y: one block of 512 bytes per 8 window columns
  double* red;                // [gridS][16 * 16 + NYT] block partials of the solve kernels, then their
                              // group partials and the totals
  unsigned* ticket;           // [ticket_count] tickets of the solve kernels' block sums (self-resetting)
  int* perm;                  // [mcap] window columns in the order of their passive sets
  int* perm_tmp;              // [mcap] the order after the first radix pass
  int* keys;                  // [mcap] passive-set mask of each window column
};

struct Plan {
  int SB, SP;                 // row splits of the B-GEMM, column splits of the P-GEMM
  int gridB, gridP, gridS;
  int cpg;                    // consecutive columns per 16-lane group of the FP64 solve kernel (grid gridS)
  int cpgF, gridF;            // the same for the FP32 solve kernel
  int NSB, NSP;               // stages of the two TMA rings
  size_t smemB, smemP;
};

// Tensor maps of M (FP32, ld rows x mcap + MIRROR columns, 128-byte swizzle)
// with the boxes of the two GEMMs: 32 rows x 128 columns and 32 x 64.
struct Maps {
  CUtensorMap b, p;
};

// Sizes of the buffers for ld rows and mcap columns on nsm SMs (bytes).
size_t bpart_bytes(int mcap);
size_t xs_bytes(int ld);
size_t ys_bytes(int mcap);
size_t red_bytes(int nsm);
size_t ticket_count(int nsm);   // unsigned counters behind Bufs::ticket
// the three column-order arrays (perm, perm_tmp, keys), each of this size
size_t perm_bytes(int mcap);
// false when the driver entry point is missing or rejects the shape
bool encode_maps(void* M, int ld, int mcap, Maps* out);
// Plan for ld rows and m resident columns (host arithmetic only); false if
// the shared memory of a CTA cannot hold two stages of either ring.
bool plan(int ld, int m, int nsm, int smem_optin, Plan* out);
// The launches of one M pass: MODE_SWEEP / MODE_KKT: X split, B-GEMM, solves
// (+ P-GEMM for SWEEP); MODE_PRIME: solves (masks, H) and P-GEMM.  Returns
// the number of launches in *nl.
cudaError_t launch(const Problem& p, int mode, const Plan& L, const Bufs& B, const Maps& T, cudaStream_t s,
                   int* nl);

}  // namespace tc16s

// Reference (compensated) and incremental sweeps of the rank-16 refinement
// where n is beyond the cluster-fused FP64-class kernels (nmf_tc16r.cuh).
struct RefPlan {
  int nrbB, slicesB, gridB;   // B partials: row blocks x column slices
  int nrbP, SPd, gridP;       // P partials: 256-row blocks x column splits (= Q of the row pass)
};

namespace tc16r {

enum Pass { REF_PASS = 0, INC_PASS = 1 };
size_t bdf_bytes(int ld, int mcap);
bool plan(int ld, int m, int nsm, RefPlan* out);
// The M pass of a reference sweep (pass REF_PASS: compensated B and P, FP64
// solves; MODE_KKT: B and the terms only; MODE_PRIME: masks, H and P) or of
// an incremental sweep (INC_PASS: tensor-core change terms, FP64 solves).
// *Q: the P partials the row pass sums; *nl: launches.
cudaError_t launch(const Problem& p, int mode, int pass, const RefPlan& R, const tc16s::Plan& L,
                   const tc16s::Bufs& B, const tc16s::Maps& T, double* Bdf, cudaStream_t s, int* nl, int* Q);

}  // namespace tc16r

}  // namespace nmfgb

// Internal interface between the one-problem handle (nmf_api.cu) and the
// batched form (nmf_batch.cu).  Not part of the C ABI.
#pragma once

#include "nmf.h"
#include "nmf_launch.cuh"

namespace nmfgb {

struct HandleInfo {
  int n, ld, k, m, mcap, nsm, smem_optin, nxblk;
  bool store_f32, factors_set;
  int qcap;             // capacity of the partial buffers (column groups)
  int phase;            // host mixed schedule: 0 FP32 passes, 1 refinement passes
  DevState* dSt;        // device control block
  const DevState* hSt;  // its host mirror (valid after handle_sync_state)
  cudaStream_t stream;
};

bool handle_info(nmf_handle* h, HandleInfo* out);
// the problem as variant `var` sees it (kkt_target / stol of that variant)
bool handle_problem(nmf_handle* h, int var, Problem* out);
// the one-problem launch plan of variant `var` (cluster size and rows per CTA)
bool handle_plan(nmf_handle* h, int var, YPlan* out);
const KernelSet* handle_kernels(nmf_handle* h, int var);
nmf_status handle_sync_state(nmf_handle* h);
void handle_set_phase(nmf_handle* h, int phase);
void handle_fill_stats(nmf_handle* h, int measured, int sweeps, int fp64_sweeps, nmf_stats* out);
nmf_status handle_fail(nmf_handle* h, nmf_status s, const char* msg);

// device bytes nmf_create allocates for one problem (admission by footprint)
int64_t handle_footprint(int64_t n, int k, int64_t mcap, bool store_f32, int nsm);

// dynamic membership of a batch (the streaming server): slots are created
// on admission and destroyed on close; inactive slots are left out of sweeps
nmf_status batch_create_empty(void* cuda_stream, nmf_batch** out);
nmf_status batch_add(nmf_batch* b, const nmf_config& cfg, int* slot);
void batch_remove(nmf_batch* b, int j);
void batch_set_active(nmf_batch* b, int j, bool on);
cudaStream_t batch_stream(nmf_batch* b);

}  // namespace nmfgb

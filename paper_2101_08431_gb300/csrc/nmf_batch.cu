// C ABI of the batched form (declared in include/nmf.h): many independent
// problems of uneven n, m and k swept by persistent work-item launches (one
// per (k, cluster size) class, concurrent on forked streams), captured in a
// CUDA graph that is replayed until every problem has stopped.  Each problem
// is an ordinary handle (its ring of columns, factors, partial buffers and
// device control block); the batch adds the work lists, the dependency
// counters, the device-driven mixed schedule and the autotuner.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "nmf_batch.cuh"
#include "nmf_internal.h"

using namespace nmfgb;

namespace {

constexpr int BATCH_CHUNK = 16;                  // sweeps per graph replay
constexpr int STALL_SWEEPS = 256;                // FP32 sweeps without 2% progress before switching
constexpr unsigned SMEM_RESERVE = 128;           // claim words and a flag behind the bodies' budget

// stop flags of every problem at the start of a batched call, and the
// variant each problem resumes with (the schedule's progress record,
// best_rel and since_best, carries over from call to call)
__global__ void batch_reset_kernel(DevState* const* sts, const int* pass_init, int n) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    DevState* st = sts[j];
    st->done = 0;
    st->stop_reason = 0;
    st->pass_var = pass_init[j];
  }
}

// Self-test of the bounded dependency wait: thread 0 waits on a counter that
// nothing increments, with the given poll limit, exactly as a batch item does.
__global__ void wait_selftest_kernel(const unsigned* ctr, DevState* st, long long polls) {
  if (threadIdx.x == 0) batch_wait(ctr, 1u, st, polls);
}

// number of problems that have stopped
__global__ void batch_count_kernel(DevState* const* sts, int n, int* out) {
  __shared__ int c;
  if (threadIdx.x == 0) c = 0;
  __syncthreads();
  int mine = 0;
  for (int j = threadIdx.x; j < n; j += blockDim.x) mine += *reinterpret_cast<volatile int*>(&sts[j]->done) != 0;
  atomicAdd(&c, mine);
  __syncthreads();
  if (threadIdx.x == 0) *out = c;
}

struct Class {
  int k = 0, C = 0;
  std::vector<int> probs;              // batch indices
  BatchProb* dProbs = nullptr;
  int* dOff = nullptr;                 // aoff [np+1] then boff [np+1]
  unsigned* dCnt = nullptr;            // counter, a_done[np], t_done[np]
  int nclusters = 0;
  double work = 0.0;
  cudaStream_t s = nullptr;
  cudaEvent_t ev = nullptr;
  BatchArgs args{};
};

}  // namespace

namespace nmfgb {
cudaError_t launch_batch_lo(int k, const BatchArgs& a, int C, int nclusters, cudaStream_t s);
cudaError_t launch_batch_hi(int k, const BatchArgs& a, int C, int nclusters, cudaStream_t s);
int batch_max_clusters_lo(int k, int C);
int batch_max_clusters_hi(int k, int C);

cudaError_t launch_batch(int k, const BatchArgs& a, int C, int nclusters, cudaStream_t s) {
  return k <= 4 ? launch_batch_lo(k, a, C, nclusters, s) : launch_batch_hi(k, a, C, nclusters, s);
}
int batch_max_clusters(int k, int C) { return k <= 4 ? batch_max_clusters_lo(k, C) : batch_max_clusters_hi(k, C); }
size_t batch_smem_bytes(unsigned budget) { return (size_t)budget + SMEM_RESERVE; }
}  // namespace nmfgb

struct nmf_batch {
  std::vector<nmf_handle*> h;          // problem slots (null: free)
  std::vector<nmf_config> cfg;
  std::vector<char> active;            // slots included in the sweeps
  std::vector<int> plan_idx;           // slots of the current plan, in plan order
  int sts_cap = 0;                     // capacity of dSts / dPassInit
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int nsm = 0, smem_optin = 0;
  int cols_per_item = 64;              // columns per M-pass item (autotuned)
  int stage_cap = 8;                   // stages of the M pass at most (autotuned)
  int force_var = -1;                  // -1 device schedule, 0 FP32 pass, 1 compensated pass
  std::vector<Class> cls;
  bool plan_valid = false;
  cudaEvent_t fork = nullptr;
  cudaGraphExec_t gexec = nullptr;
  int graph_sweeps = 0;
  DevState** dSts = nullptr;
  int* dPassInit = nullptr;
  int* dDone = nullptr;
  int* hDone = nullptr;
  int64_t launches = 0;
  std::string last_error;
  nmf_status poisoned = NMF_OK;
};

namespace {

nmf_status bfail(nmf_batch* b, nmf_status s, const std::string& msg) {
  if (b) {
    b->last_error = msg;
    if (s == NMF_ECUDA || s == NMF_ETIMEOUT) b->poisoned = s;
  }
  return s;
}

#define BCUDA(b, expr)                                                               \
  do {                                                                               \
    cudaError_t e_ = (expr);                                                         \
    if (e_ != cudaSuccess)                                                           \
      return bfail((b), NMF_ECUDA, std::string(#expr ": ") + cudaGetErrorString(e_)); \
  } while (0)

void free_plan(nmf_batch* b) {
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  b->gexec = nullptr;
  b->graph_sweeps = 0;
  for (Class& c : b->cls) {
    cudaFree(c.dProbs);
    cudaFree(c.dOff);
    cudaFree(c.dCnt);
    if (c.ev) cudaEventDestroy(c.ev);
    if (c.s) cudaStreamDestroy(c.s);
  }
  b->cls.clear();
  b->plan_valid = false;
}

// Stages of one variant's M pass for the batch's shared-memory budget.
int batch_stages(const KernelSet& ks, int R, int Q, int m, int cap, unsigned budget) {
  const int cpc = (std::max(m, 1) + Q - 1) / Q;
  const int ntiles = (cpc + ks.TJ - 1) / ks.TJ;
  const long long stage = (long long)ks.TJ * R * ks.tm_size;
  const long long pacc = (long long)R * ks.pacc_row_bytes;
  long long S = ((long long)budget - (long long)ks.small_bytes - pacc) / stage;
  S = std::min<long long>(std::min<long long>(S, cap), std::max(ntiles, 1));
  if (S < (ntiles > 1 ? 2 : 1)) return 0;
  return (int)S;
}

// Group the problems into (k, cluster size) classes, build their device
// work lists and per-problem plans, and size each class's persistent grid.
nmf_status build_plan(nmf_batch* b) {
  free_plan(b);
  const int np = (int)b->h.size();
  const unsigned budget = (unsigned)b->smem_optin - SMEM_RESERVE;
  std::map<std::pair<int, int>, int> index;
  std::vector<std::vector<BatchProb>> hp;
  double total_work = 0.0;
  b->plan_idx.clear();
  for (int j = 0; j < np; ++j) {
    if (!b->h[j] || !b->active[j]) continue;
    b->plan_idx.push_back(j);
    HandleInfo hi;
    handle_info(b->h[j], &hi);
    if (!hi.factors_set) return bfail(b, NMF_ESTATE, "problem " + std::to_string(j) + ": factors not set");
    if (hi.m < 1) return bfail(b, NMF_ESTATE, "problem " + std::to_string(j) + ": no resident columns");
    YPlan L;
    if (!handle_plan(b->h[j], VAR_DF, &L)) return bfail(b, NMF_EINVAL, "no launch plan for a problem");
    const int C = L.C, R = L.R;
    const KernelSet* k0 = handle_kernels(b->h[j], VAR_F32);
    const KernelSet* k1 = handle_kernels(b->h[j], VAR_DF);
    if (!k0 || !k1) return bfail(b, NMF_EINVAL, "no kernels for this rank");
    int Q = (hi.m + b->cols_per_item - 1) / b->cols_per_item;
    Q = std::max(1, std::min(Q, std::min(hi.m, std::min(hi.qcap, b->nsm / C))));
    BatchProb bp{};
    if (!handle_problem(b->h[j], VAR_F32, &bp.pv[0]) || !handle_problem(b->h[j], VAR_DF, &bp.pv[1]))
      return bfail(b, NMF_EINVAL, "no problem view");
    for (int v = 0; v < 2; ++v) {
      bp.pv[v].tab_global = 1;
      // the chain warm start is a one-problem form: batched items start
      // every column from its previous-sweep solution
      if (bp.pv[v].warm == NMF_WARM_CHAIN) bp.pv[v].warm = NMF_WARM_PREV;
      bp.pv[v].auto_mixed = b->force_var < 0 ? 1 : 0;
      bp.pv[v].stall_sweeps = STALL_SWEEPS;
      bp.pv[v].mixed_switch = b->cfg[j].mixed_switch;
    }
    if (b->force_var >= 0) {
      // a fixed pass: every sweep may stop on the targets
      bp.pv[0].kkt_target = bp.pv[1].kkt_target;
      bp.pv[0].kkt_abs_target = bp.pv[1].kkt_abs_target;
      bp.pv[0].stol = bp.pv[1].stol;
    }
    bp.S[0] = batch_stages(*k0, R, Q, hi.m, b->stage_cap, budget);
    bp.S[1] = batch_stages(*k1, R, Q, hi.m, b->stage_cap, budget);
    if (!bp.S[0] || !bp.S[1]) return bfail(b, NMF_EINVAL, "a problem does not fit the batch's shared memory");
    bp.R = R;
    bp.Q = Q;
    bp.nxblk = hi.nxblk;
    bp.nxg = (hi.nxblk + C - 1) / C;
    const auto key = std::make_pair(hi.k, C);
    auto it = index.find(key);
    if (it == index.end()) {
      it = index.emplace(key, (int)b->cls.size()).first;
      b->cls.emplace_back();
      b->cls.back().k = hi.k;
      b->cls.back().C = C;
      hp.emplace_back();
    }
    Class& c = b->cls[it->second];
    c.probs.push_back(j);
    hp[it->second].push_back(bp);
    // CTA time of one sweep (cycles, rough): the M-pass items are paced by
    // their tiles (the NNLS warp's solve and the rows' contraction), the
    // row-pass items by their row blocks
    const int cpc = (hi.m + Q - 1) / Q;
    const double tiles = (double)((cpc + k0->TJ - 1) / k0->TJ);
    const double w = (double)Q * C * tiles * (4000.0 + (double)R * k0->TJ * hi.k / 16.0) + hi.nxblk * 4000.0;
    c.work += w;
    total_work += w;
  }
  for (size_t ci = 0; ci < b->cls.size(); ++ci) {
    Class& c = b->cls[ci];
    const int n = (int)c.probs.size();
    std::vector<int> off(2 * (n + 1), 0);
    for (int i = 0; i < n; ++i) {
      off[i + 1] = off[i] + hp[ci][i].Q;
      off[n + 1 + i + 1] = off[n + 1 + i] + hp[ci][i].nxg;
    }
    BCUDA(b, cudaMalloc(&c.dProbs, sizeof(BatchProb) * n));
    BCUDA(b, cudaMalloc(&c.dOff, sizeof(int) * off.size()));
    BCUDA(b, cudaMalloc(&c.dCnt, sizeof(unsigned) * (1 + 2 * n)));
    BCUDA(b, cudaMemcpy(c.dProbs, hp[ci].data(), sizeof(BatchProb) * n, cudaMemcpyHostToDevice));
    BCUDA(b, cudaMemcpy(c.dOff, off.data(), sizeof(int) * off.size(), cudaMemcpyHostToDevice));
    BCUDA(b, cudaStreamCreateWithFlags(&c.s, cudaStreamNonBlocking));
    BCUDA(b, cudaEventCreateWithFlags(&c.ev, cudaEventDisableTiming));
    const int fit = std::max(1, batch_max_clusters(c.k, c.C));
    const int items = off[n] + off[2 * n + 1];
    // CTAs in proportion to the class's share of the work
    int g = (int)((double)b->nsm * c.work / std::max(total_work, 1.0) / c.C + 0.5);
    c.nclusters = std::max(1, std::min(g, std::min(fit, items)));
    BatchArgs& a = c.args;
    a.probs = c.dProbs;
    a.nprob = n;
    a.aoff = c.dOff;
    a.boff = c.dOff + (n + 1);
    a.counter = c.dCnt;
    a.a_done = c.dCnt + 1;
    a.t_done = c.dCnt + 1 + n;
    a.force_var = b->force_var;
    a.smem_budget = budget;
  }
  // control blocks of the plan's problems, in plan order
  const int npl = (int)b->plan_idx.size();
  if (npl > b->sts_cap) {
    cudaFree(b->dSts);
    cudaFree(b->dPassInit);
    b->dSts = nullptr;
    b->dPassInit = nullptr;
    BCUDA(b, cudaMalloc(&b->dSts, sizeof(DevState*) * npl));
    BCUDA(b, cudaMalloc(&b->dPassInit, sizeof(int) * npl));
    b->sts_cap = npl;
  }
  std::vector<DevState*> sts(npl);
  for (int i = 0; i < npl; ++i) {
    HandleInfo hi;
    handle_info(b->h[b->plan_idx[i]], &hi);
    sts[i] = hi.dSt;
  }
  if (npl) BCUDA(b, cudaMemcpy(b->dSts, sts.data(), sizeof(DevState*) * npl, cudaMemcpyHostToDevice));
  b->plan_valid = true;
  return NMF_OK;
}

// Enqueue `nsweeps` sweeps of every class on the batch stream (fork / join).
nmf_status enqueue_sweeps(nmf_batch* b, int nsweeps) {
  // NMF_DEBUG_BATCH: the class table and each class kernel's time (outside
  // graph capture only)
  static const bool dbg = std::getenv("NMF_DEBUG_BATCH") != nullptr;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(b->stream, &cs);
  const bool timed = dbg && cs == cudaStreamCaptureStatusNone;
  std::vector<cudaEvent_t> evs;
  BCUDA(b, cudaEventRecord(b->fork, b->stream));
  for (Class& c : b->cls) {
    BCUDA(b, cudaStreamWaitEvent(c.s, b->fork, 0));
    BCUDA(b, cudaMemsetAsync(c.dCnt, 0, sizeof(unsigned) * (1 + 2 * c.probs.size()), c.s));
    c.args.nsweeps = nsweeps;
    if (timed) {
      evs.emplace_back();
      cudaEventCreate(&evs.back());
      cudaEventRecord(evs.back(), c.s);
    }
    BCUDA(b, launch_batch(c.k, c.args, c.C, c.nclusters, c.s));
    if (timed) {
      evs.emplace_back();
      cudaEventCreate(&evs.back());
      cudaEventRecord(evs.back(), c.s);
    }
    BCUDA(b, cudaEventRecord(c.ev, c.s));
    BCUDA(b, cudaStreamWaitEvent(b->stream, c.ev, 0));
  }
  if (timed) {
    cudaStreamSynchronize(b->stream);
    for (size_t i = 0; i < b->cls.size(); ++i) {
      const Class& c = b->cls[i];
      float ms = 0.f;
      cudaEventElapsedTime(&ms, evs[2 * i], evs[2 * i + 1]);
      std::fprintf(stderr, "nmf batch class k=%d C=%d problems=%zu clusters=%d sweeps=%d: %.3f ms\n", c.k, c.C,
                   c.probs.size(), c.nclusters, nsweeps, ms);
    }
    for (cudaEvent_t e : evs) cudaEventDestroy(e);
  }
  batch_count_kernel<<<1, 256, 0, b->stream>>>(b->dSts, (int)b->plan_idx.size(), b->dDone);
  BCUDA(b, cudaGetLastError());
  return NMF_OK;
}

// The graph of one replay (BATCH_CHUNK sweeps), captured on first use.
nmf_status run_chunk(nmf_batch* b, int nsweeps) {
  if (nsweeps != BATCH_CHUNK) {   // the remainder of a call: plain launches
    nmf_status s = enqueue_sweeps(b, nsweeps);
    if (s != NMF_OK) return s;
    b->launches += (int64_t)b->cls.size() + 1;
    return NMF_OK;
  }
  if (!b->gexec) {
    cudaGraph_t g = nullptr;
    BCUDA(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    nmf_status s = enqueue_sweeps(b, nsweeps);
    cudaError_t e = cudaStreamEndCapture(b->stream, &g);
    if (s != NMF_OK) {
      if (g) cudaGraphDestroy(g);
      return s;
    }
    if (e != cudaSuccess) return bfail(b, NMF_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(&b->gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return bfail(b, NMF_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    b->graph_sweeps = nsweeps;
  }
  BCUDA(b, cudaGraphLaunch(b->gexec, b->stream));
  b->launches += (int64_t)b->cls.size() + 1;
  return NMF_OK;
}

}  // namespace

namespace nmfgb {

nmf_status batch_create_empty(void* cuda_stream, nmf_batch** out) {
  *out = nullptr;
  nmf_batch* b = new nmf_batch();
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    delete b;
    return NMF_ECUDA;
  }
  cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&b->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  bool ok = true;
  if (cuda_stream) {
    b->stream = static_cast<cudaStream_t>(cuda_stream);
  } else {
    ok &= cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) == cudaSuccess;
    b->own_stream = ok;
  }
  ok &= cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) == cudaSuccess;
  ok &= cudaMalloc(&b->dDone, sizeof(int)) == cudaSuccess;
  ok &= cudaMallocHost(&b->hDone, sizeof(int)) == cudaSuccess;
  if (!ok) {
    nmf_batch_destroy(b);
    return NMF_ECUDA;
  }
  *out = b;
  return NMF_OK;
}

nmf_status batch_add(nmf_batch* b, const nmf_config& cfg, int* slot) {
  nmf_config c = cfg;
  c.cuda_stream = b->stream;   // every problem's work is ordered with the batch launches
  nmf_handle* h = nullptr;
  nmf_status s = nmf_create(&c, &h);
  if (s != NMF_OK) return s;
  int j = 0;
  while (j < (int)b->h.size() && b->h[j]) ++j;
  if (j == (int)b->h.size()) {
    b->h.push_back(nullptr);
    b->cfg.emplace_back();
    b->active.push_back(0);
  }
  b->h[j] = h;
  b->cfg[j] = c;
  b->active[j] = 1;
  b->plan_valid = false;
  *slot = j;
  return NMF_OK;
}

void batch_remove(nmf_batch* b, int j) {
  if (j < 0 || j >= (int)b->h.size() || !b->h[j]) return;
  cudaStreamSynchronize(b->stream);
  nmf_destroy(b->h[j]);
  b->h[j] = nullptr;
  b->active[j] = 0;
  b->plan_valid = false;
}

void batch_set_active(nmf_batch* b, int j, bool on) {
  if (j < 0 || j >= (int)b->h.size() || !b->h[j]) return;
  if ((b->active[j] != 0) != on) b->plan_valid = false;
  b->active[j] = on ? 1 : 0;
}

cudaStream_t batch_stream(nmf_batch* b) { return b->stream; }

}  // namespace nmfgb

extern "C" {

nmf_status nmf_batch_create(const nmf_config* cfgs, int32_t nprob, void* cuda_stream, nmf_batch** out) {
  if (!cfgs || nprob < 1 || !out) return NMF_EINVAL;
  *out = nullptr;
  for (int j = 0; j < nprob; ++j)
    if (cfgs[j].prec != NMF_PREC_MIXED || cfgs[j].k < 1 || (cfgs[j].k > 8 && cfgs[j].k != 16))
      return NMF_EINVAL;
  nmf_batch* b = nullptr;
  nmf_status s = batch_create_empty(cuda_stream, &b);
  if (s != NMF_OK) return s;
  for (int j = 0; j < nprob; ++j) {
    int slot = -1;
    s = batch_add(b, cfgs[j], &slot);
    if (s != NMF_OK) {
      nmf_batch_destroy(b);
      return s;
    }
  }
  *out = b;
  return NMF_OK;
}

nmf_status nmf_batch_destroy(nmf_batch* b) {
  if (!b) return NMF_OK;
  if (b->stream) cudaStreamSynchronize(b->stream);
  free_plan(b);
  for (nmf_handle* h : b->h)
    if (h) nmf_destroy(h);
  cudaFree(b->dSts);
  cudaFree(b->dPassInit);
  cudaFree(b->dDone);
  if (b->hDone) cudaFreeHost(b->hDone);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
  return NMF_OK;
}

int32_t nmf_batch_size(const nmf_batch* b) { return b ? (int32_t)b->h.size() : 0; }

nmf_handle* nmf_batch_problem(nmf_batch* b, int32_t j) {
  if (!b || j < 0 || j >= (int32_t)b->h.size()) return nullptr;
  return b->h[j];   // null for a free slot
}

nmf_status nmf_batch_append_columns(nmf_batch* b, int32_t j, const void* cols, int64_t ncols, int64_t ld,
                                    int32_t dtype, int32_t on_device) {
  if (!b || j < 0 || j >= (int32_t)b->h.size() || !b->h[j]) return NMF_EINVAL;
  if (b->poisoned) return b->poisoned;
  b->plan_valid = false;
  return nmf_append_columns(b->h[j], cols, ncols, ld, dtype, on_device);
}

nmf_status nmf_batch_set_factors(nmf_batch* b, int32_t j, const double* X, const double* Y,
                                 int32_t on_device) {
  if (!b || j < 0 || j >= (int32_t)b->h.size() || !b->h[j]) return NMF_EINVAL;
  if (b->poisoned) return b->poisoned;
  b->plan_valid = false;
  return nmf_set_factors(b->h[j], X, Y, on_device);
}

nmf_status nmf_batch_get_factors(nmf_batch* b, int32_t j, double* X, double* Y, uint32_t* xmask,
                                 uint32_t* ymask, int32_t on_device) {
  if (!b || j < 0 || j >= (int32_t)b->h.size() || !b->h[j]) return NMF_EINVAL;
  if (b->poisoned) return b->poisoned;
  return nmf_get_factors(b->h[j], X, Y, xmask, ymask, on_device);
}

nmf_status nmf_batch_set_pass_mode(nmf_batch* b, int32_t mode) {
  if (!b || (mode != -1 && mode != 0 && mode != 2)) return NMF_EINVAL;
  const int fv = mode < 0 ? -1 : (mode == 0 ? 0 : 1);
  if (fv != b->force_var) b->plan_valid = false;
  b->force_var = fv;
  return NMF_OK;
}

nmf_status nmf_batch_set_schedule(nmf_batch* b, int32_t cols_per_item, int32_t stage_cap) {
  if (!b || cols_per_item < 1 || stage_cap < 1 || stage_cap > 8) return NMF_EINVAL;
  if (cols_per_item != b->cols_per_item || stage_cap != b->stage_cap) b->plan_valid = false;
  b->cols_per_item = cols_per_item;
  b->stage_cap = stage_cap;
  return NMF_OK;
}

nmf_status nmf_batch_sweep(nmf_batch* b, int32_t max_sweeps, nmf_stats* stats, int32_t* sweeps_run) {
  if (!b || max_sweeps < 0) return NMF_EINVAL;
  if (b->poisoned) return b->poisoned;
  if (!b->plan_valid) {
    nmf_status s = build_plan(b);
    if (s != NMF_OK) return s;
  }
  const int np = (int)b->plan_idx.size();
  if (np == 0) {
    if (sweeps_run) *sweeps_run = 0;
    return NMF_OK;
  }
  int cap = max_sweeps;
  if (cap == 0)
    for (int jj : b->plan_idx) cap = std::max(cap, std::max(1, (int)b->cfg[jj].max_sweeps));
  // resume every problem: its schedule phase, and the iterate index before the call
  std::vector<int> pass_init(np), iter0(np), fp0(np);
  for (int i = 0; i < np; ++i) {
    const int j = b->plan_idx[i];
    nmf_status s = handle_sync_state(b->h[j]);
    if (s != NMF_OK) return bfail(b, s, "problem " + std::to_string(j) + ": state");
    HandleInfo hi;
    handle_info(b->h[j], &hi);
    iter0[i] = hi.hSt->iter;
    fp0[i] = hi.hSt->fp64_sweeps;
    pass_init[i] = (b->force_var == 1 || (b->force_var < 0 && hi.phase == 1)) ? VAR_DF : VAR_F32;
  }
  BCUDA(b, cudaMemcpyAsync(b->dPassInit, pass_init.data(), sizeof(int) * np, cudaMemcpyHostToDevice, b->stream));
  batch_reset_kernel<<<(np + 255) / 256, 256, 0, b->stream>>>(b->dSts, b->dPassInit, np);
  BCUDA(b, cudaGetLastError());
  b->launches++;
  int done_sweeps = 0;
  bool all_done = false;
  while (done_sweeps < cap) {
    const int chunk = std::min(BATCH_CHUNK, cap - done_sweeps);
    nmf_status s = run_chunk(b, chunk);
    if (s != NMF_OK) return s;
    BCUDA(b, cudaMemcpyAsync(b->hDone, b->dDone, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
    BCUDA(b, cudaStreamSynchronize(b->stream));
    done_sweeps += chunk;
    if (*b->hDone >= np) {
      all_done = true;
      break;
    }
  }
  nmf_status worst = NMF_OK;
  for (int i = 0; i < np; ++i) {
    const int j = b->plan_idx[i];
    nmf_status s = handle_sync_state(b->h[j]);
    HandleInfo hi;
    handle_info(b->h[j], &hi);
    if (s == NMF_ETIMEOUT || s == NMF_ECUDA) return bfail(b, s, "problem " + std::to_string(j) + ": device wait");
    if (s != NMF_OK && worst == NMF_OK) worst = s;
    handle_set_phase(b->h[j], hi.hSt->pass_var == VAR_DF ? 1 : 0);
    if (stats) {
      const int it = hi.hSt->iter;
      const bool stop_kkt = hi.hSt->done && hi.hSt->stop_reason == 1;
      const int worked = (it - iter0[i]) + (stop_kkt ? 1 : 0);
      const int measured = stop_kkt ? it : it - 1;
      handle_fill_stats(b->h[j], measured, worked, -1, &stats[j]);
      stats[j].fp64_sweeps = hi.hSt->fp64_sweeps - fp0[i];
    }
  }
  if (sweeps_run) *sweeps_run = done_sweeps;
  if (worst != NMF_OK) return worst;
  if (max_sweeps == 0 && !all_done) return bfail(b, NMF_ENOTCONV, "sweep cap reached");
  return NMF_OK;
}

nmf_status nmf_batch_autotune(nmf_batch* b, int32_t trial_sweeps, int32_t* cols_per_item,
                              int32_t* stage_cap, double* best_ms_per_sweep) {
  if (!b || trial_sweeps < 1) return NMF_EINVAL;
  if (b->poisoned) return b->poisoned;
  // Candidate schedules: columns per M-pass item (the tile of column groups,
  // hence the number of P partials the row pass reduces) and the stage cap
  // of the TMA pipeline.  Each is timed over trial_sweeps FP32-pass sweeps
  // (the tuning sweeps are ordinary sweeps of the iteration).
  static const int kCols[] = {16, 32, 64, 128, 256};
  static const int kStages[] = {2, 8};
  const int keep_force = b->force_var;
  b->force_var = 0;
  b->plan_valid = false;
  cudaEvent_t e0, e1;
  BCUDA(b, cudaEventCreate(&e0));
  BCUDA(b, cudaEventCreate(&e1));
  double best = 1e30;
  int bc = b->cols_per_item, bs = b->stage_cap;
  for (int c : kCols) {
    for (int sc : kStages) {
      b->cols_per_item = c;
      b->stage_cap = sc;
      b->plan_valid = false;
      nmf_status s = build_plan(b);
      if (s != NMF_OK) continue;
      std::vector<int> pass_init(b->plan_idx.size(), VAR_F32);
      BCUDA(b, cudaMemcpyAsync(b->dPassInit, pass_init.data(), sizeof(int) * pass_init.size(),
                               cudaMemcpyHostToDevice, b->stream));
      batch_reset_kernel<<<((int)pass_init.size() + 255) / 256, 256, 0, b->stream>>>(
          b->dSts, b->dPassInit, (int)pass_init.size());
      s = enqueue_sweeps(b, 1);   // warm-up (attributes, caches)
      if (s != NMF_OK) return s;
      BCUDA(b, cudaEventRecord(e0, b->stream));
      s = enqueue_sweeps(b, trial_sweeps);
      if (s != NMF_OK) return s;
      BCUDA(b, cudaEventRecord(e1, b->stream));
      BCUDA(b, cudaEventSynchronize(e1));
      float ms = 0.f;
      BCUDA(b, cudaEventElapsedTime(&ms, e0, e1));
      b->launches += 2 * ((int64_t)b->cls.size() + 1) + 1;
      const double per = ms / trial_sweeps;
      if (per < best) {
        best = per;
        bc = c;
        bs = sc;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->cols_per_item = bc;
  b->stage_cap = bs;
  b->force_var = keep_force;
  b->plan_valid = false;
  if (cols_per_item) *cols_per_item = bc;
  if (stage_cap) *stage_cap = bs;
  if (best_ms_per_sweep) *best_ms_per_sweep = best;
  return NMF_OK;
}

nmf_status nmf_selftest_bounded_wait(int64_t polls, void* cuda_stream) {
  if (polls < 1 || polls > (int64_t(1) << 24)) return NMF_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  unsigned* ctr = nullptr;
  DevState* st = nullptr;
  DevState hst;
  if (cudaMalloc(&ctr, sizeof(unsigned)) != cudaSuccess) return NMF_ENOMEM;
  if (cudaMalloc(&st, sizeof(DevState)) != cudaSuccess) {
    cudaFree(ctr);
    return NMF_ENOMEM;
  }
  nmf_status out = NMF_ECUDA;
  if (cudaMemsetAsync(ctr, 0, sizeof(unsigned), s) == cudaSuccess &&
      cudaMemsetAsync(st, 0, sizeof(DevState), s) == cudaSuccess) {
    wait_selftest_kernel<<<1, 32, 0, s>>>(ctr, st, (long long)polls);
    if (cudaGetLastError() == cudaSuccess &&
        cudaMemcpyAsync(&hst, st, sizeof(DevState), cudaMemcpyDeviceToHost, s) == cudaSuccess &&
        cudaStreamSynchronize(s) == cudaSuccess)
      out = (hst.err & ERR_TIMEOUT) && hst.done ? NMF_ETIMEOUT : NMF_OK;
  }
  cudaFree(ctr);
  cudaFree(st);
  return out;
}

int64_t nmf_batch_launch_count(const nmf_batch* b) { return b ? b->launches : 0; }

const char* nmf_batch_last_error(const nmf_batch* b) { return b ? b->last_error.c_str() : "null batch"; }

}  // extern "C"

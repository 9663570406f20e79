// C ABI of the GB300 streaming-NMF library (declared in include/nmf.h):
// handle life cycle, the resident column ring, priming, the sweep driver with
// the mixed-precision schedule, and the read-only objective / KKT pass.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>

#include "nmf.h"
#include "nmf_internal.h"
#include "nmf_tc16.h"

using namespace nmfgb;

namespace {

constexpr int CHUNK = 32;                  // sweeps between host checks
constexpr int STALL_CHUNKS = 8;            // MIXED: FP32 passes without progress before switching
constexpr int APPEND_STAGE_COLS = 256;     // host-to-device staging width

int round_up(int v, int a) { return (v + a - 1) / a * a; }

// ---------------------------------------------------------------------------
// small kernels
// ---------------------------------------------------------------------------

// Copy one staged column block into the ring (converting the element type),
// zero the padding rows, record ||M_{:,j}||^2 and seed y_j from *seed.
template <typename TS, typename TM>
__global__ void append_kernel(const TS* __restrict__ src, long long ld_src, int ncols, TM* M, int ld,
                              int n, int mcap, int first_phys, double* colsq, const double* seed,
                              const uint32_t* seed_mask, DevState* st, double* Y0, double* Y1,
                              uint32_t* ym0, uint32_t* ym1, int k, unsigned* nonfinite, int mirror) {
  const int c = blockIdx.x;
  if (c >= ncols) return;
  int phys = first_phys + c;
  if (phys >= mcap) phys -= mcap;
  const TS* s = src + (size_t)c * ld_src;
  TM* d = M + (size_t)phys * ld;
  // the first `mirror` columns of the ring are repeated after its last one
  TM* d2 = phys < mirror ? M + (size_t)(mcap + phys) * ld : nullptr;
  double acc = 0.0;
  unsigned bad = 0;
  for (int i = threadIdx.x; i < ld; i += blockDim.x) {
    TM v = TM(0);
    if (i < n) {
      v = (TM)s[i];
      if (!isfinite((double)v)) ++bad;
    }
    d[i] = v;
    if (d2) d2[i] = v;
    acc = fma((double)v, (double)v, acc);
  }
  __shared__ double red[32];
  acc = warp_sum(acc);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) red[warp] = acc;
  if (bad) atomicAdd(nonfinite, bad);
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    colsq[phys] = t;
  }
  if (threadIdx.x < k) {
    const int cur = st->iter & 1;
    double* Y = cur ? Y1 : Y0;
    uint32_t* ym = cur ? ym1 : ym0;
    Y[(size_t)phys * k + threadIdx.x] = seed ? seed[threadIdx.x] : 0.0;
    if (threadIdx.x == 0) ym[phys] = seed_mask ? *seed_mask : 0u;
  }
}

// seed <- y and mask of the physical column `phys` of the current buffers
__global__ void seed_kernel(DevState* st, const double* Y0, const double* Y1, const uint32_t* ym0,
                            const uint32_t* ym1, int phys, int k, double* seed, uint32_t* seed_mask) {
  const int cur = st->iter & 1;
  const double* Y = cur ? Y1 : Y0;
  const uint32_t* ym = cur ? ym1 : ym0;
  for (int a = threadIdx.x; a < k; a += blockDim.x) seed[a] = Y[(size_t)phys * k + a];
  if (threadIdx.x == 0) *seed_mask = ym[phys];
}

// ||M||^2 of the resident window (fixed order) and, with invalidate, of the
// X-half terms of the current iterate (P = M Y^T changed).
__global__ void msq_kernel(DevState* st, const double* colsq, int head, int m, int mcap, int invalidate = 1) {
  __shared__ double red[256];
  double t = 0.0;
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    int ph = head + j;
    if (ph >= mcap) ph -= mcap;
    t += colsq[ph];
  }
  red[threadIdx.x] = t;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    st->msq = red[0];
    if (invalidate) {
      st->xiter[0][XT_VALID] = 0.0;
      st->xiter[1][XT_VALID] = 0.0;
    }
  }
}

// Statistics of the current iterate after a read-only (MODE_KKT) M pass.
__global__ void kkt_stats_kernel(Problem p, int Q, double* out) {
  __shared__ double yfin[NYT];
  const int tid = threadIdx.x;
  DevState* st = p.st;
  if (tid < NYT) {
    double r = 0.0;
    for (int qq = 0; qq < Q; ++qq) {
      const double w = p.Yterms[(size_t)qq * NYT + tid];
      r = (tid == YT_YMAX) ? fmax(r, w) : r + w;
    }
    yfin[tid] = r;
  }
  __syncthreads();
  if (tid < 32) {
    const int iter = st->iter;
    combine_stats_warp(yfin, st->xiter[iter & 1], st->msq, -1.0, iter, p.fp64_pass, out);
  }
}

// Column sharding: this rank's contribution to the X half of a sweep, in
// fixed order -- P = sum over the Q column groups of the partials of
// M_shard Y_shard^T (n x k), H = Y_shard Y_shard^T, the Y-half terms, and the
// shard's ||M||^2 -- into out[]; the largest y into outmax[0].
template <typename TA>
__global__ void shard_export_kernel(Problem p, int Q, double* out, double* outmax) {
  using PO = PartOps<TA>;
  const TA* Pp = static_cast<const TA*>(p.Ppart);
  const int k = p.k;
  const long long nk = (long long)p.n * k;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nk;
       e += (long long)gridDim.x * blockDim.x) {
    const long long row = e / k, a = e % k;
    TA acc = PO::zero();
    for (int q = 0; q < Q; ++q) acc = PO::add(acc, Pp[((size_t)q * p.ld + row) * k + a]);
    out[e] = PO::to_double(acc);
  }
  if (blockIdx.x != 0) return;
  for (int e = threadIdx.x; e < k * k + NYT + 1; e += blockDim.x) {
    double r = 0.0;
    if (e < k * k) {
      for (int q = 0; q < Q; ++q) r += p.Hpart[(size_t)q * k * k + e];
    } else if (e < k * k + NYT) {
      const int t = e - k * k;
      for (int q = 0; q < Q; ++q) {
        const double w = p.Yterms[(size_t)q * NYT + t];
        r = (t == YT_YMAX) ? fmax(r, w) : r + w;
      }
      if (t == YT_YMAX) {
        outmax[0] = r;
        r = 0.0;
      }
    } else {
      for (int j = 0; j < p.m; ++j) r += p.colsq[wrap_col(p.head, j, p.mcap)];
    }
    out[nk + e] = r;
  }
}

// The all-reduced buffers into the row pass's inputs (one partial, FP64):
// P rows, H, the Y-half terms (the largest y from inmax), and the global
// ||M||^2 into the control block for the objective of this sweep's record.
__global__ void shard_import_kernel(const double* in, const double* inmax, int n, int k, double* P, double* H,
                                    double* Yterms, DevState* st) {
  const long long nk = (long long)n * k;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nk;
       e += (long long)gridDim.x * blockDim.x)
    P[e] = in[e];
  if (blockIdx.x != 0) return;
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) H[e] = in[nk + e];
  for (int t = threadIdx.x; t < NYT; t += blockDim.x) Yterms[t] = (t == YT_YMAX) ? inmax[0] : in[nk + k * k + t];
  if (threadIdx.x == 0) {
    st->msq = in[nk + k * k + NYT];
    // the X-half terms of iterate 0 came from the priming pass over this
    // rank's columns alone: its record is marked unmeasured
    if (st->iter == 0) st->xiter[0][XT_VALID] = 0.0;
  }
}

__global__ void clamp_kernel(double* v, long long count) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x)
    if (!(v[i] > 0.0)) v[i] = 0.0;
}

}  // namespace

// ---------------------------------------------------------------------------
// handle
// ---------------------------------------------------------------------------
struct nmf_handle {
  nmf_config cfg{};
  int dev = 0, nsm = 0, smem_optin = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int n = 0, ld = 0, k = 0, mcap = 0, m = 0, head = 0;
  bool store_f32 = true;
  void* dM = nullptr;
  double* dX[2] = {nullptr, nullptr};
  float* dX32[2] = {nullptr, nullptr};
  float* dX32lo[2] = {nullptr, nullptr};
  double* dY[2] = {nullptr, nullptr};
  uint32_t* dYm[2] = {nullptr, nullptr};
  uint32_t* dXm[2] = {nullptr, nullptr};
  double* dG = nullptr;
  double* dGtab = nullptr;
  int* dGok = nullptr;
  double* dHg = nullptr;
  double* dHtab = nullptr;
  int* dHok = nullptr;
  double* dColsq = nullptr;
  void* dPpart = nullptr;
  double* dHpart = nullptr;
  double* dYterms = nullptr;
  double* dXpart = nullptr;
  unsigned* dXgt = nullptr;      // k = 16: group tickets of the row pass
  DevState* dSt = nullptr;
  double* dKkt = nullptr;
  double* dSeed = nullptr;
  uint32_t* dSeedMask = nullptr;
  unsigned* dNonfinite = nullptr;
  void* dStage = nullptr;
  size_t stage_bytes = 0;
  // references and FP32 change of X for the incremental refinement sweeps
  double* dBref = nullptr;
  double* dYref = nullptr;
  double* dPref = nullptr;
  double* dXref = nullptr;
  float* dXd32[2] = {nullptr, nullptr};
  bool inc_ok = false;            // the incremental pass has a plan for this shape
  // column sharding: exchange staging (out: sum part, max part) and the
  // imported row-pass inputs
  double* dShard = nullptr;
  double* dShardP = nullptr;
  int shard_var = -1;             // pass variant of the pending Y half (-1: none)
  DevState* hSt = nullptr;      // pinned mirror
  double* hKkt = nullptr;
  unsigned* hNonfinite = nullptr;
  int nxblk = 0;
  bool factors_set = false;
  nmf_status poisoned = NMF_OK;
  int phase = 0;                // MIXED: 0 FP32 passes, 1 FP64-accumulated passes
  int forced_mode = -1;
  double best_rel = -1.0;       // MIXED schedule: best FP32-pass relative KKT so far
  int chunks_since_best = 0;
  bool snap_valid = false;      // hSt mirrors the device state
  int64_t launches = 0;
  std::string last_error;
  KernelSet ks[NVAR]{};
  bool has[NVAR] = {};
  int max_clusters[NVAR][4] = {};   // per variant, cluster size 1, 2, 4, 8 (full smem)
  // CUDA graph of one chunk of sweeps per variant, keyed by the ring state
  // it was captured with (m, head); a signature is first run uncaptured
  struct ChunkGraph {
    cudaGraphExec_t exec = nullptr;
    int m = -1, head = -1;         // signature of exec
    int seen_m = -1, seen_head = -1;   // last signature run uncaptured
  };
  ChunkGraph graphs[NVAR];
  // rank 16, mixed precision: the FP32-class pass runs on the tensor cores
  bool tc16 = false;
  int mirror = 0;                 // columns mirrored after the ring (tensor-core pass)
  tc16s::Plan tc16_L{};           // plan of the last launch, for tc16_m resident columns
  int tc16_m = -1;
  tc16s::Bufs tcb{};              // buffers of the tensor-core pass
  tc16s::Maps tcmaps{};           // its tensor maps of M
  // rank 16 beyond the rows of the cluster-fused FP64-class kernels: the
  // refinement runs the compensated reference and incremental passes
  bool tc_refine = false;
  RefPlan tcR{};
  double* dBdf = nullptr;         // B partials of the reference pass
  bool refine_ok = true;          // the FP64-class M passes have a plan for n
  // per-kernel timing (event triplets around each sweep's two launches)
  bool timing = false;
  static constexpr int NEV = 512;
  cudaEvent_t ev[NEV][3] = {};
  int ev_var[NEV] = {};
  int nev = 0;
  double y_ms = 0.0, x_ms = 0.0;
  int64_t y_launches = 0, x_launches = 0;
  double yv_ms[NVAR] = {}, xv_ms[NVAR] = {};   // the same, per pass variant
  int64_t v_launches[NVAR] = {};
};

namespace {

nmf_status fail(nmf_handle* h, nmf_status s, const std::string& msg) {
  if (h) {
    h->last_error = msg;
    if (s == NMF_ECUDA || s == NMF_ETIMEOUT) h->poisoned = s;
  }
  return s;
}

#define CUDA_TRY(h, expr)                                                           \
  do {                                                                              \
    cudaError_t e_ = (expr);                                                        \
    if (e_ != cudaSuccess)                                                          \
      return fail((h), NMF_ECUDA, std::string(#expr ": ") + cudaGetErrorString(e_)); \
  } while (0)

bool make_plan(const nmf_handle* h, int var, YPlan* L) {
  const KernelSet& K = h->ks[var];
  const int rmax = K.rows;
  int C = 1, R = 0;
  for (C = 1; C <= 8; C <<= 1) {
    R = round_up((h->ld + C - 1) / C, 32);
    if (R <= rmax) break;
  }
  if (C > 8) return false;
  int Q = std::max(1, std::min(h->nsm / C, std::max(h->m, 1)));
  // the chain warm start runs the whole window in order on one cluster
  if (h->cfg.warm_start == NMF_WARM_CHAIN && h->k <= 8) Q = 1;
  const int cpc = (std::max(h->m, 1) + Q - 1) / Q;
  const int ntiles = (cpc + K.TJ - 1) / K.TJ;
  const size_t stage = (size_t)K.TJ * R * K.tm_size;
  const size_t pacc = (size_t)R * K.pacc_row_bytes;
  long long S = ((long long)h->smem_optin - (long long)K.small_bytes - (long long)pacc) / (long long)stage;
  if (S > 8) S = 8;
  if (S > ntiles) S = ntiles;
  // the pipeline refills the stage of tile t-1 while tile t is staged: two
  // stages at least whenever there is more than one tile
  if (S < (ntiles > 1 ? 2 : 1)) return false;
  const size_t smem = K.small_bytes + (size_t)S * stage + pacc;
  // persistent grid: never more clusters than the device holds at once
  const int ci = C == 1 ? 0 : (C == 2 ? 1 : (C == 4 ? 2 : 3));
  const int fit = h->max_clusters[var][ci];
  if (fit > 0 && Q > fit) Q = fit;
  L->C = C;
  L->R = R;
  L->Q = Q;
  L->S = (int)S;
  L->smem = smem;
  static const bool debug_plan = std::getenv("NMF_DEBUG_PLAN") != nullptr;
  if (debug_plan)
    std::fprintf(stderr, "nmf plan: variant %d C=%d R=%d Q=%d S=%d smem=%zu fit=%d\n", var, C, R, Q,
                 (int)S, smem, fit);
  return true;
}

Problem make_problem(const nmf_handle* h, int var) {
  Problem p{};
  p.n = h->n;
  p.m = h->m;
  p.k = h->k;
  p.ld = h->ld;
  p.mcap = h->mcap;
  p.head = h->head;
  p.M = h->dM;
  for (int b = 0; b < 2; ++b) {
    p.X[b] = h->dX[b];
    p.X32[b] = h->dX32[b];
    p.X32lo[b] = h->dX32lo[b];
    p.Y[b] = h->dY[b];
    p.ymask[b] = h->dYm[b];
    p.xmask[b] = h->dXm[b];
  }
  p.G = h->dG;
  p.Gtab = h->dGtab;
  p.Gok = h->dGok;
  p.Hg = h->dHg;
  p.Htab = h->dHtab;
  p.Hok = h->dHok;
  p.colsq = h->dColsq;
  p.Ppart = h->dPpart;
  p.Hpart = h->dHpart;
  p.Yterms = h->dYterms;
  p.Xpart = h->dXpart;
  p.xgt = h->dXgt;
  p.st = h->dSt;
  p.Bref = h->dBref;
  p.Yref = h->dYref;
  p.Pref = h->dPref;
  p.Xref = h->dXref;
  p.Xd32[0] = h->dXd32[0];
  p.Xd32[1] = h->dXd32[1];
  p.inc = var == VAR_INC ? 1 : 0;
  p.record_refs = 0;
  p.tab_global = 0;
  // k <= 8: the row pass's last block builds the subset table of the new G
  // (beside the statistics) for the next M pass, whose NNLS warp would
  // otherwise build it before its first solve
  p.gtab_tail = h->k <= 8 ? 1 : 0;
  p.warm = h->cfg.warm_start;   // 0 cold, 1 previous sweep, 2 chain
  p.fp64_pass = var != VAR_F32;
  const bool final_phase = !(h->store_f32 && var == VAR_F32);
  p.kkt_target = final_phase ? h->cfg.kkt_target : 0.0;
  p.kkt_abs_target = final_phase ? h->cfg.kkt_abs_target : 0.0;
  p.stol = final_phase ? h->cfg.stol : 0.0;
  return p;
}

// Fold recorded event triplets into the timing totals (synchronises them).
nmf_status drain_timing(nmf_handle* h) {
  for (int i = 0; i < h->nev; ++i) {
    float a = 0.f, b = 0.f;
    CUDA_TRY(h, cudaEventSynchronize(h->ev[i][2]));
    CUDA_TRY(h, cudaEventElapsedTime(&a, h->ev[i][0], h->ev[i][1]));
    CUDA_TRY(h, cudaEventElapsedTime(&b, h->ev[i][1], h->ev[i][2]));
    h->y_ms += a;
    h->x_ms += b;
    h->yv_ms[h->ev_var[i]] += a;
    h->xv_ms[h->ev_var[i]] += b;
    h->v_launches[h->ev_var[i]]++;
  }
  h->y_launches += h->nev;
  h->x_launches += h->nev;
  h->nev = 0;
  return NMF_OK;
}

// Plan of the rank-16 tensor-core pass for the current window (kept until
// the number of resident columns changes); *Q: the partials of P it writes.
nmf_status tc_plan(nmf_handle* h, int* Q) {
  if (h->tc16_m != h->m) {
    if (!tc16s::plan(h->ld, h->m, h->nsm, h->smem_optin, &h->tc16_L) ||
        (h->tc_refine && !tc16r::plan(h->ld, h->m, h->nsm, &h->tcR)))
      return fail(h, NMF_EINVAL, "no tensor-core launch plan for this shape");
    h->tc16_m = h->m;
  }
  *Q = h->tc16_L.SP;
  return NMF_OK;
}

// One sweep (M pass + row pass) or, with mode PRIME, the priming pair;
// record: this (compensated) sweep records the incremental references.
nmf_status launch_pair(nmf_handle* h, int var, int mode, bool record = false) {
  YPlan L{};
  const bool use_tc = h->tc16 && (var == VAR_F32 || h->tc_refine);
  if (use_tc) {
    nmf_status ts = tc_plan(h, &L.Q);
    if (ts != NMF_OK) return ts;
  } else if (!make_plan(h, var, &L)) {
    return fail(h, NMF_EINVAL, "no launch plan for this shape");
  }
  Problem p = make_problem(h, var);
  p.record_refs = record ? 1 : 0;
  // the row pass of the rank-16 refinement passes: FP64 partials (reference
  // sweeps) or FP32 partials of the change (incremental sweeps)
  const int xvar = (use_tc && var != VAR_F32) ? (var == VAR_INC ? VAR_F32 : VAR_REF) : var;
  const bool timed = h->timing && mode == MODE_SWEEP;
  if (timed && h->nev == nmf_handle::NEV) {
    nmf_status s = drain_timing(h);
    if (s != NMF_OK) return s;
  }
  if (timed) {
    if (!h->ev[h->nev][0])
      for (int j = 0; j < 3; ++j) CUDA_TRY(h, cudaEventCreate(&h->ev[h->nev][j]));
    h->ev_var[h->nev] = var;
    CUDA_TRY(h, cudaEventRecord(h->ev[h->nev][0], h->stream));
  }
  int nl = 1;
  if (use_tc && var == VAR_F32)
    CUDA_TRY(h, tc16s::launch(p, mode, h->tc16_L, h->tcb, h->tcmaps, h->stream, &nl));
  else if (use_tc)
    CUDA_TRY(h, tc16r::launch(p, mode, var == VAR_INC ? tc16r::INC_PASS : tc16r::REF_PASS, h->tcR, h->tc16_L, h->tcb,
                              h->tcmaps, h->dBdf, h->stream, &nl, &L.Q));
  else
    CUDA_TRY(h, h->ks[var].ypass(p, mode, L, h->stream));
  if (timed) CUDA_TRY(h, cudaEventRecord(h->ev[h->nev][1], h->stream));
  CUDA_TRY(h, h->ks[xvar].xpass(p, mode, L.Q, h->nxblk, h->stream));
  if (timed) {
    CUDA_TRY(h, cudaEventRecord(h->ev[h->nev][2], h->stream));
    h->nev++;
  }
  h->launches += nl + 1;
  return NMF_OK;
}

// The passes of one chunk of sweeps: `first` for its first sweep (which
// records the incremental references when `record`), `rest` for the others.
struct ChunkPlan {
  int first, rest;
  bool record;
};

// CHUNK sweeps of a plan: replay of the captured graph when its signature
// matches, otherwise plain launches (captured the second time the same
// signature is seen).  Graphs are kept per plan (indexed by `rest`).
nmf_status launch_chunk(nmf_handle* h, const ChunkPlan& cp, int chunk) {
  nmf_handle::ChunkGraph& g = h->graphs[cp.rest];
  auto launch_all = [&]() -> nmf_status {
    for (int i = 0; i < chunk; ++i) {
      nmf_status s = launch_pair(h, i == 0 ? cp.first : cp.rest, MODE_SWEEP, i == 0 && cp.record);
      if (s != NMF_OK) return s;
    }
    return NMF_OK;
  };
  const bool graphable = !h->timing && chunk == CHUNK;
  if (graphable && g.exec && g.m == h->m && g.head == h->head) {
    CUDA_TRY(h, cudaGraphLaunch(g.exec, h->stream));
    h->launches += 2 * chunk;
    return NMF_OK;
  }
  if (graphable && g.seen_m == h->m && g.seen_head == h->head) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    g.exec = nullptr;
    cudaGraph_t graph = nullptr;
    CUDA_TRY(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    const int64_t l0 = h->launches;
    nmf_status s = launch_all();
    h->launches = l0;
    const cudaError_t e = cudaStreamEndCapture(h->stream, &graph);
    if (s != NMF_OK) {
      if (graph) cudaGraphDestroy(graph);
      return s;
    }
    if (e != cudaSuccess) return fail(h, NMF_ECUDA, std::string("sweep graph capture: ") + cudaGetErrorString(e));
    const cudaError_t e2 = cudaGraphInstantiate(&g.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e2 != cudaSuccess) return fail(h, NMF_ECUDA, std::string("sweep graph: ") + cudaGetErrorString(e2));
    g.m = h->m;
    g.head = h->head;
    CUDA_TRY(h, cudaGraphLaunch(g.exec, h->stream));
    h->launches += 2 * chunk;
    return NMF_OK;
  }
  nmf_status s = launch_all();
  if (s != NMF_OK) return s;
  if (graphable) {
    g.seen_m = h->m;
    g.seen_head = h->head;
  }
  return NMF_OK;
}

// Passes of the next chunk.  The refinement phase of the mixed form, where
// the incremental pass has a plan: a compensated sweep that records the
// references, then incremental sweeps; otherwise compensated sweeps.
ChunkPlan plan_for(const nmf_handle* h) {
  auto one = [](int v) { return ChunkPlan{v, v, false}; };
  if (!h->store_f32) return one(VAR_F64);
  if (!h->refine_ok) return one(VAR_F32);
  const ChunkPlan incremental = h->inc_ok ? ChunkPlan{VAR_DF, VAR_INC, true} : one(VAR_DF);
  switch (h->forced_mode) {
    case 0: return one(VAR_F32);
    case 1: return one(VAR_REF);
    case 2: return one(VAR_DF);
    case 3: return incremental;
    default: return h->phase ? incremental : one(VAR_F32);
  }
}

nmf_status read_state(nmf_handle* h) {
  CUDA_TRY(h, cudaMemcpyAsync(h->hSt, h->dSt, sizeof(DevState), cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  h->snap_valid = true;
  if (h->hSt->err & ERR_TIMEOUT) return fail(h, NMF_ETIMEOUT, "a device wait exceeded its bound");
  if (h->hSt->err & ERR_NONFINITE) return fail(h, NMF_ENUMERIC, "non-finite value in a sweep");
  return NMF_OK;
}

void fill_stats(const nmf_handle* h, int measured, int sweeps, int fp64_sweeps, nmf_stats* out) {
  std::memset(out, 0, sizeof(*out));
  out->sweeps = sweeps;
  out->iter = h->hSt->iter;
  out->fp64_sweeps = fp64_sweeps;
  out->converged = h->hSt->done ? h->hSt->stop_reason : 0;
  out->measured_iter = measured;
  if (measured < 0) return;
  const double* r = h->hSt->stats[measured % STAT_CAP];
  out->f = r[ST_F];
  out->kkt_abs = r[ST_EABS];
  out->kkt_rel = r[ST_VALID] > 0.0 ? r[ST_REL] : -1.0;
  out->step_rel = r[ST_STEP];
  out->changed_cols = (int64_t)r[ST_CHANGED_COLS];
  out->changed_rows = (int64_t)r[ST_CHANGED_ROWS];
  out->nnls_notconv = (int64_t)r[ST_NOTCONV];
  out->entering_steps = (int32_t)r[ST_ENTER];
}

template <typename T>
cudaError_t dalloc(T** p, size_t count) {
  return cudaMalloc(reinterpret_cast<void**>(p), sizeof(T) * std::max<size_t>(count, 1));
}

}  // namespace

// ---------------------------------------------------------------------------
// ABI
// ---------------------------------------------------------------------------
extern "C" {

void nmf_config_init(nmf_config* cfg) {
  if (!cfg) return;
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->prec = NMF_PREC_MIXED;
  cfg->stol = 0.0;
  cfg->kkt_target = 1e-8;
  cfg->mixed_switch = 1e-6;
  cfg->max_sweeps = 100000;
  cfg->warm_start = NMF_WARM_PREV;
  cfg->cuda_stream = nullptr;
}

const char* nmf_status_string(nmf_status s) {
  switch (s) {
    case NMF_OK: return "ok";
    case NMF_EINVAL: return "invalid argument";
    case NMF_ENOMEM: return "out of memory";
    case NMF_ECUDA: return "CUDA error";
    case NMF_ENOTCONV: return "not converged";
    case NMF_ETIMEOUT: return "device wait timed out";
    case NMF_ECAPACITY: return "capacity exceeded";
    case NMF_ENUMERIC: return "non-finite value";
    case NMF_ESTATE: return "call out of order";
  }
  return "unknown status";
}

const char* nmf_last_error(const nmf_handle* h) { return h ? h->last_error.c_str() : ""; }

int64_t nmf_launch_count(const nmf_handle* h) { return h ? h->launches : 0; }

int64_t nmf_num_columns(const nmf_handle* h) { return h ? h->m : 0; }

nmf_status nmf_get_config(const nmf_handle* h, nmf_config* out) {
  if (!h || !out) return NMF_EINVAL;
  *out = h->cfg;
  out->cuda_stream = h->stream;
  return NMF_OK;
}

nmf_status nmf_destroy(nmf_handle* h) {
  if (!h) return NMF_OK;
  if (h->stream) cudaStreamSynchronize(h->stream);
  for (auto& g : h->graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  for (int i = 0; i < nmf_handle::NEV; ++i)
    for (int j = 0; j < 3; ++j)
      if (h->ev[i][j]) cudaEventDestroy(h->ev[i][j]);
  void* dptrs[] = {h->dM, h->dX[0], h->dX[1], h->dX32[0], h->dX32[1], h->dX32lo[0], h->dX32lo[1], h->dY[0], h->dY[1],
                   h->dYm[0], h->dYm[1], h->dXm[0], h->dXm[1], h->dG, h->dGtab, h->dGok, h->dHg, h->dHtab, h->dHok, h->dColsq, h->dPpart,
                   h->dHpart, h->dYterms, h->dXpart, h->dSt, h->dKkt, h->dSeed, h->dSeedMask,
                   h->dNonfinite, h->dStage, h->dBref, h->dYref, h->dPref, h->dXref, h->dXd32[0], h->dXd32[1],
                   h->dShard, h->dShardP, h->tcb.Bpart, h->tcb.Xs, h->tcb.Ys, h->tcb.red, h->tcb.ticket, h->tcb.perm, h->tcb.perm_tmp,
                   h->tcb.keys, h->dBdf, h->dXgt};
  for (void* p : dptrs)
    if (p) cudaFree(p);
  if (h->hSt) cudaFreeHost(h->hSt);
  if (h->hKkt) cudaFreeHost(h->hKkt);
  if (h->hNonfinite) cudaFreeHost(h->hNonfinite);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  delete h;
  return NMF_OK;
}

nmf_status nmf_create(const nmf_config* cfg, nmf_handle** out) {
  if (!cfg || !out) return NMF_EINVAL;
  *out = nullptr;
  const int k = cfg->k;
  if (cfg->n < 1 || cfg->n > (1 << 20) || cfg->m_capacity < 1 || cfg->m_capacity > (1 << 24) ||
      !((k >= 1 && k <= 8) || k == 16) || (cfg->prec != NMF_PREC_FP64 && cfg->prec != NMF_PREC_MIXED) ||
      cfg->warm_start < NMF_WARM_COLD || cfg->warm_start > NMF_WARM_CHAIN)
    return NMF_EINVAL;
  nmf_handle* h = new (std::nothrow) nmf_handle();
  if (!h) return NMF_ENOMEM;
  h->cfg = *cfg;
  h->n = (int)cfg->n;
  h->k = k;
  h->mcap = (int)cfg->m_capacity;
  h->ld = round_up(h->n, 32);
  h->store_f32 = cfg->prec == NMF_PREC_MIXED;
  h->nxblk = (h->n + XTraits<1>::RB - 1) / XTraits<1>::RB;
  auto bail = [&](nmf_status s, const char* msg) {
    std::string m = msg;
    nmf_destroy(h);
    (void)m;
    return s;
  };
  if (cudaGetDevice(&h->dev) != cudaSuccess) return bail(NMF_ECUDA, "no CUDA device");
  cudaDeviceGetAttribute(&h->nsm, cudaDevAttrMultiProcessorCount, h->dev);
  cudaDeviceGetAttribute(&h->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->dev);
  h->has[VAR_F32] = get_kernels_f32(k, &h->ks[VAR_F32]);
  h->has[VAR_REF] = get_kernels_ref(k, &h->ks[VAR_REF]);
  h->has[VAR_F64] = get_kernels_f64(k, &h->ks[VAR_F64]);
  h->has[VAR_DF] = get_kernels_df(k, &h->ks[VAR_DF]);
  h->has[VAR_INC] = get_kernels_inc(k, &h->ks[VAR_INC]);
  for (int v = 0; v < NVAR; ++v)
    if (h->has[v])
      for (int ci = 0; ci < 4; ++ci)
        h->max_clusters[v][ci] = h->ks[v].max_clusters(1 << ci, (size_t)h->smem_optin);
  {
    // every variant this handle may run must have a plan for n; at rank 16
    // with FP32 M the FP32-class pass is the tensor-core pass, and a handle
    // whose n is beyond the FP64-class kernels runs that pass alone
    tc16s::Plan T{};
    h->tc16 = h->store_f32 && k == 16 && tc16s::plan(h->ld, h->mcap, h->nsm, h->smem_optin, &T);
    const int need[3] = {h->store_f32 ? VAR_F32 : VAR_F64, h->store_f32 ? VAR_REF : VAR_F64,
                         h->store_f32 ? VAR_DF : VAR_F64};
    for (int v : need) {
      if (v == VAR_F32 && h->tc16) continue;
      YPlan L;
      int msave = h->m;
      h->m = h->mcap;
      const bool ok = h->has[v] && make_plan(h, v, &L);
      h->m = msave;
      if (!ok && h->tc16 && v != VAR_F32) {
        h->refine_ok = false;
        continue;
      }
      if (!ok) return bail(NMF_EINVAL, "n too large for the kernels of this precision");
    }
    if (h->tc16 && !h->refine_ok) {   // the rank-16 reference and incremental passes refine
      h->tc_refine = true;
      h->refine_ok = true;
      h->inc_ok = true;
    } else if (h->store_f32 && h->refine_ok && h->has[VAR_INC]) {
      YPlan L;
      int msave = h->m;
      h->m = h->mcap;
      h->inc_ok = make_plan(h, VAR_INC, &L);
      h->m = msave;
    }
  }
  if (cfg->cuda_stream) {
    h->stream = static_cast<cudaStream_t>(cfg->cuda_stream);
  } else {
    if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess)
      return bail(NMF_ECUDA, "stream creation failed");
    h->own_stream = true;
  }
  const size_t nk = (size_t)h->n * k, mk = (size_t)h->mcap * k;
  const int Qmax = h->nsm;
  bool ok = true;
  h->mirror = h->tc16 ? tc16s::MIRROR : 0;
  ok &= cudaMalloc(&h->dM, (size_t)h->ld * (h->mcap + h->mirror) * (h->store_f32 ? 4 : 8)) == cudaSuccess;
  for (int b = 0; b < 2; ++b) {
    ok &= dalloc(&h->dX[b], nk) == cudaSuccess;
    ok &= dalloc(&h->dX32[b], nk) == cudaSuccess;
    ok &= dalloc(&h->dX32lo[b], nk) == cudaSuccess;
    ok &= dalloc(&h->dY[b], mk) == cudaSuccess;
    ok &= dalloc(&h->dYm[b], h->mcap) == cudaSuccess;
    ok &= dalloc(&h->dXm[b], h->n) == cudaSuccess;
  }
  ok &= dalloc(&h->dG, (size_t)k * k) == cudaSuccess;
  if (h->inc_ok) {
    ok &= dalloc(&h->dBref, mk) == cudaSuccess;
    ok &= dalloc(&h->dYref, mk) == cudaSuccess;
    ok &= dalloc(&h->dPref, nk) == cudaSuccess;
    ok &= dalloc(&h->dXref, nk) == cudaSuccess;
    ok &= dalloc(&h->dXd32[0], nk) == cudaSuccess;
    ok &= dalloc(&h->dXd32[1], nk) == cudaSuccess;
  }
  if (k <= 8) {
    ok &= dalloc(&h->dGtab, ((size_t)1 << k) * k * k) == cudaSuccess;
    ok &= dalloc(&h->dGok, (size_t)1 << k) == cudaSuccess;
    ok &= dalloc(&h->dHg, (size_t)k * k) == cudaSuccess;
    ok &= dalloc(&h->dHtab, ((size_t)1 << k) * k * k) == cudaSuccess;
    ok &= dalloc(&h->dHok, (size_t)1 << k) == cudaSuccess;
  }
  ok &= dalloc(&h->dColsq, h->mcap) == cudaSuccess;
  ok &= cudaMalloc(&h->dPpart, (size_t)Qmax * h->ld * k * 8) == cudaSuccess;
  ok &= dalloc(&h->dHpart, (size_t)Qmax * k * k) == cudaSuccess;
  ok &= dalloc(&h->dYterms, (size_t)Qmax * NYT) == cudaSuccess;
  const int nxgrp = (h->nxblk + XGROUP - 1) / XGROUP;
  ok &= dalloc(&h->dXpart, (size_t)(h->nxblk + (k == 16 ? nxgrp : 0)) * (k * k + NXT)) == cudaSuccess;
  if (k == 16) ok &= cudaMalloc(&h->dXgt, (size_t)nxgrp * sizeof(unsigned)) == cudaSuccess;
  if (h->tc16) {
    ok &= cudaMalloc(&h->tcb.Bpart, tc16s::bpart_bytes(h->mcap)) == cudaSuccess;
    ok &= cudaMalloc(&h->tcb.Xs, tc16s::xs_bytes(h->ld)) == cudaSuccess;
    ok &= cudaMalloc(&h->tcb.Ys, tc16s::ys_bytes(h->mcap)) == cudaSuccess;
    ok &= cudaMalloc(&h->tcb.red, tc16s::red_bytes(h->nsm)) == cudaSuccess;
    ok &= cudaMalloc(&h->tcb.ticket, tc16s::ticket_count(h->nsm) * sizeof(unsigned)) == cudaSuccess;
    ok &= cudaMalloc(&h->tcb.perm, tc16s::perm_bytes(h->mcap)) == cudaSuccess;
    ok &= cudaMalloc(&h->tcb.perm_tmp, tc16s::perm_bytes(h->mcap)) == cudaSuccess;
    ok &= cudaMalloc(&h->tcb.keys, tc16s::perm_bytes(h->mcap)) == cudaSuccess;
    if (h->tc_refine) ok &= cudaMalloc(&h->dBdf, tc16r::bdf_bytes(h->ld, h->mcap)) == cudaSuccess;
  }
  ok &= dalloc(&h->dSt, 1) == cudaSuccess;
  ok &= dalloc(&h->dKkt, NSTAT) == cudaSuccess;
  ok &= dalloc(&h->dSeed, KMAX) == cudaSuccess;
  ok &= dalloc(&h->dSeedMask, 1) == cudaSuccess;
  ok &= dalloc(&h->dNonfinite, 1) == cudaSuccess;
  ok &= cudaMallocHost(&h->hSt, sizeof(DevState)) == cudaSuccess;
  ok &= cudaMallocHost(&h->hKkt, sizeof(double) * NSTAT) == cudaSuccess;
  ok &= cudaMallocHost(&h->hNonfinite, sizeof(unsigned)) == cudaSuccess;
  if (!ok) return bail(NMF_ENOMEM, "device allocation failed");
  cudaMemsetAsync(h->dM, 0, (size_t)h->ld * (h->mcap + h->mirror) * (h->store_f32 ? 4 : 8), h->stream);
  cudaMemsetAsync(h->dSt, 0, sizeof(DevState), h->stream);
  if (h->dXgt) cudaMemsetAsync(h->dXgt, 0, (size_t)nxgrp * sizeof(unsigned), h->stream);
  if (h->tc16) {
    cudaMemsetAsync(h->tcb.ticket, 0, tc16s::ticket_count(h->nsm) * sizeof(unsigned), h->stream);
    if (!tc16s::encode_maps(h->dM, h->ld, h->mcap, &h->tcmaps)) return bail(NMF_ECUDA, "tensor maps of M rejected");
  }
  cudaMemsetAsync(h->dColsq, 0, sizeof(double) * h->mcap, h->stream);
  for (int b = 0; b < 2; ++b) {
    cudaMemsetAsync(h->dY[b], 0, sizeof(double) * mk, h->stream);
    cudaMemsetAsync(h->dYm[b], 0, sizeof(uint32_t) * h->mcap, h->stream);
  }
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return bail(NMF_ECUDA, "initialisation failed");
  *out = h;
  return NMF_OK;
}

nmf_status nmf_append_columns(nmf_handle* h, const void* cols, int64_t ncols, int64_t ld,
                              int32_t dtype, int32_t on_device) {
  if (!h) return NMF_EINVAL;
  if (h->poisoned) return h->poisoned;
  if (ncols < 0 || (ncols > 0 && !cols) || ld < h->n || (dtype != NMF_DTYPE_F32 && dtype != NMF_DTYPE_F64))
    return fail(h, NMF_EINVAL, "bad append arguments");
  if (ncols == 0) return NMF_OK;
  const size_t esz = dtype == NMF_DTYPE_F32 ? 4 : 8;
  const char* src = static_cast<const char*>(cols);
  if (ncols > h->mcap) {          // only the newest m_capacity columns can stay
    src += (size_t)(ncols - h->mcap) * ld * esz;
    ncols = h->mcap;
  }
  // seed for the new columns: the newest resident column (before eviction)
  const bool have_seed = h->m > 0;
  if (have_seed) {
    const int seed_phys = wrap_col(h->head, h->m - 1, h->mcap);
    seed_kernel<<<1, 32, 0, h->stream>>>(h->dSt, h->dY[0], h->dY[1], h->dYm[0], h->dYm[1], seed_phys,
                                         h->k, h->dSeed, h->dSeedMask);
    h->launches++;
  }
  const int first_phys = wrap_col(h->head, h->m, h->mcap);   // slot of the first new column
  const int evict = std::max(0, h->m + (int)ncols - h->mcap);
  CUDA_TRY(h, cudaMemsetAsync(h->dNonfinite, 0, sizeof(unsigned), h->stream));
  auto run = [&](const void* s, long long lds, int nc, int fp) -> cudaError_t {
    if (h->store_f32) {
      if (dtype == NMF_DTYPE_F32)
        append_kernel<float, float><<<nc, 256, 0, h->stream>>>(
            (const float*)s, lds, nc, (float*)h->dM, h->ld, h->n, h->mcap, fp, h->dColsq,
            have_seed ? h->dSeed : nullptr, have_seed ? h->dSeedMask : nullptr, h->dSt, h->dY[0],
            h->dY[1], h->dYm[0], h->dYm[1], h->k, h->dNonfinite, h->mirror);
      else
        append_kernel<double, float><<<nc, 256, 0, h->stream>>>(
            (const double*)s, lds, nc, (float*)h->dM, h->ld, h->n, h->mcap, fp, h->dColsq,
            have_seed ? h->dSeed : nullptr, have_seed ? h->dSeedMask : nullptr, h->dSt, h->dY[0],
            h->dY[1], h->dYm[0], h->dYm[1], h->k, h->dNonfinite, h->mirror);
    } else {
      if (dtype == NMF_DTYPE_F32)
        append_kernel<float, double><<<nc, 256, 0, h->stream>>>(
            (const float*)s, lds, nc, (double*)h->dM, h->ld, h->n, h->mcap, fp, h->dColsq,
            have_seed ? h->dSeed : nullptr, have_seed ? h->dSeedMask : nullptr, h->dSt, h->dY[0],
            h->dY[1], h->dYm[0], h->dYm[1], h->k, h->dNonfinite, h->mirror);
      else
        append_kernel<double, double><<<nc, 256, 0, h->stream>>>(
            (const double*)s, lds, nc, (double*)h->dM, h->ld, h->n, h->mcap, fp, h->dColsq,
            have_seed ? h->dSeed : nullptr, have_seed ? h->dSeedMask : nullptr, h->dSt, h->dY[0],
            h->dY[1], h->dYm[0], h->dYm[1], h->k, h->dNonfinite, h->mirror);
    }
    h->launches++;
    return cudaGetLastError();
  };
  if (on_device) {
    CUDA_TRY(h, run(src, ld, (int)ncols, first_phys));
  } else {
    const size_t need = (size_t)h->n * APPEND_STAGE_COLS * 8;
    if (h->stage_bytes < need) {
      if (h->dStage) cudaFree(h->dStage);
      h->dStage = nullptr;
      h->stage_bytes = 0;
      CUDA_TRY(h, cudaMalloc(&h->dStage, need));
      h->stage_bytes = need;
    }
    for (int64_t c0 = 0; c0 < ncols; c0 += APPEND_STAGE_COLS) {
      const int nc = (int)std::min<int64_t>(APPEND_STAGE_COLS, ncols - c0);
      CUDA_TRY(h, cudaMemcpy2DAsync(h->dStage, (size_t)h->n * esz, src + (size_t)c0 * ld * esz,
                                    (size_t)ld * esz, (size_t)h->n * esz, nc, cudaMemcpyHostToDevice,
                                    h->stream));
      CUDA_TRY(h, run(h->dStage, h->n, nc, wrap_col(first_phys, (int)c0 % h->mcap, h->mcap)));
    }
  }
  h->head = wrap_col(h->head, evict % h->mcap, h->mcap);
  h->m = h->m + (int)ncols - evict;
  msq_kernel<<<1, 256, 0, h->stream>>>(h->dSt, h->dColsq, h->head, h->m, h->mcap);
  h->launches++;
  CUDA_TRY(h, cudaGetLastError());
  CUDA_TRY(h, cudaMemcpyAsync(h->hNonfinite, h->dNonfinite, sizeof(unsigned), cudaMemcpyDeviceToHost,
                              h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  if (*h->hNonfinite) return fail(h, NMF_ENUMERIC, "appended data contain NaN or Inf");
  return NMF_OK;
}

nmf_status nmf_set_factors(nmf_handle* h, const double* X, const double* Y, int32_t on_device) {
  if (!h || !X || !Y) return NMF_EINVAL;
  if (h->poisoned) return h->poisoned;
  if (h->m < 1) return fail(h, NMF_ESTATE, "no resident column");
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  // fresh iterate 0 in buffers 0 (keep ||M||^2)
  CUDA_TRY(h, cudaMemsetAsync(h->dSt, 0, sizeof(DevState), h->stream));
  msq_kernel<<<1, 256, 0, h->stream>>>(h->dSt, h->dColsq, h->head, h->m, h->mcap);
  h->launches++;
  const size_t k = h->k;
  CUDA_TRY(h, cudaMemcpyAsync(h->dX[0], X, sizeof(double) * h->n * k, kind, h->stream));
  const int first = std::min(h->m, h->mcap - h->head);
  CUDA_TRY(h, cudaMemcpyAsync(h->dY[0] + (size_t)h->head * k, Y, sizeof(double) * first * k, kind,
                              h->stream));
  if (first < h->m)
    CUDA_TRY(h, cudaMemcpyAsync(h->dY[0], Y + (size_t)first * k, sizeof(double) * (h->m - first) * k,
                                kind, h->stream));
  clamp_kernel<<<64, 256, 0, h->stream>>>(h->dX[0], (long long)h->n * k);
  clamp_kernel<<<64, 256, 0, h->stream>>>(h->dY[0], (long long)h->mcap * k);
  h->launches += 2;
  CUDA_TRY(h, cudaGetLastError());
  h->phase = 0;
  h->best_rel = -1.0;
  h->chunks_since_best = 0;
  nmf_status s = launch_pair(h, h->store_f32 ? (h->refine_ok ? VAR_REF : VAR_F32) : VAR_F64, MODE_PRIME);
  if (s != NMF_OK) return s;
  s = read_state(h);
  if (s != NMF_OK) return s;
  h->factors_set = true;
  return NMF_OK;
}

nmf_status nmf_get_factors(nmf_handle* h, double* X, double* Y, uint32_t* xmask, uint32_t* ymask,
                           int32_t on_device) {
  if (!h) return NMF_EINVAL;
  if (h->poisoned) return h->poisoned;
  if (!h->factors_set) return fail(h, NMF_ESTATE, "factors not set");
  nmf_status s = read_state(h);
  if (s != NMF_OK && s != NMF_ENUMERIC) return s;
  const int cur = h->hSt->iter & 1;
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  const size_t k = h->k;
  if (X) CUDA_TRY(h, cudaMemcpyAsync(X, h->dX[cur], sizeof(double) * h->n * k, kind, h->stream));
  if (xmask) CUDA_TRY(h, cudaMemcpyAsync(xmask, h->dXm[cur], sizeof(uint32_t) * h->n, kind, h->stream));
  const int first = std::min(h->m, h->mcap - h->head);
  if (Y) {
    CUDA_TRY(h, cudaMemcpyAsync(Y, h->dY[cur] + (size_t)h->head * k, sizeof(double) * first * k, kind,
                                h->stream));
    if (first < h->m)
      CUDA_TRY(h, cudaMemcpyAsync(Y + (size_t)first * k, h->dY[cur], sizeof(double) * (h->m - first) * k,
                                  kind, h->stream));
  }
  if (ymask) {
    CUDA_TRY(h, cudaMemcpyAsync(ymask, h->dYm[cur] + h->head, sizeof(uint32_t) * first, kind, h->stream));
    if (first < h->m)
      CUDA_TRY(h, cudaMemcpyAsync(ymask + first, h->dYm[cur], sizeof(uint32_t) * (h->m - first), kind,
                                  h->stream));
  }
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  return NMF_OK;
}

nmf_status nmf_set_timing(nmf_handle* h, int32_t on) {
  if (!h) return NMF_EINVAL;
  if (h->poisoned) return h->poisoned;
  nmf_status s = drain_timing(h);
  if (s != NMF_OK) return s;
  h->timing = on != 0;
  h->y_ms = h->x_ms = 0.0;
  h->y_launches = h->x_launches = 0;
  for (int v = 0; v < NVAR; ++v) {
    h->yv_ms[v] = h->xv_ms[v] = 0.0;
    h->v_launches[v] = 0;
  }
  return NMF_OK;
}

nmf_status nmf_get_timing(nmf_handle* h, double* ypass_ms, int64_t* ypass_launches, double* xpass_ms,
                          int64_t* xpass_launches) {
  if (!h) return NMF_EINVAL;
  if (h->poisoned) return h->poisoned;
  nmf_status s = drain_timing(h);
  if (s != NMF_OK) return s;
  if (ypass_ms) *ypass_ms = h->y_ms;
  if (ypass_launches) *ypass_launches = h->y_launches;
  if (xpass_ms) *xpass_ms = h->x_ms;
  if (xpass_launches) *xpass_launches = h->x_launches;
  return NMF_OK;
}

int64_t nmf_shard_buffer_len(int64_t n, int32_t k) {
  if (n < 1 || k < 1) return 0;
  return n * k + (int64_t)k * k + NYT + 1;
}

nmf_status nmf_shard_y_half(nmf_handle* h, double* sum_buf, double* max_buf, int32_t on_device) {
  if (!h || !sum_buf || !max_buf) return NMF_EINVAL;
  if (h->poisoned) return h->poisoned;
  if (!h->factors_set) return fail(h, NMF_ESTATE, "factors not set");
  if (h->shard_var >= 0) return fail(h, NMF_ESTATE, "the previous Y half has not been completed");
  // FP64 form: the FP64 pass; mixed: the pass mode's contraction (automatic
  // and incremental modes use the compensated one)
  int var = VAR_F64;
  if (h->store_f32) var = h->forced_mode == 0 ? VAR_F32 : (h->forced_mode == 1 ? VAR_REF : VAR_DF);
  if (!h->refine_ok && var != VAR_F32) var = VAR_F32;
  const size_t len = (size_t)nmf_shard_buffer_len(h->n, h->k);
  if (!h->dShard) {
    CUDA_TRY(h, cudaMalloc(&h->dShard, sizeof(double) * (len + 1)));
    CUDA_TRY(h, cudaMalloc(&h->dShardP, sizeof(double) * ((size_t)h->ld * h->k + h->k * h->k + NYT)));
  }
  YPlan L{};
  const bool use_tc = h->tc16 && (var == VAR_F32 || h->tc_refine);
  if (use_tc) {
    nmf_status ts = tc_plan(h, &L.Q);
    if (ts != NMF_OK) return ts;
  } else if (!make_plan(h, var, &L)) {
    return fail(h, NMF_EINVAL, "no launch plan for this shape");
  }
  Problem p = make_problem(h, var);
  p.tab_global = 0;     // H is formed from the reduced buffers by the X half
  CUDA_TRY(h, cudaMemsetAsync(&h->dSt->done, 0, sizeof(int), h->stream));
  int nl = 1;
  if (use_tc && var == VAR_F32)
    CUDA_TRY(h, tc16s::launch(p, MODE_SWEEP, h->tc16_L, h->tcb, h->tcmaps, h->stream, &nl));
  else if (use_tc)
    CUDA_TRY(h, tc16r::launch(p, MODE_SWEEP, tc16r::REF_PASS, h->tcR, h->tc16_L, h->tcb, h->tcmaps, h->dBdf,
                              h->stream, &nl, &L.Q));
  else
    CUDA_TRY(h, h->ks[var].ypass(p, MODE_SWEEP, L, h->stream));
  double* out = h->dShard;
  double* outmax = h->dShard + len;
  const int nb = std::max(1, std::min(h->nsm, (int)(((size_t)h->n * h->k + 255) / 256)));
  if (var == VAR_F32) shard_export_kernel<float><<<nb, 256, 0, h->stream>>>(p, L.Q, out, outmax);
  else if (var == VAR_DF && !use_tc) shard_export_kernel<DF><<<nb, 256, 0, h->stream>>>(p, L.Q, out, outmax);
  else shard_export_kernel<double><<<nb, 256, 0, h->stream>>>(p, L.Q, out, outmax);
  h->launches += nl + 1;
  CUDA_TRY(h, cudaGetLastError());
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  CUDA_TRY(h, cudaMemcpyAsync(sum_buf, out, sizeof(double) * len, kind, h->stream));
  CUDA_TRY(h, cudaMemcpyAsync(max_buf, outmax, sizeof(double), kind, h->stream));
  if (!on_device) CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  h->shard_var = var;
  h->snap_valid = false;
  return NMF_OK;
}

nmf_status nmf_shard_x_half(nmf_handle* h, const double* sum_buf, const double* max_buf, int32_t on_device,
                            nmf_stats* stats) {
  if (!h || !sum_buf || !max_buf) return NMF_EINVAL;
  if (h->poisoned) return h->poisoned;
  if (h->shard_var < 0) return fail(h, NMF_ESTATE, "no Y half is pending");
  const size_t len = (size_t)nmf_shard_buffer_len(h->n, h->k);
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  CUDA_TRY(h, cudaMemcpyAsync(h->dShard, sum_buf, sizeof(double) * len, kind, h->stream));
  CUDA_TRY(h, cudaMemcpyAsync(h->dShard + len, max_buf, sizeof(double), kind, h->stream));
  double* P = h->dShardP;
  double* H = P + (size_t)h->ld * h->k;
  double* Yt = H + h->k * h->k;
  const int nb = std::max(1, std::min(h->nsm, (int)(((size_t)h->n * h->k + 255) / 256)));
  shard_import_kernel<<<nb, 256, 0, h->stream>>>(h->dShard, h->dShard + len, h->n, h->k, P, H, Yt, h->dSt);
  // the FP64-class row pass on the global P and H (one partial)
  const int var_x = h->store_f32 ? VAR_REF : VAR_F64;
  Problem p = make_problem(h, h->shard_var);
  p.Ppart = P;
  p.Hpart = H;
  p.Yterms = Yt;
  p.tab_global = 0;     // the row blocks form H's table from the reduced H
  p.fp64_pass = h->shard_var != VAR_F32;
  CUDA_TRY(h, h->ks[var_x].xpass(p, MODE_SWEEP, 1, h->nxblk, h->stream));
  h->launches += 2;
  CUDA_TRY(h, cudaGetLastError());
  h->shard_var = -1;
  // the control block holds this rank's own ||M||^2 again (nmf_objective_kkt
  // measures the rank's own columns)
  msq_kernel<<<1, 256, 0, h->stream>>>(h->dSt, h->dColsq, h->head, h->m, h->mcap, 0);
  h->launches++;
  nmf_status s = read_state(h);
  if (s != NMF_OK) return s;
  if (stats) fill_stats(h, h->hSt->done && h->hSt->stop_reason == 1 ? h->hSt->iter : h->hSt->iter - 1, 1,
                        p.fp64_pass, stats);
  return NMF_OK;
}

nmf_status nmf_get_pass_timing(nmf_handle* h, int32_t pass, double* ypass_ms, double* xpass_ms,
                               int64_t* sweeps) {
  static const int var_of[5] = {VAR_F32, VAR_REF, VAR_DF, VAR_INC, VAR_F64};
  if (!h || pass < 0 || pass > 4) return NMF_EINVAL;
  if (h->poisoned) return h->poisoned;
  nmf_status s = drain_timing(h);
  if (s != NMF_OK) return s;
  const int v = var_of[pass];
  if (ypass_ms) *ypass_ms = h->yv_ms[v];
  if (xpass_ms) *xpass_ms = h->xv_ms[v];
  if (sweeps) *sweeps = h->v_launches[v];
  return NMF_OK;
}

nmf_status nmf_set_pass_mode(nmf_handle* h, int32_t mode) {
  if (!h || mode < -1 || mode > 3) return NMF_EINVAL;
  h->forced_mode = mode;
  return NMF_OK;
}

nmf_status nmf_sweep(nmf_handle* h, int32_t nsweeps, nmf_stats* stats) {
  if (!h || nsweeps < 0) return NMF_EINVAL;
  if (h->poisoned) return h->poisoned;
  if (!h->factors_set) return fail(h, NMF_ESTATE, "factors not set");
  CUDA_TRY(h, cudaMemsetAsync(&h->dSt->done, 0, sizeof(int), h->stream));
  const bool until = nsweeps == 0;
  const int cap = until ? std::max(1, h->cfg.max_sweeps) : nsweeps;
  const bool adaptive = h->store_f32 && h->forced_mode < 0;
  const bool need_checks = until || adaptive || stats;
  nmf_status s = NMF_OK;
  if (need_checks && !h->snap_valid) {
    s = read_state(h);
    if (s != NMF_OK) return s;
  }
  int iter_prev = h->hSt->iter;
  int launched = 0, worked = 0, fp64_sweeps = 0, measured = -1;
  bool done = false;
  while (launched < cap) {
    const ChunkPlan cp = plan_for(h);
    // chunks of incremental sweeps never exceed CHUNK: each starts from the
    // references its first sweep records
    const bool split = need_checks || cp.first != cp.rest;
    const int chunk = split ? std::min(CHUNK, cap - launched) : cap - launched;
    const int var = cp.rest;
    s = launch_chunk(h, cp, chunk);
    if (s != NMF_OK) return s;
    launched += chunk;
    if (!need_checks) {
      h->snap_valid = false;
      if (launched < cap) continue;
      break;
    }
    s = read_state(h);
    if (s != NMF_OK) return s;
    const int iter_now = h->hSt->iter;
    done = h->hSt->done != 0;
    const bool stop_kkt = done && h->hSt->stop_reason == 1;
    const int w = (iter_now - iter_prev) + (stop_kkt ? 1 : 0);
    worked += w;
    if (var != VAR_F32) fp64_sweeps += w;
    measured = stop_kkt ? iter_now : iter_now - 1;
    iter_prev = iter_now;
    if (done) break;
    if (adaptive && h->phase == 0 && measured >= 0) {
      // FP32 passes until the relative KKT error reaches mixed_switch, or
      // until it has not improved by 2% over STALL_CHUNKS checks (the FP32
      // contraction's floor), then FP64-accumulated passes.
      const double* r = h->hSt->stats[measured % STAT_CAP];
      const double rel = r[ST_VALID] > 0.0 ? r[ST_REL] : -1.0;
      if (rel > 0.0) {
        if (h->best_rel < 0.0 || rel < 0.98 * h->best_rel) {
          h->best_rel = rel;
          h->chunks_since_best = 0;
        } else {
          ++h->chunks_since_best;
        }
        if (rel <= h->cfg.mixed_switch || h->chunks_since_best >= STALL_CHUNKS) h->phase = 1;
      }
    }
  }
  if (stats) fill_stats(h, measured, worked, fp64_sweeps, stats);
  if (until && !done) return fail(h, NMF_ENOTCONV, "sweep cap reached");
  return NMF_OK;
}

nmf_status nmf_objective_kkt(nmf_handle* h, double* f, double* kkt_abs, double* kkt_rel) {
  if (!h) return NMF_EINVAL;
  if (h->poisoned) return h->poisoned;
  if (!h->factors_set) return fail(h, NMF_ESTATE, "factors not set");
  // the FP64-contraction pass where it has a plan, else (rank 16 beyond its
  // rows) the tensor-core pass
  const int var = h->store_f32 ? (h->refine_ok ? VAR_REF : VAR_F32) : VAR_F64;
  YPlan L{};
  const bool use_tc = h->tc16 && (var == VAR_F32 || h->tc_refine);
  if (use_tc) {
    nmf_status ts = tc_plan(h, &L.Q);
    if (ts != NMF_OK) return ts;
  } else if (!make_plan(h, var, &L)) {
    return fail(h, NMF_EINVAL, "no launch plan for this shape");
  }
  Problem p = make_problem(h, var);
  CUDA_TRY(h, cudaMemsetAsync(&h->dSt->done, 0, sizeof(int), h->stream));
  int nl = 1;
  if (use_tc && var == VAR_F32)
    CUDA_TRY(h, tc16s::launch(p, MODE_KKT, h->tc16_L, h->tcb, h->tcmaps, h->stream, &nl));
  else if (use_tc)
    CUDA_TRY(h, tc16r::launch(p, MODE_KKT, tc16r::REF_PASS, h->tcR, h->tc16_L, h->tcb, h->tcmaps, h->dBdf,
                              h->stream, &nl, &L.Q));
  else
    CUDA_TRY(h, h->ks[var].ypass(p, MODE_KKT, L, h->stream));
  kkt_stats_kernel<<<1, 32, 0, h->stream>>>(p, L.Q, h->dKkt);
  h->launches += nl + 1;
  CUDA_TRY(h, cudaGetLastError());
  CUDA_TRY(h, cudaMemcpyAsync(h->hKkt, h->dKkt, sizeof(double) * NSTAT, cudaMemcpyDeviceToHost, h->stream));
  nmf_status s = read_state(h);
  if (s != NMF_OK) return s;
  if (f) *f = h->hKkt[ST_F];
  if (kkt_abs) *kkt_abs = h->hKkt[ST_EABS];
  if (kkt_rel) *kkt_rel = h->hKkt[ST_VALID] > 0.0 ? h->hKkt[ST_REL] : -1.0;
  return NMF_OK;
}

// ---------------------------------------------------------------------------
// persistence: the resident window, the iterate and the sweep state
// ---------------------------------------------------------------------------
namespace {

constexpr char SAVE_MAGIC[8] = {'N', 'M', 'F', 'G', 'B', '3', '0', '0'};
constexpr uint32_t SAVE_VERSION = 1;

struct SaveHeader {
  char magic[8];
  uint32_t version, devstate_bytes;
  int64_t n, ld, mcap, m;
  int32_t k, prec, max_sweeps, warm_start;
  double stol, kkt_target, mixed_switch, kkt_abs_target;
  int32_t factors_set, phase, forced_mode, chunks_since_best;
  double best_rel;
};

// copy the logical columns [0, m) of a ring of `width` elements per column
// (physical column of logical j: (head + j) mod mcap) between device and host
cudaError_t ring_copy(void* host, void* dev, size_t width_bytes, int head, int m, int mcap, bool to_host,
                      cudaStream_t s) {
  const int first = std::min(m, mcap - head);
  char* hp = static_cast<char*>(host);
  char* dp = static_cast<char*>(dev);
  const cudaMemcpyKind kind = to_host ? cudaMemcpyDeviceToHost : cudaMemcpyHostToDevice;
  cudaError_t e = cudaSuccess;
  if (first > 0) {
    e = to_host ? cudaMemcpyAsync(hp, dp + (size_t)head * width_bytes, (size_t)first * width_bytes, kind, s)
                : cudaMemcpyAsync(dp + (size_t)head * width_bytes, hp, (size_t)first * width_bytes, kind, s);
    if (e != cudaSuccess) return e;
  }
  if (first < m)
    e = to_host ? cudaMemcpyAsync(hp + (size_t)first * width_bytes, dp, (size_t)(m - first) * width_bytes, kind, s)
                : cudaMemcpyAsync(dp, hp + (size_t)first * width_bytes, (size_t)(m - first) * width_bytes, kind, s);
  return e;
}

struct FileCloser {
  FILE* f;
  ~FileCloser() {
    if (f) std::fclose(f);
  }
};

}  // namespace

nmf_status nmf_save(nmf_handle* h, const char* path) {
  if (!h || !path) return NMF_EINVAL;
  if (h->poisoned) return h->poisoned;
  nmf_status s = read_state(h);
  if (s != NMF_OK && s != NMF_ENUMERIC) return s;
  SaveHeader hd{};
  std::memcpy(hd.magic, SAVE_MAGIC, 8);
  hd.version = SAVE_VERSION;
  hd.devstate_bytes = (uint32_t)sizeof(DevState);
  hd.n = h->n;
  hd.ld = h->ld;
  hd.mcap = h->mcap;
  hd.m = h->m;
  hd.k = h->k;
  hd.prec = h->cfg.prec;
  hd.max_sweeps = h->cfg.max_sweeps;
  hd.warm_start = h->cfg.warm_start;
  hd.stol = h->cfg.stol;
  hd.kkt_target = h->cfg.kkt_target;
  hd.kkt_abs_target = h->cfg.kkt_abs_target;
  hd.mixed_switch = h->cfg.mixed_switch;
  hd.factors_set = h->factors_set ? 1 : 0;
  hd.phase = h->phase;
  hd.forced_mode = h->forced_mode;
  hd.chunks_since_best = h->chunks_since_best;
  hd.best_rel = h->best_rel;
  const int cur = h->hSt->iter & 1;
  const size_t k = h->k, esz = h->store_f32 ? 4 : 8, nk = (size_t)h->n * k;
  std::string buf;
  const size_t mbytes = (size_t)h->ld * h->m * esz;
  const size_t tab = k <= 8 ? ((size_t)1 << k) : 0;
  buf.resize(mbytes + h->m * 8 + h->m * k * 8 + h->m * 4 + nk * (8 + 4 + 4) + h->n * 4 + k * k * 8 +
             tab * k * k * 8 + tab * 4);
  char* p = &buf[0];
  char* const pm = p;                 p += mbytes;
  char* const pcol = p;               p += (size_t)h->m * 8;
  char* const py = p;                 p += (size_t)h->m * k * 8;
  char* const pym = p;                p += (size_t)h->m * 4;
  char* const px = p;                 p += nk * 8;
  char* const px32 = p;               p += nk * 4;
  char* const px32lo = p;             p += nk * 4;
  char* const pxm = p;                p += (size_t)h->n * 4;
  char* const pg = p;                 p += k * k * 8;
  char* const ptab = p;               p += tab * k * k * 8;
  char* const pok = p;
  cudaStream_t st = h->stream;
  CUDA_TRY(h, ring_copy(pm, h->dM, (size_t)h->ld * esz, h->head, h->m, h->mcap, true, st));
  CUDA_TRY(h, ring_copy(pcol, h->dColsq, 8, h->head, h->m, h->mcap, true, st));
  CUDA_TRY(h, ring_copy(py, h->dY[cur], k * 8, h->head, h->m, h->mcap, true, st));
  CUDA_TRY(h, ring_copy(pym, h->dYm[cur], 4, h->head, h->m, h->mcap, true, st));
  CUDA_TRY(h, cudaMemcpyAsync(px, h->dX[cur], nk * 8, cudaMemcpyDeviceToHost, st));
  CUDA_TRY(h, cudaMemcpyAsync(px32, h->dX32[cur], nk * 4, cudaMemcpyDeviceToHost, st));
  CUDA_TRY(h, cudaMemcpyAsync(px32lo, h->dX32lo[cur], nk * 4, cudaMemcpyDeviceToHost, st));
  CUDA_TRY(h, cudaMemcpyAsync(pxm, h->dXm[cur], (size_t)h->n * 4, cudaMemcpyDeviceToHost, st));
  CUDA_TRY(h, cudaMemcpyAsync(pg, h->dG, k * k * 8, cudaMemcpyDeviceToHost, st));
  if (tab) {
    CUDA_TRY(h, cudaMemcpyAsync(ptab, h->dGtab, tab * k * k * 8, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(h, cudaMemcpyAsync(pok, h->dGok, tab * 4, cudaMemcpyDeviceToHost, st));
  }
  CUDA_TRY(h, cudaStreamSynchronize(st));
  FileCloser fc{std::fopen(path, "wb")};
  if (!fc.f) return fail(h, NMF_EINVAL, std::string("cannot open ") + path + " for writing");
  bool ok = std::fwrite(&hd, sizeof(hd), 1, fc.f) == 1;
  ok = ok && std::fwrite(h->hSt, sizeof(DevState), 1, fc.f) == 1;
  ok = ok && std::fwrite(buf.data(), 1, buf.size(), fc.f) == buf.size();
  ok = (std::fclose(fc.f) == 0) && ok;
  fc.f = nullptr;
  if (!ok) return fail(h, NMF_EINVAL, std::string("write to ") + path + " failed");
  return NMF_OK;
}

nmf_status nmf_load(const char* path, void* cuda_stream, nmf_handle** out) {
  if (!path || !out) return NMF_EINVAL;
  *out = nullptr;
  FileCloser fc{std::fopen(path, "rb")};
  if (!fc.f) return NMF_EINVAL;
  SaveHeader hd{};
  if (std::fread(&hd, sizeof(hd), 1, fc.f) != 1) return NMF_EINVAL;
  if (std::memcmp(hd.magic, SAVE_MAGIC, 8) != 0 || hd.version != SAVE_VERSION ||
      hd.devstate_bytes != (uint32_t)sizeof(DevState))
    return NMF_EINVAL;
  if (hd.n < 1 || hd.n > (1 << 20) || hd.ld != (int64_t)round_up((int)hd.n, 32) || hd.mcap < 1 ||
      hd.mcap > (1 << 24) || hd.m < 0 || hd.m > hd.mcap || !((hd.k >= 1 && hd.k <= 8) || hd.k == 16) ||
      (hd.prec != NMF_PREC_FP64 && hd.prec != NMF_PREC_MIXED) || hd.forced_mode < -1 || hd.forced_mode > 2 ||
      (hd.factors_set && hd.m < 1))
    return NMF_EINVAL;
  DevState ds;
  if (std::fread(&ds, sizeof(ds), 1, fc.f) != 1) return NMF_EINVAL;
  const size_t k = hd.k, m = hd.m, n = hd.n, nk = n * k, esz = hd.prec == NMF_PREC_MIXED ? 4 : 8;
  const size_t tab = k <= 8 ? ((size_t)1 << k) : 0;
  const size_t total = (size_t)hd.ld * m * esz + m * 8 + m * k * 8 + m * 4 + nk * 16 + n * 4 + k * k * 8 +
                       tab * k * k * 8 + tab * 4;
  std::string buf(total, '\0');
  if (std::fread(&buf[0], 1, total, fc.f) != total) return NMF_EINVAL;
  char extra;
  if (std::fread(&extra, 1, 1, fc.f) != 0) return NMF_EINVAL;     // trailing bytes: not this format
  nmf_config cfg;
  nmf_config_init(&cfg);
  cfg.n = hd.n;
  cfg.m_capacity = hd.mcap;
  cfg.k = hd.k;
  cfg.prec = hd.prec;
  cfg.stol = hd.stol;
  cfg.kkt_target = hd.kkt_target;
  cfg.kkt_abs_target = hd.kkt_abs_target;
  cfg.mixed_switch = hd.mixed_switch;
  cfg.max_sweeps = hd.max_sweeps;
  cfg.warm_start = hd.warm_start;
  cfg.cuda_stream = cuda_stream;
  nmf_handle* h = nullptr;
  nmf_status s = nmf_create(&cfg, &h);
  if (s != NMF_OK) return s;
  auto bail = [&](nmf_status e) {
    nmf_destroy(h);
    return e;
  };
  const char* p = buf.data();
  const char* pm = p;      p += (size_t)hd.ld * m * esz;
  const char* pcol = p;    p += m * 8;
  const char* py = p;      p += m * k * 8;
  const char* pym = p;     p += m * 4;
  const char* px = p;      p += nk * 8;
  const char* px32 = p;    p += nk * 4;
  const char* px32lo = p;  p += nk * 4;
  const char* pxm = p;     p += n * 4;
  const char* pg = p;      p += k * k * 8;
  const char* ptab = p;    p += tab * k * k * 8;
  const char* pok = p;
  const int cur = ds.iter & 1;
  cudaStream_t st = h->stream;
  // the window lands in physical columns 0 .. m-1 (head 0); every partition
  // of the sweep follows logical column order, so results do not depend on it
  bool ok = cudaMemcpyAsync(h->dM, pm, (size_t)hd.ld * m * esz, cudaMemcpyHostToDevice, st) == cudaSuccess;
  if (h->mirror > 0 && m > 0)   // the mirrored columns after the ring
    ok = ok && cudaMemcpyAsync(static_cast<char*>(h->dM) + (size_t)hd.ld * h->mcap * esz, h->dM,
                               (size_t)hd.ld * std::min<size_t>(m, (size_t)h->mirror) * esz,
                               cudaMemcpyDeviceToDevice, st) == cudaSuccess;
  ok = ok && cudaMemcpyAsync(h->dColsq, pcol, m * 8, cudaMemcpyHostToDevice, st) == cudaSuccess;
  ok = ok && cudaMemcpyAsync(h->dY[cur], py, m * k * 8, cudaMemcpyHostToDevice, st) == cudaSuccess;
  ok = ok && cudaMemcpyAsync(h->dYm[cur], pym, m * 4, cudaMemcpyHostToDevice, st) == cudaSuccess;
  ok = ok && cudaMemcpyAsync(h->dX[cur], px, nk * 8, cudaMemcpyHostToDevice, st) == cudaSuccess;
  ok = ok && cudaMemcpyAsync(h->dX32[cur], px32, nk * 4, cudaMemcpyHostToDevice, st) == cudaSuccess;
  ok = ok && cudaMemcpyAsync(h->dX32lo[cur], px32lo, nk * 4, cudaMemcpyHostToDevice, st) == cudaSuccess;
  ok = ok && cudaMemcpyAsync(h->dXm[cur], pxm, n * 4, cudaMemcpyHostToDevice, st) == cudaSuccess;
  ok = ok && cudaMemcpyAsync(h->dG, pg, k * k * 8, cudaMemcpyHostToDevice, st) == cudaSuccess;
  if (tab) {
    ok = ok && cudaMemcpyAsync(h->dGtab, ptab, tab * k * k * 8, cudaMemcpyHostToDevice, st) == cudaSuccess;
    ok = ok && cudaMemcpyAsync(h->dGok, pok, tab * 4, cudaMemcpyHostToDevice, st) == cudaSuccess;
  }
  ds.done = 0;
  ds.xblocks_done = 0;
  ok = ok && cudaMemcpyAsync(h->dSt, &ds, sizeof(ds), cudaMemcpyHostToDevice, st) == cudaSuccess;
  ok = ok && cudaStreamSynchronize(st) == cudaSuccess;
  if (!ok) return bail(NMF_ECUDA);
  h->m = (int)m;
  h->head = 0;
  h->factors_set = hd.factors_set != 0;
  h->phase = hd.phase;
  h->forced_mode = hd.forced_mode;
  h->chunks_since_best = hd.chunks_since_best;
  h->best_rel = hd.best_rel;
  h->snap_valid = false;
  *out = h;
  return NMF_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// internal interface for the batched form
// ---------------------------------------------------------------------------
namespace nmfgb {

int64_t handle_footprint(int64_t n, int k, int64_t mcap, bool store_f32, int nsm) {
  const int64_t ld = (n + 31) / 32 * 32, nk = n * k, mk = mcap * k;
  const int64_t nxblk = (n + XTraits<1>::RB - 1) / XTraits<1>::RB;
  int64_t b = ld * mcap * (store_f32 ? 4 : 8);                       // the ring of M
  b += 2 * (nk * 8 + 2 * nk * 4 + mk * 8 + mcap * 4 + n * 4);        // X, X32, X32lo, Y, masks
  if (k <= 8) b += 2 * ((int64_t(1) << k) * k * k * 8 + (int64_t(1) << k) * 4 + k * k * 8);
  b += mcap * 8;                                                     // column norms
  b += (int64_t)nsm * (ld * k * 8 + k * k * 8 + NYT * 8);            // cluster partials
  b += nxblk * (k * k + NXT) * 8 + (int64_t)sizeof(DevState) + 4096;
  b += (int64_t)APPEND_STAGE_COLS * ld * 8;                          // append staging
  if (store_f32) b += 2 * mk * 8 + 2 * nk * 8 + 2 * nk * 4;           // incremental references
  return b;
}

bool handle_info(nmf_handle* h, HandleInfo* o) {
  if (!h || !o) return false;
  o->n = h->n;
  o->ld = h->ld;
  o->k = h->k;
  o->m = h->m;
  o->mcap = h->mcap;
  o->nsm = h->nsm;
  o->smem_optin = h->smem_optin;
  o->nxblk = h->nxblk;
  o->store_f32 = h->store_f32;
  o->factors_set = h->factors_set;
  o->qcap = h->nsm;
  o->phase = h->phase;
  o->dSt = h->dSt;
  o->hSt = h->hSt;
  o->stream = h->stream;
  return true;
}

bool handle_problem(nmf_handle* h, int var, Problem* out) {
  if (!h || var < 0 || var >= NVAR || !h->has[var]) return false;
  *out = make_problem(h, var);
  return true;
}

bool handle_plan(nmf_handle* h, int var, YPlan* out) {
  if (!h || var < 0 || var >= NVAR || !h->has[var]) return false;
  return make_plan(h, var, out);
}

const KernelSet* handle_kernels(nmf_handle* h, int var) {
  if (!h || var < 0 || var >= NVAR || !h->has[var]) return nullptr;
  return &h->ks[var];
}

nmf_status handle_sync_state(nmf_handle* h) { return read_state(h); }

void handle_set_phase(nmf_handle* h, int phase) {
  h->phase = phase;
  h->snap_valid = false;
}

void handle_fill_stats(nmf_handle* h, int measured, int sweeps, int fp64_sweeps, nmf_stats* out) {
  fill_stats(h, measured, sweeps, fp64_sweeps, out);
}

nmf_status handle_fail(nmf_handle* h, nmf_status s, const char* msg) { return fail(h, s, msg); }

}  // namespace nmfgb


// Streaming server (declared in include/nmf.h): per-stream time columns
// arrive in chunks (Sec. 1's streaming setting); a worker thread keeps every
// admitted stream's ring of columns, X, Y and passive sets resident on the
// device and, round after round, appends the chunks that have arrived and
// sweeps every stream with pending chunks in one batched launch
// (continuous batching: a chunk that arrives while a round runs joins at
// the next round).  A chunk completes when its stream reaches the relative
// KKT target, or after max_sweeps_per_chunk sweeps, with all chunks of the
// stream appended before it.  Streams are admitted in arrival order while
// their device footprint fits the HBM budget; closing a stream frees its
// memory for the next one.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <random>
#include <string>
#include <thread>
#include <vector>

#include "nmf_internal.h"

using namespace nmfgb;

namespace {

struct SChunk {
  uint64_t ticket = 0;
  int64_t ncols = 0;
  std::vector<float> data;   // n x ncols, column-major
  double t_submit = 0.0;
};

enum { S_QUEUED = 0, S_ADMITTED = 1, S_CLOSED = 2 };

// A stream.  Guarded by nmf_server::mu: state, closing, waiting (n, k,
// mcap, seed, bytes are fixed at open).  Owned by the worker and touched
// only under nmf_server::dev_mu: slot, factors, inflight, sweeps_since.
struct SStream {
  int id = 0;
  int64_t n = 0, mcap = 0;
  int k = 0;
  uint64_t seed = 0;
  int64_t bytes = 0;
  int state = S_QUEUED;
  bool closing = false;
  std::deque<SChunk> waiting;    // submitted, not yet appended
  int slot = -1;
  bool factors = false;
  std::vector<SChunk> inflight;  // appended, waiting for the stream to converge
  int sweeps_since = 0;          // sweeps since its oldest in-flight chunk was appended
};

}  // namespace

struct nmf_server {
  nmf_server_config cfg{};
  nmf_batch* batch = nullptr;
  int dev = 0, nsm = 0;
  std::chrono::steady_clock::time_point t0;
  std::mutex mu;                 // requests, streams, results
  std::condition_variable cv_work, cv_done;
  std::mutex dev_mu;             // device work (the worker's rounds, reads of factors)
  std::vector<std::unique_ptr<SStream>> streams;   // addresses stable across opens
  std::deque<int> admit_queue;
  std::vector<nmf_chunk_result> results;
  int64_t bytes_in_use = 0;
  int admitted = 0;
  uint64_t next_ticket = 1;
  bool stop = false;
  std::thread worker;
  nmf_server_stats stats{};
  nmf_status poisoned = NMF_OK;
  std::string last_error;
};

namespace {

double now_s(const nmf_server* s) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - s->t0).count();
}

// The worker: round after round, admit, append, sweep, complete; a device
// error poisons the server and ends the worker.
void worker_main(nmf_server* s) {
  cudaSetDevice(s->dev);
  std::vector<nmf_stats> st;
  for (;;) {
    std::vector<SStream*> snap, to_admit, to_remove;
    std::vector<std::pair<SStream*, std::vector<SChunk>>> to_append;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      // worker-owned fields are read here by the worker itself
      auto has_work = [&] {
        if (s->stop) return true;
        for (const auto& x : s->streams)
          if (x->state == S_ADMITTED && (!x->waiting.empty() || !x->inflight.empty() || x->closing)) return true;
        if (!s->admit_queue.empty()) {
          const SStream& x = *s->streams[s->admit_queue.front()];
          if (x.closing || (s->bytes_in_use + x.bytes <= s->cfg.hbm_budget_bytes && s->admitted < s->cfg.max_streams))
            return true;
        }
        return false;
      };
      s->cv_work.wait(lk, has_work);
      if (s->stop) return;
      // admission in the order the streams were opened, while the footprint fits
      while (!s->admit_queue.empty()) {
        SStream& x = *s->streams[s->admit_queue.front()];
        if (x.closing) {   // closed before admission
          x.state = S_CLOSED;
          s->admit_queue.pop_front();
          continue;
        }
        if (s->bytes_in_use + x.bytes > s->cfg.hbm_budget_bytes || s->admitted >= s->cfg.max_streams) break;
        s->admit_queue.pop_front();
        s->bytes_in_use += x.bytes;
        s->admitted++;
        x.state = S_ADMITTED;
        to_admit.push_back(&x);
      }
      for (auto& up : s->streams) {
        SStream& x = *up;
        if (x.state != S_ADMITTED) continue;
        snap.push_back(&x);
        if (!x.waiting.empty()) {
          std::vector<SChunk> v(std::make_move_iterator(x.waiting.begin()), std::make_move_iterator(x.waiting.end()));
          x.waiting.clear();
          to_append.emplace_back(&x, std::move(v));
        } else if (x.closing && x.inflight.empty()) {
          to_remove.push_back(&x);
        }
      }
    }
    std::vector<nmf_chunk_result> done;
    nmf_status err = NMF_OK;
    int active_streams = 0, swept = 0;
    {
      std::lock_guard<std::mutex> dl(s->dev_mu);
      for (SStream* xp : to_admit) {
        SStream& x = *xp;
        nmf_config c;
        nmf_config_init(&c);
        c.n = x.n;
        c.k = x.k;
        c.m_capacity = x.mcap;
        c.prec = NMF_PREC_MIXED;
        c.kkt_target = s->cfg.kkt_target;
        c.mixed_switch = s->cfg.mixed_switch;
        int slot = -1;
        err = batch_add(s->batch, c, &slot);
        if (err != NMF_OK) break;
        batch_set_active(s->batch, slot, false);
        x.slot = slot;
      }
      for (SStream* xp : to_remove) {
        batch_remove(s->batch, xp->slot);
        xp->slot = -1;
      }
      for (auto& pr : to_append) {
        if (err != NMF_OK) break;
        SStream& x = *pr.first;
        for (SChunk& ch : pr.second) {
          err = nmf_batch_append_columns(s->batch, x.slot, ch.data.data(), ch.ncols, x.n, NMF_DTYPE_F32, 0);
          if (err != NMF_OK) break;
          if (!x.factors) {
            // a new stream starts from U[0,1] factors drawn from its seed
            nmf_handle* h = nmf_batch_problem(s->batch, x.slot);
            const int64_t m = nmf_num_columns(h);
            std::mt19937_64 g(x.seed);
            std::uniform_real_distribution<double> u(0.0, 1.0);
            std::vector<double> X((size_t)x.n * x.k), Y((size_t)m * x.k);
            for (double& v : X) v = u(g);
            for (double& v : Y) v = u(g);
            err = nmf_batch_set_factors(s->batch, x.slot, X.data(), Y.data(), 0);
            if (err != NMF_OK) break;
            x.factors = true;
          }
          if (x.inflight.empty()) x.sweeps_since = 0;
          ch.data.clear();
          ch.data.shrink_to_fit();
          x.inflight.push_back(std::move(ch));
        }
      }
      // the streams with chunks in flight are this round's batch
      std::vector<SStream*> act;
      for (SStream* xp : snap) {
        if (err != NMF_OK || xp->slot < 0) continue;
        const bool on = !xp->inflight.empty();
        batch_set_active(s->batch, xp->slot, on);
        if (on) act.push_back(xp);
      }
      active_streams = (int)act.size();
      if (err == NMF_OK && active_streams) {
        st.assign((size_t)nmf_batch_size(s->batch), nmf_stats{});
        err = nmf_batch_sweep(s->batch, s->cfg.sweeps_per_round, st.data(), &swept);
        const double t = now_s(s);
        for (SStream* xp : act) {
          if (err != NMF_OK) break;
          SStream& x = *xp;
          const nmf_stats& r = st[x.slot];
          x.sweeps_since += r.sweeps;
          const bool conv = r.converged == 1;
          if (conv || x.sweeps_since >= s->cfg.max_sweeps_per_chunk) {
            const int32_t m = (int32_t)nmf_num_columns(nmf_batch_problem(s->batch, x.slot));
            for (const SChunk& ch : x.inflight) {
              nmf_chunk_result o{};
              o.ticket = ch.ticket;
              o.stream = -1;
              o.ncols = (int32_t)ch.ncols;
              o.t_submit_s = ch.t_submit;
              o.t_done_s = t;
              o.sweeps = x.sweeps_since;
              o.converged = conv ? 1 : 0;
              o.kkt_rel = r.kkt_rel;
              o.f = r.f;
              o.m = m;
              done.push_back(o);
              done.back().stream = x.id;
            }
            x.inflight.clear();
            x.sweeps_since = 0;
          }
        }
      }
    }
    {
      std::lock_guard<std::mutex> lk(s->mu);
      if (err != NMF_OK) {
        s->poisoned = err;
        s->last_error = std::string("worker: ") + nmf_status_string(err) + ": " + nmf_batch_last_error(s->batch);
        s->stop = true;
        s->cv_done.notify_all();
        return;
      }
      for (SStream* xp : to_remove) {
        xp->state = S_CLOSED;
        s->bytes_in_use -= xp->bytes;
        s->admitted--;
      }
      for (const nmf_chunk_result& o : done) {
        s->stats.chunks_done++;
        s->stats.columns_done += o.ncols;
      }
      if (active_streams) {
        s->stats.rounds++;
        s->stats.batch_sweeps += swept;
        s->stats.stream_rounds += active_streams;
        s->stats.max_streams_in_round = std::max<int32_t>(s->stats.max_streams_in_round, active_streams);
      }
      s->results.insert(s->results.end(), done.begin(), done.end());
      s->cv_done.notify_all();
    }
  }
}

}  // namespace

extern "C" {

void nmf_server_config_init(nmf_server_config* c) {
  if (!c) return;
  std::memset(c, 0, sizeof(*c));
  c->hbm_budget_bytes = 0;
  c->max_streams = 64;
  c->kkt_target = 1e-6;
  c->mixed_switch = 1e-6;
  c->max_sweeps_per_chunk = 500;
  c->sweeps_per_round = 8;
  c->cuda_stream = nullptr;
}

nmf_status nmf_server_create(const nmf_server_config* cfg, nmf_server** out) {
  if (!cfg || !out || cfg->max_streams < 1 || cfg->sweeps_per_round < 1 || cfg->max_sweeps_per_chunk < 1 ||
      cfg->hbm_budget_bytes < 0)
    return NMF_EINVAL;
  *out = nullptr;
  nmf_server* s = new nmf_server();
  s->cfg = *cfg;
  s->t0 = std::chrono::steady_clock::now();
  if (cudaGetDevice(&s->dev) != cudaSuccess) {
    delete s;
    return NMF_ECUDA;
  }
  cudaDeviceGetAttribute(&s->nsm, cudaDevAttrMultiProcessorCount, s->dev);
  if (s->cfg.hbm_budget_bytes == 0) {   // 90% of the memory free now
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    s->cfg.hbm_budget_bytes = (int64_t)(0.9 * (double)fr);
  }
  nmf_status st = batch_create_empty(cfg->cuda_stream, &s->batch);
  if (st != NMF_OK) {
    delete s;
    return st;
  }
  s->worker = std::thread(worker_main, s);
  *out = s;
  return NMF_OK;
}

nmf_status nmf_server_destroy(nmf_server* s) {
  if (!s) return NMF_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  nmf_batch_destroy(s->batch);
  delete s;
  return NMF_OK;
}

nmf_status nmf_server_open_stream(nmf_server* s, int64_t n, int32_t k, int64_t m_capacity, uint64_t seed,
                                  int32_t* id) {
  if (!s || !id || n < 1 || m_capacity < 1 || k < 1 || (k > 8 && k != 16)) return NMF_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->poisoned) return s->poisoned;
  auto x = std::make_unique<SStream>();
  x->id = (int)s->streams.size();
  x->n = n;
  x->k = k;
  x->mcap = m_capacity;
  x->seed = seed;
  x->bytes = handle_footprint(n, k, m_capacity, true, s->nsm);
  if (x->bytes > s->cfg.hbm_budget_bytes) return NMF_ECAPACITY;
  s->streams.push_back(std::move(x));
  *id = (int32_t)s->streams.size() - 1;
  s->admit_queue.push_back(*id);
  s->cv_work.notify_all();
  return NMF_OK;
}

nmf_status nmf_server_submit(nmf_server* s, int32_t id, const float* cols, int64_t ncols, int64_t ld,
                             uint64_t* ticket) {
  if (!s || !cols || ncols < 1) return NMF_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->poisoned) return s->poisoned;
  if (id < 0 || id >= (int32_t)s->streams.size()) return NMF_EINVAL;
  SStream& x = *s->streams[id];
  if (x.state == S_CLOSED || x.closing || ld < x.n) return NMF_EINVAL;
  SChunk ch;
  ch.ticket = s->next_ticket++;
  ch.ncols = ncols;
  ch.t_submit = now_s(s);
  ch.data.resize((size_t)x.n * ncols);
  for (int64_t c = 0; c < ncols; ++c)
    std::memcpy(ch.data.data() + (size_t)c * x.n, cols + (size_t)c * ld, sizeof(float) * x.n);
  if (ticket) *ticket = ch.ticket;
  x.waiting.push_back(std::move(ch));
  s->cv_work.notify_all();
  return NMF_OK;
}

nmf_status nmf_server_close_stream(nmf_server* s, int32_t id) {
  if (!s) return NMF_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  if (id < 0 || id >= (int32_t)s->streams.size()) return NMF_EINVAL;
  s->streams[id]->closing = true;
  s->cv_work.notify_all();
  return NMF_OK;
}

nmf_status nmf_server_poll(nmf_server* s, nmf_chunk_result* out, int32_t cap, int32_t* nout, int32_t wait_ms) {
  if (!s || !nout || cap < 0 || (cap > 0 && !out)) return NMF_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  if (wait_ms > 0 && s->results.empty() && !s->poisoned)
    s->cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms), [&] { return !s->results.empty() || s->stop; });
  const int n = std::min<int>(cap, (int)s->results.size());
  std::copy(s->results.begin(), s->results.begin() + n, out);
  s->results.erase(s->results.begin(), s->results.begin() + n);
  *nout = n;
  return s->poisoned ? s->poisoned : NMF_OK;
}

nmf_status nmf_server_get_factors(nmf_server* s, int32_t id, double* X, double* Y, uint32_t* xmask,
                                  uint32_t* ymask, int64_t* m) {
  if (!s) return NMF_EINVAL;
  SStream* xp = nullptr;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->poisoned) return s->poisoned;
    if (id < 0 || id >= (int32_t)s->streams.size()) return NMF_EINVAL;
    if (s->streams[id]->state != S_ADMITTED) return NMF_ESTATE;
    xp = s->streams[id].get();
  }
  std::lock_guard<std::mutex> dl(s->dev_mu);
  if (xp->slot < 0 || !xp->factors) return NMF_ESTATE;
  if (m) *m = nmf_num_columns(nmf_batch_problem(s->batch, xp->slot));
  return nmf_batch_get_factors(s->batch, xp->slot, X, Y, xmask, ymask, 0);
}

nmf_status nmf_server_get_stats(nmf_server* s, nmf_server_stats* out) {
  if (!s || !out) return NMF_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->stats;
  out->streams_admitted = s->admitted;
  out->streams_queued = (int32_t)s->admit_queue.size();
  out->hbm_in_use_bytes = s->bytes_in_use;
  out->hbm_budget_bytes = s->cfg.hbm_budget_bytes;
  return s->poisoned ? s->poisoned : NMF_OK;
}

const char* nmf_server_last_error(nmf_server* s) {
  if (!s) return "null server";
  std::lock_guard<std::mutex> lk(s->mu);
  return s->last_error.c_str();
}

}  // extern "C"

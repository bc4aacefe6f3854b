// Continuous-batching serving of many independent Lindblad solves on one GPU
// (the request loop of the serving workload: solves of different mode counts,
// Fock sizes and bond caps arriving over time).
//
// A server owns a context for its lifetime and runs one worker thread, the only
// thread that touches the context's device work while the server exists.  The
// caller's calls only take the queue lock:
//   qlb_submit  deep-copies the request (system terms, start vectors, step plan,
//               observables) into the pending queue and returns a ticket;
//   qlb_poll    reads a request's status and, once it is done, its observables
//               and timestamps;
//   qlb_cancel  marks a request; the worker drops it between two chunks.
// The worker admits pending requests in arrival order while a live slot is free
// and the request's estimated device memory fits the budget next to the live
// ones; it builds the request's system and state and plans its step.  Live
// requests whose plans have the same shape (sites, precision form, Kraus MPO
// bonds, bond capacities) form a bucket, and a bucket steps its idle members
// together as a group (one launch per phase of the step over all of them, on the
// bucket's stream, enqueued without host synchronisation, so the buckets overlap
// on the GPU), in chunks of at most `chunk` steps.  When a state has taken all
// its steps the worker evaluates the requested observables, releases the state's
// memory and slot, and admits the next arrival.  A request's result does not
// depend on the other requests in flight: every state has its own buffers, and a
// group member computes bit for bit what it computes alone.

#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <algorithm>
#include <thread>
#include <vector>

#include "step.cuh"

#define QLB_API extern "C" __attribute__((visibility("default")))

namespace qlb {
namespace {

// A term list copied out of the caller's structures (dense factors included).
struct TermCopy {
  std::vector<qlb_term> terms;
  std::vector<std::vector<qlb_factor>> factors;
  std::vector<std::vector<double>> dense;  // one per dense factor, in order
  void copy_from(const qlb_term* t, int n, const std::vector<int>& R) {
    terms.assign(t, t + n);
    factors.resize(n);
    for (int i = 0; i < n; i++) {
      factors[i].assign(t[i].factors, t[i].factors + (t[i].n_factors > 0 ? t[i].n_factors : 0));
      for (auto& f : factors[i]) {
        if (f.kind == QLB_F_DENSE && f.dense && f.mode >= 0 && f.mode < (int)R.size()) {
          long N = 1L << R[f.mode];
          dense.emplace_back(f.dense, f.dense + 2 * N * N);
        } else {
          dense.emplace_back();
        }
      }
    }
    // re-point the copies at the copied storage
    size_t di = 0;
    for (int i = 0; i < n; i++) {
      for (auto& f : factors[i]) {
        if (f.kind == QLB_F_DENSE && !dense[di].empty()) f.dense = dense[di].data();
        di++;
      }
      terms[i].factors = factors[i].empty() ? nullptr : factors[i].data();
    }
  }
};

enum JobState { J_PENDING = 0, J_LIVE = 1, J_DONE = 2, J_FAILED = 3, J_CANCELLED = 4 };

struct Job {
  int64_t ticket = 0;
  std::vector<int> R;
  TermCopy H;
  std::vector<TermCopy> jumps;
  std::vector<TermCopy> obs;
  std::vector<std::vector<double>> vecs;
  double dt = 0;
  int64_t steps = 0, remaining = 0;
  double tol = 0;
  int chi_max = 0, chi_mu_max = 0;
  size_t est = 0;
  double t_arrive = 0, t_admit = 0, t_done = 0;
  std::atomic<int> state{J_PENDING};
  std::atomic<bool> cancel{false};
  std::vector<double> results;  // 2 per observable
  std::string error;
  qlb_status status = QLB_OK;
  // device objects (worker thread only)
  std::string bucket;  // planned shape: requests with equal keys step as one group
  qlb_system* sys = nullptr;
  std::vector<qlb_op*> ops;
  std::vector<qlb_op*> obs_ops;
  qlb_state* st = nullptr;
};

}  // namespace
}  // namespace qlb

using namespace qlb;

// The live requests of one planned shape (sites, precision form, Kraus MPO bonds
// and bond capacities) step together as a group: one launch per phase of the step
// over all of them, on the bucket's own stream.
struct Bucket {
  qlb::GroupExec exec;
  cudaStream_t stream = nullptr;
  cudaEvent_t ev = nullptr;
  std::vector<std::shared_ptr<qlb::Job>> running;  // members of the chunk in flight
};

struct qlb_server {
  qlb_ctx* ctx = nullptr;
  size_t budget = 0;
  int max_live = 0;
  int chunk = 0;
  std::mutex mu;
  std::map<int64_t, std::shared_ptr<Job>> jobs;
  std::deque<std::shared_ptr<Job>> pending;
  std::vector<std::shared_ptr<Job>> live;
  std::map<std::string, Bucket> buckets;  // worker thread only
  int64_t next_ticket = 1;
  size_t used = 0;
  std::atomic<bool> stop{false};
  std::thread worker;
  std::chrono::steady_clock::time_point t0;
  // statistics (written by the worker, read by qlb_server_stats)
  std::atomic<int> n_live{0};
  std::atomic<int> peak_live{0};
  std::atomic<size_t> peak_bytes{0};
  std::atomic<int64_t> completed{0};
  std::atomic<int64_t> steps_done{0};
  std::atomic<int64_t> n_pending{0};
  double now() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  void run();
  bool admit(std::shared_ptr<Job>& j);
  void finish(std::shared_ptr<Job>& j, bool ok);
};

namespace qlb {
namespace {

// Device bytes one request may hold: sites and the step's scratch under the same
// capacity rules as plan_buffers (zip-up bonds <= chi, purification rows chi_mu B,
// an MPO bond of at most 16 per jump term and 24 for the no-jump branch).
size_t estimate_bytes(const Job& j) {
  int L = 0;
  for (int r : j.R) L += r;
  const long B = 1 + (long)j.jumps.size();
  long D = 24;
  for (auto& t : j.jumps) D += 16 * (long)t.terms.size();
  const long chi = j.chi_max, z = std::max<long>(chi, (long)j.chi_mu_max * B);
  const long sites = (long)L * 2 * z * z;
  const long X = z * D * 2 * chi, M = 2 * z * chi * D, C = 2 * z * chi * D;
  const long G = 16 * (2 * z) * (2 * z);  // Gram, projections, split-K partial sums
  const long kraus = (long)L * 4 * D * D;
  return (size_t)16 * (sites + X + M + C + G + kraus) + (size_t)(2u << 20);
}

qlb_status build_job(qlb_ctx* ctx, Job& j) {
  qlb_status s;
  if ((s = qlb_system_create(ctx, (int)j.R.size(), j.R.data(), &j.sys))) return s;
  qlb_op* H = nullptr;
  if (!j.H.terms.empty()) {
    if ((s = qlb_op_build(j.sys, j.H.terms.data(), (int)j.H.terms.size(), 0.0, 0, &H))) return s;
    j.ops.push_back(H);
    if ((s = qlb_set_hamiltonian(j.sys, H, nullptr, nullptr, 0))) return s;
  }
  for (auto& t : j.jumps) {
    qlb_op* L = nullptr;
    if ((s = qlb_op_build(j.sys, t.terms.data(), (int)t.terms.size(), 0.0, 0, &L))) return s;
    j.ops.push_back(L);
    if ((s = qlb_add_jump(j.sys, L))) return s;
  }
  for (auto& t : j.obs) {
    qlb_op* O = nullptr;
    if ((s = qlb_op_build(j.sys, t.terms.data(), (int)t.terms.size(), 0.0, 0, &O))) return s;
    j.obs_ops.push_back(O);
  }
  std::vector<const double*> vp;
  for (auto& v : j.vecs) vp.push_back(v.data());
  if ((s = qlb_state_init_product(j.sys, vp.data(), &j.st))) return s;
  if ((s = qlb_truncate(j.st, j.tol, j.chi_max, j.chi_mu_max)) < 0) return s;
  // the step plan (Kraus MPO and buffers) is made once, before the first chunk
  if ((s = build_kraus(j.st, j.dt))) return s;
  if ((s = plan_buffers(j.st, j.st->kraus))) return s;
  // requests whose plans have the same shape share a group (and so its launches):
  // the same kernels, grids and K splits as each would get alone
  std::string key = std::to_string(j.st->L) + "|" + std::to_string(j.st->prec) + "|" + std::to_string(j.sys->order);
  for (int v : j.st->kraus.D) key += "," + std::to_string(v);
  key += "|";
  for (int v : j.st->cap_state) key += "," + std::to_string(v);
  j.bucket = key;
  return QLB_OK;
}

void release_job(Job& j) {
  if (j.st) qlb_state_destroy(j.st);
  j.st = nullptr;
  for (auto o : j.obs_ops) qlb_op_destroy(o);
  for (auto o : j.ops) qlb_op_destroy(o);
  j.obs_ops.clear();
  j.ops.clear();
  if (j.sys) qlb_system_destroy(j.sys);
  j.sys = nullptr;
}

}  // namespace
}  // namespace qlb

bool qlb_server::admit(std::shared_ptr<Job>& j) {
  j->t_admit = now();
  qlb_status s = build_job(ctx, *j);
  if (s < 0) {
    j->status = s;
    j->error = get_error();
    return false;
  }
  j->remaining = j->steps;
  return true;
}

void qlb_server::finish(std::shared_ptr<Job>& j, bool ok) {
  if (ok && j->st) {
    cudaStreamSynchronize(j->st->stream);
    int err = 0;
    cudaMemcpy(&err, j->st->d_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (err) {
      j->status = (err & 4) ? QLB_ETIMEOUT : (err & 2) ? QLB_ENONFINITE : QLB_ENOTCONV;
      j->error = (err & 4)   ? "a bounded wait of the tensor-core contraction gave up"
                 : (err & 2) ? "non-finite values met in a truncation"
                             : "a Jacobi eigen-solve hit its sweep limit";
      ok = false;
    }
  }
  if (ok) {
    j->results.assign(2 * j->obs_ops.size(), 0.0);
    for (size_t k = 0; k < j->obs_ops.size() && ok; k++) {
      qlb_status s = qlb_expectation(j->st, j->obs_ops[k], &j->results[2 * k]);
      if (s < 0) {
        j->status = s;
        j->error = get_error();
        ok = false;
      }
    }
  }
  release_job(*j);
  j->t_done = now();
  std::lock_guard<std::mutex> lk(mu);
  used -= std::min(used, j->est);
  j->state = j->cancel ? J_CANCELLED : (ok ? J_DONE : J_FAILED);
  if (ok) completed++;
}

void qlb_server::run() {
  cudaSetDevice(ctx->opt.device);
  while (!stop) {
    bool progressed = false;
    // admission: arrival order, a free slot, and the estimate fits next to the live ones
    for (;;) {
      std::shared_ptr<Job> j;
      {
        std::lock_guard<std::mutex> lk(mu);
        while (!pending.empty() && pending.front()->cancel) {
          pending.front()->state = J_CANCELLED;
          pending.pop_front();
        }
        if (pending.empty() || (int)live.size() >= max_live) break;
        j = pending.front();
        if (budget && used + j->est > budget && !live.empty()) break;
        pending.pop_front();
        n_pending = (int64_t)pending.size();
        used += j->est;
      }
      if (admit(j)) {
        j->state = J_LIVE;
        live.push_back(j);
        n_live = (int)live.size();
        if (n_live > peak_live) peak_live = n_live.load();
      } else {
        finish(j, false);
      }
      progressed = true;
    }
    if (ctx->mem_held > peak_bytes) peak_bytes = ctx->mem_held;
    // a bucket whose chunk has finished takes its next one
    for (auto& kv : buckets) {
      Bucket& b = kv.second;
      if (b.running.empty()) continue;
      cudaError_t q = cudaStreamQuery(b.stream);
      if (q == cudaErrorNotReady) {
        cudaGetLastError();
        continue;
      }
      b.running.clear();
    }
    std::map<std::string, std::vector<std::shared_ptr<Job>>> ready;
    for (size_t i = 0; i < live.size();) {
      auto& j = live[i];
      auto bit = buckets.find(j->bucket);
      if (bit != buckets.end() && !bit->second.running.empty()) {
        i++;  // its bucket's chunk is still in flight
        continue;
      }
      if (j->cancel || j->remaining <= 0) {
        progressed = true;
        finish(j, !j->cancel);
        live.erase(live.begin() + i);
        n_live = (int)live.size();
        continue;
      }
      ready[j->bucket].push_back(j);
      i++;
    }
    for (auto& kv : ready) {
      auto& js = kv.second;
      Bucket& b = buckets[kv.first];
      b.exec.ctx = ctx;
      qlb_status s = QLB_OK;
      if (!b.stream && (cudaStreamCreateWithFlags(&b.stream, cudaStreamNonBlocking) != cudaSuccess ||
                        cudaEventCreateWithFlags(&b.ev, cudaEventDisableTiming) != cudaSuccess)) {
        set_error("bucket stream creation failed");
        s = QLB_EDEVICE;
      }
      int64_t n = chunk;
      std::vector<qlb_state*> ms;
      for (auto& j : js) {
        n = std::min<int64_t>(n, j->remaining);
        ms.push_back(j->st);
      }
      if (s == QLB_OK) s = group_run(b.exec, ms, b.stream, b.ev, n, false);  // enqueued, no wait
      progressed = true;
      if (s < 0) {
        const std::string msg = get_error();
        for (auto& j : js) {
          j->status = s;
          j->error = msg;
          finish(j, false);
          live.erase(std::find(live.begin(), live.end(), j));
        }
        n_live = (int)live.size();
        continue;
      }
      for (auto& j : js) j->remaining -= n;
      steps_done += n * (int64_t)js.size();
      b.running = js;
    }
    // buckets without live requests give back their graph and table
    for (auto it = buckets.begin(); it != buckets.end();) {
      bool used = !it->second.running.empty();
      for (auto& j : live) used = used || j->bucket == it->first;
      if (used) {
        ++it;
        continue;
      }
      if (it->second.stream) cudaStreamSynchronize(it->second.stream);
      it->second.exec.release();
      if (it->second.ev) cudaEventDestroy(it->second.ev);
      if (it->second.stream) cudaStreamDestroy(it->second.stream);
      it = buckets.erase(it);
    }
    if (!progressed) std::this_thread::sleep_for(std::chrono::microseconds(100));
  }
  for (auto& kv : buckets)
    if (kv.second.stream) cudaStreamSynchronize(kv.second.stream);
  for (auto& j : live) finish(j, false);
  live.clear();
  for (auto& kv : buckets) {
    kv.second.exec.release();
    if (kv.second.ev) cudaEventDestroy(kv.second.ev);
    if (kv.second.stream) cudaStreamDestroy(kv.second.stream);
  }
  buckets.clear();
}

#define CHECK_ARG(cond, msg) \
  do {                       \
    if (!(cond)) {           \
      set_error(msg);        \
      return QLB_EINVAL;     \
    }                        \
  } while (0)

QLB_API qlb_status qlb_server_create(qlb_ctx* ctx, size_t hbm_budget, int max_live, int chunk, qlb_server** out) {
  CHECK_ARG(ctx && out, "null argument");
  CHECK_ARG(max_live >= 1 && chunk >= 1, "max_live and chunk must be >= 1");
  qlb_server* s = new qlb_server();
  s->ctx = ctx;
  s->budget = hbm_budget;
  s->max_live = max_live;
  s->chunk = chunk;
  s->t0 = std::chrono::steady_clock::now();
  s->worker = std::thread([s]() { s->run(); });
  *out = s;
  return QLB_OK;
}

QLB_API void qlb_server_destroy(qlb_server* s) {
  if (!s) return;
  s->stop = true;
  if (s->worker.joinable()) s->worker.join();
  delete s;
}

QLB_API qlb_status qlb_submit(qlb_server* s, const qlb_request* r, int64_t* ticket) {
  CHECK_ARG(s && r && ticket, "null argument");
  CHECK_ARG(r->n_modes >= 1 && r->n_modes <= 16 && r->R, "bad mode list");
  CHECK_ARG(std::isfinite(r->dt) && r->dt > 0 && r->steps >= 0, "dt must be positive and steps >= 0");
  CHECK_ARG(r->n_jumps >= 0 && r->n_obs >= 0 && (r->n_jumps == 0 || (r->jumps && r->n_jump_terms)) &&
                (r->n_obs == 0 || (r->obs && r->n_obs_terms)) && r->mode_vecs,
            "bad request arrays");
  CHECK_ARG(r->n_H > 0 || r->n_jumps > 0, "a request needs a Hamiltonian or jump operators");
  CHECK_ARG(r->chi_max <= s->ctx->opt.chi_max && r->chi_mu_max <= s->ctx->opt.chi_mu_max,
            "request caps above the server context's caps");
  auto j = std::make_shared<Job>();
  j->R.assign(r->R, r->R + r->n_modes);
  for (int m = 0; m < r->n_modes; m++) CHECK_ARG(j->R[m] >= 1 && j->R[m] <= 12, "R[m] must be in [1, 12]");
  if (r->n_H > 0) j->H.copy_from(r->H, r->n_H, j->R);
  j->jumps.resize(r->n_jumps);
  for (int k = 0; k < r->n_jumps; k++) j->jumps[k].copy_from(r->jumps[k], r->n_jump_terms[k], j->R);
  j->obs.resize(r->n_obs);
  for (int k = 0; k < r->n_obs; k++) j->obs[k].copy_from(r->obs[k], r->n_obs_terms[k], j->R);
  for (int m = 0; m < r->n_modes; m++) {
    CHECK_ARG(r->mode_vecs[m], "null mode vector");
    long N = 1L << j->R[m];
    j->vecs.emplace_back(r->mode_vecs[m], r->mode_vecs[m] + 2 * N);
  }
  j->dt = r->dt;
  j->steps = r->steps;
  j->tol = r->tol;
  j->chi_max = r->chi_max;
  j->chi_mu_max = r->chi_mu_max;
  j->est = estimate_bytes(*j);
  std::lock_guard<std::mutex> lk(s->mu);
  j->ticket = s->next_ticket++;
  j->t_arrive = s->now();
  s->jobs[j->ticket] = j;
  s->pending.push_back(j);
  s->n_pending = (int64_t)s->pending.size();
  *ticket = j->ticket;
  return QLB_OK;
}

QLB_API qlb_status qlb_poll(qlb_server* s, int64_t ticket, double* results, int cap, double* times3) {
  CHECK_ARG(s, "null server");
  std::shared_ptr<Job> j;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->jobs.find(ticket);
    CHECK_ARG(it != s->jobs.end(), "unknown ticket");
    j = it->second;
  }
  const int st = j->state;
  if (st == J_PENDING || st == J_LIVE) return QLB_BUSY;
  if (times3) {
    times3[0] = j->t_arrive;
    times3[1] = j->t_admit;
    times3[2] = j->t_done;
  }
  if (st == J_CANCELLED) {
    set_error("request cancelled");
    return QLB_ESTATE;
  }
  if (st == J_FAILED) {
    set_error(j->error.empty() ? "request failed" : j->error);
    return j->status < 0 ? j->status : QLB_EDEVICE;
  }
  if (results)
    for (int k = 0; k < cap && k < (int)j->results.size(); k++) results[k] = j->results[k];
  return QLB_OK;
}

QLB_API qlb_status qlb_cancel(qlb_server* s, int64_t ticket) {
  CHECK_ARG(s, "null server");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->jobs.find(ticket);
  CHECK_ARG(it != s->jobs.end(), "unknown ticket");
  it->second->cancel = true;
  return QLB_OK;
}

QLB_API qlb_status qlb_server_stats(qlb_server* s, double* out6) {
  CHECK_ARG(s && out6, "null argument");
  out6[0] = (double)s->n_live.load();
  out6[1] = (double)s->peak_live.load();
  out6[2] = (double)s->peak_bytes.load();
  out6[3] = (double)s->completed.load();
  out6[4] = (double)s->steps_done.load();
  out6[5] = (double)s->n_pending.load();
  return QLB_OK;
}

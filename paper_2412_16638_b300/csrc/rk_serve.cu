// Batched stepping (rk_integrate_batch) and the serving loop (rk_server_*).
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <map>
#include <mutex>
#include <tuple>

#include "rk_batch.cuh"
#include "rk_internal.h"

namespace rk {

// Launch-shape autotuner: per (storage, block size, log2 of the work-list
// length) the cap on CTAs per SM of the work-list kernels (0 = the occupancy
// limit).  The per-problem reductions add their partials in item order, so
// the results do not depend on the launch shape: candidates are timed on the
// call's own first steps.
static std::mutex g_tune_mu;
static std::map<std::tuple<int, int, int>, int> g_tune;
static const int kTuneCaps[] = {0, 4, 2};

static rk_status run_group(int storage, rk_problem** ps, int count, double dt, int nsteps, cudaStream_t st, int cap,
                           BatchTotals* tot) {
  switch (storage) {
    case RK_F64: return batch_group_run<double>(ps, count, dt, nsteps, st, cap, tot);
    case RK_F32: return batch_group_run<float>(ps, count, dt, nsteps, st, cap, tot);
    case RK_F16: return batch_group_run<__half>(ps, count, dt, nsteps, st, cap, tot);
    default: return batch_group_run<__nv_bfloat16>(ps, count, dt, nsteps, st, cap, tot);
  }
}

// A group: problems with the same storage, block size, correction mode and
// tableau (the stage loop is shared by the work-list launches).
struct GroupKey {
  int storage, bs, correct, q;
  std::vector<double> tab;
  bool operator<(const GroupKey& o) const {
    return std::tie(storage, bs, correct, q, tab) < std::tie(o.storage, o.bs, o.correct, o.q, o.tab);
  }
};

}  // namespace rk

using namespace rk;

extern "C" rk_status rk_integrate_batch(rk_problem** ps, int count, double dt, int nsteps, rk_stats* stats) {
  NvtxRange range_batch("rk_integrate_batch");
  if (!ps || count < 1) {
    set_error("rk_integrate_batch: need at least one problem");
    return RK_ERR_ARG;
  }
  if (!(dt > 0.0) || !std::isfinite(dt) || nsteps < 0) {
    set_error("rk_integrate_batch: dt must be positive and finite, nsteps >= 0");
    return RK_ERR_ARG;
  }
  for (int i = 0; i < count; ++i) {
    rk_problem* p = ps[i];
    if (!p) {
      set_error("rk_integrate_batch: problem %d is NULL", i);
      return RK_ERR_ARG;
    }
    if (p->desc.op != RK_OP_HEAT7 || p->sol.krylov != RK_KRYLOV_CG || p->sol.precond != RK_PREC_BLOCK_JACOBI ||
        p->src) {
      set_error("rk_integrate_batch: problem %d is not a heat/CG/block-Jacobi problem without forcing", i);
      return RK_ERR_ARG;
    }
    if (p->ke_hi || p->sol.tol_true > 0.0) {
      set_error("rk_integrate_batch: problem %d refines its solves against the true residual (tol_true > 0), "
                "which the batched kernels do not; step it with rk_integrate",
                i);
      return RK_ERR_ARG;
    }
    if (p->q == 0) {
      set_error("rk_integrate_batch: problem %d has no tableau", i);
      return RK_ERR_ARG;
    }
    for (int j = 0; j < i; ++j)
      if (ps[j] == p) {
        set_error("rk_integrate_batch: problem %d appears twice", i);
        return RK_ERR_ARG;
      }
  }
  for (int i = 0; i < count; ++i) ps[i]->batch_status = RK_OK;
  auto t0 = std::chrono::steady_clock::now();
  cudaStream_t user = ps[0]->st;
  for (int i = 1; i < count; ++i)
    if (ps[i]->st != user) RK_CUDA(cudaStreamSynchronize(ps[i]->st));
  std::map<GroupKey, std::vector<rk_problem*>> groups;
  for (int i = 0; i < count; ++i) {
    rk_problem* p = ps[i];
    GroupKey k{p->sol.storage, p->sol.bj_block, p->sol.correct ? 1 : 0, p->q, {}};
    k.tab.assign(p->Ah, p->Ah + p->q * p->q);
    k.tab.insert(k.tab.end(), p->Al, p->Al + p->q * p->q);
    k.tab.insert(k.tab.end(), p->b, p->b + p->q);
    groups[k].push_back(p);
  }
  BatchTotals tot;
  rk_status status = RK_OK;
  for (auto& kv : groups) {
    std::vector<rk_problem*>& g = kv.second;
    // largest problems first: their items head the work list
    std::stable_sort(g.begin(), g.end(), [](rk_problem* a, rk_problem* b) { return a->N > b->N; });
    long long items = 0;
    for (auto* p : g) {
      const int seg = kv.first.storage == RK_F16 || kv.first.storage == RK_BF16 ? std::max(8, kv.first.bs)
                                                                                   : std::max(4, kv.first.bs);
      items += ((long long)p->n * p->n * ((p->n + seg - 1) / seg) + kThreads - 1) / kThreads;
    }
    const auto key = std::make_tuple(kv.first.storage, kv.first.bs, (int)std::log2((double)items + 1.0));
    const long long launches_before = tot.launches;
    int cap = -1;
    if (const char* env = std::getenv("RK_BATCH_GRID_CAP")) {
      // a fixed launch shape (CTAs per SM of the work-list kernels, 0 = the
      // occupancy limit) instead of the autotuned one
      char* end = nullptr;
      const long v = std::strtol(env, &end, 10);
      if (end != env && v >= 0 && v <= 64) cap = (int)v;
    }
    if (cap < 0) {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      auto it = g_tune.find(key);
      if (it != g_tune.end()) cap = it->second;
    }
    int done = 0;
    if (cap < 0) {
      // autotune on the call's own steps (results do not depend on the shape)
      double best = 1e30;
      int best_cap = 0;
      for (int c : kTuneCaps) {
        if (done >= nsteps) break;
        cudaStreamSynchronize(user);
        auto a = std::chrono::steady_clock::now();
        status = run_group(kv.first.storage, g.data(), (int)g.size(), dt, 1, user, c, &tot);
        const double sec = std::chrono::duration<double>(std::chrono::steady_clock::now() - a).count();
        if (status != RK_OK) break;
        ++done;
        if (sec < best) {
          best = sec;
          best_cap = c;
        }
      }
      if (status != RK_OK) break;
      if (done == (int)(sizeof(kTuneCaps) / sizeof(kTuneCaps[0]))) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune[key] = best_cap;
      }
      cap = best_cap;
    }
    if (done < nsteps) status = run_group(kv.first.storage, g.data(), (int)g.size(), dt, nsteps - done, user, cap, &tot);
    if (status != RK_OK) break;
    for (auto* p : g) p->launches += tot.launches - launches_before;
  }
  // the batched kernels keep k^eps in padded lines: it is no initial guess for
  // a later single-problem solve
  for (int i = 0; i < count; ++i)
    for (auto& v : ps[i]->warm_valid) v = false;
  rk_stats acc{};
  acc.iters_total = tot.iters_total;
  acc.iters_max = tot.iters_max;
  acc.solves = tot.solves;
  acc.not_converged = tot.not_converged;
  acc.true_res = tot.true_res;
  acc.bytes = tot.bytes;
  acc.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (stats) *stats = acc;
  if (status != RK_OK) return status;
  if (tot.nonfinite) {
    set_error("rk_integrate_batch: non-finite value or CG breakdown in %d problem(s)", tot.nonfinite);
    return RK_ERR_NONFINITE;
  }
  return acc.not_converged ? RK_ERR_NOT_CONVERGED : RK_OK;
}

// ----------------------------------------------------------------- server
// Continuous batching of time-integration jobs.  A worker thread owns the
// device state of every resident job.  Each tick it (1) admits queued jobs in
// arrival order while a slot is free and their estimated footprint fits the
// HBM budget (first fit: a job that fits may pass a larger one ahead of it),
// (2) advances every resident job by one step -- all small heat/CG jobs of a
// step size together in one persistent batched launch, every other job on
// its own stream from a pool of host threads, so their kernels overlap on the
// device -- and (3) retires finished jobs: the state is copied to host memory,
// the device memory is freed and waiters are woken.
#include <condition_variable>
#include <deque>
#include <functional>
#include <memory>
#include <thread>
#include <unordered_map>

namespace rk {

enum JobState { JOB_PENDING, JOB_ACTIVE, JOB_DONE };

struct Job {
  uint64_t id = 0;
  rk_problem_desc desc{};
  std::vector<double> kappa;  // copy of kappa_field
  std::vector<double> source;  // copy of the forcing term
  rk_solver_desc sol{};
  int q = 0;
  std::vector<double> Ah, Al, b, u0;
  double dt = 0.0;
  int nsteps = 0, done_steps = 0;
  size_t est_bytes = 0;
  rk_problem* p = nullptr;
  cudaStream_t stream = nullptr;
  JobState state = JOB_PENDING;
  rk_status status = RK_OK;
  std::string error;
  rk_stats stats{};
  std::vector<double> result;
  std::chrono::steady_clock::time_point t_submit, t_admit, t_first, t_done;
  long long first_tick = -1, last_tick = -1;  // server ticks in which the job stepped
};

constexpr int kBatchMaxN = 64;  // jobs up to this size step in the batched kernel

// Estimated device footprint of a job (what rk_create_problem + rk_set_tableau allocate).
static size_t job_footprint(const rk_problem_desc& d, const rk_solver_desc& s, int q, const double* Al) {
  const size_t N = (size_t)d.n * d.n * d.n;
  const size_t sb = dtype_size(s.storage), xb = xsize(s.storage);
  size_t implicit = 0;
  for (int i = 0; i < q; ++i)
    if (Al[i * q + i] != 0.0) ++implicit;
  size_t bytes = N * 8 * 3 + N * sb * 4 + N * 8 * q + N * xb * implicit + N * xb + (1u << 20);
  if (d.source) bytes += N * 8;
  if (d.op != RK_OP_HEAT7) {
    const size_t nnz = N * 7;
    bytes += nnz * (4 + 8 + sb) + (N + 1) * 4 + (size_t)(s.restart + 2) * N * sb + N * s.bj_block * sb * 4;
  }
  if (s.precond == RK_PREC_FDM) bytes += N * sb + (size_t)d.n * d.n * sb;
  return bytes;
}

class Pool {
 public:
  explicit Pool(int n) {
    for (int i = 0; i < n; ++i) threads_.emplace_back([this] { run(); });
  }
  ~Pool() {
    {
      std::lock_guard<std::mutex> lk(mu_);
      stop_ = true;
    }
    cv_.notify_all();
    for (auto& t : threads_) t.join();
  }
  // run all tasks, return when every one has finished
  void run_all(std::vector<std::function<void()>>& tasks) {
    std::unique_lock<std::mutex> lk(mu_);
    for (auto& t : tasks) q_.push_back(&t);
    pending_ += (int)tasks.size();
    cv_.notify_all();
    done_cv_.wait(lk, [&] { return pending_ == 0; });
  }

 private:
  void run() {
    while (true) {
      std::function<void()>* t = nullptr;
      {
        std::unique_lock<std::mutex> lk(mu_);
        cv_.wait(lk, [&] { return stop_ || !q_.empty(); });
        if (stop_ && q_.empty()) return;
        t = q_.front();
        q_.pop_front();
      }
      (*t)();
      std::lock_guard<std::mutex> lk(mu_);
      if (--pending_ == 0) done_cv_.notify_all();
    }
  }
  std::vector<std::thread> threads_;
  std::deque<std::function<void()>*> q_;
  std::mutex mu_;
  std::condition_variable cv_, done_cv_;
  int pending_ = 0;
  bool stop_ = false;
};

static void add_stats(rk_stats& a, const rk_stats& b) {
  a.iters_total += b.iters_total;
  a.iters_max = std::max(a.iters_max, b.iters_max);
  a.solves += b.solves;
  a.refinements += b.refinements;
  a.not_converged += b.not_converged;
  a.true_res = std::max(a.true_res, b.true_res);
}

}  // namespace rk

struct rk_server {
  size_t budget = 0;
  int max_slots = 0;
  int device = 0;
  std::mutex mu;
  std::condition_variable cv;       // wakes the worker
  std::condition_variable done_cv;  // wakes waiters
  std::deque<std::shared_ptr<rk::Job>> pending;
  std::vector<std::shared_ptr<rk::Job>> active;
  std::unordered_map<uint64_t, std::shared_ptr<rk::Job>> jobs;
  uint64_t next_id = 1;
  size_t used = 0;
  bool stop = false;
  long long tick = 0;  // rounds of one step for every resident job
  std::chrono::steady_clock::time_point t0;  // creation time
  std::thread worker;
  std::unique_ptr<rk::Pool> pool;
};

namespace rk {

static void finish_job(rk_server* s, const std::shared_ptr<Job>& j, rk_status st, const std::string& err) {
  if (j->p) {
    if (st == RK_OK || st == RK_ERR_NOT_CONVERGED) {
      j->result.resize((size_t)j->p->N);
      rk_status gs = rk_get_state(j->p, j->result.data(), 0);
      if (gs != RK_OK) {
        st = gs;
        j->result.clear();
      }
    }
    rk_destroy_problem(j->p);
    j->p = nullptr;
  }
  if (j->stream) {
    cudaStreamDestroy(j->stream);
    j->stream = nullptr;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  s->used -= j->est_bytes;
  j->status = st;
  j->error = err;
  j->t_done = std::chrono::steady_clock::now();
  j->state = JOB_DONE;
  s->done_cv.notify_all();
}

// Create the device state of an admitted job.
static rk_status start_job(Job& j) {
  if (cudaStreamCreateWithFlags(&j.stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    set_error("server: stream creation failed");
    return RK_ERR_CUDA;
  }
  rk_problem_desc d = j.desc;
  d.kappa_field = j.kappa.empty() ? nullptr : j.kappa.data();
  d.source = j.source.empty() ? nullptr : j.source.data();
  RK_TRY(rk_create_problem(&d, &j.sol, j.stream, &j.p));
  RK_TRY(rk_set_tableau(j.p, j.q, j.Ah.data(), j.Al.data(), j.b.data()));
  RK_TRY(rk_set_state(j.p, j.u0.data(), 0));
  return RK_OK;
}

static void worker_loop(rk_server* s) {
  cudaSetDevice(s->device);
  while (true) {
    std::vector<std::shared_ptr<Job>> admitted;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv.wait(lk, [&] { return s->stop || !s->pending.empty() || !s->active.empty(); });
      if (s->stop && s->active.empty()) break;
      if (!s->stop) {
        for (auto it = s->pending.begin(); it != s->pending.end();) {
          if ((int)(s->active.size() + admitted.size()) >= s->max_slots) break;
          if (s->used + (*it)->est_bytes <= s->budget) {
            s->used += (*it)->est_bytes;
            (*it)->state = JOB_ACTIVE;
            (*it)->t_admit = std::chrono::steady_clock::now();
            admitted.push_back(*it);
            it = s->pending.erase(it);
          } else {
            ++it;
          }
        }
      }
    }
    for (auto& j : admitted) {
      rk_status st = start_job(*j);
      if (st != RK_OK) {
        finish_job(s, j, st, rk_last_error());
        continue;
      }
      if (j->nsteps == 0) {
        finish_job(s, j, RK_OK, "");
        continue;
      }
      std::lock_guard<std::mutex> lk(s->mu);
      s->active.push_back(j);
    }
    std::vector<std::shared_ptr<Job>> act;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      act = s->active;
    }
    if (act.empty()) continue;
    // one step for every resident job: this tick's index and start time
    const long long tick = s->tick++;
    NvtxRange range_tick("serve tick");
    {
      const auto now = std::chrono::steady_clock::now();
      std::lock_guard<std::mutex> lk(s->mu);
      for (auto& j : act) {
        if (j->first_tick < 0) {
          j->first_tick = tick;
          j->t_first = now;
        }
        j->last_tick = tick;
      }
    }
    std::map<double, std::vector<std::shared_ptr<Job>>> small;  // by step size
    std::vector<std::function<void()>> tasks;
    std::vector<rk_status> results(act.size(), RK_OK);
    std::vector<std::string> errors(act.size());
    std::vector<rk_stats> stepstats(act.size());
    for (size_t i = 0; i < act.size(); ++i) {
      Job* j = act[i].get();
      if (j->desc.op == RK_OP_HEAT7 && j->sol.krylov == RK_KRYLOV_CG && j->sol.precond == RK_PREC_BLOCK_JACOBI &&
          j->source.empty() && j->desc.n <= kBatchMaxN && !(j->sol.tol_true > 0.0)) {
        small[j->dt].push_back(act[i]);
      } else {
        tasks.push_back([&, i, j] {
          cudaSetDevice(s->device);
          results[i] = rk_step(j->p, j->dt, &stepstats[i]);
          if (results[i] != RK_OK) errors[i] = rk_last_error();
        });
      }
    }
    for (auto& kv : small) {
      const double dt = kv.first;
      auto group = kv.second;
      tasks.push_back([&, dt, group] {
        cudaSetDevice(s->device);
        std::vector<rk_problem*> ps;
        for (auto& j : group) ps.push_back(j->p);
        rk_stats bst{};
        rk_status st = rk_integrate_batch(ps.data(), (int)ps.size(), dt, 1, &bst);
        const std::string err = st == RK_OK ? "" : rk_last_error();
        // each job gets its own outcome: a job that went non-finite fails
        // alone, the others of the group were stepped correctly
        const bool per_problem = st == RK_OK || st == RK_ERR_NOT_CONVERGED || st == RK_ERR_NONFINITE;
        for (auto& j : group) {
          for (size_t i = 0; i < act.size(); ++i)
            if (act[i] == j) {
              results[i] = per_problem ? j->p->batch_status : st;
              errors[i] = results[i] == RK_ERR_NONFINITE ? "non-finite value or CG breakdown in the batched step"
                                                         : (per_problem ? "" : err);
            }
        }
        // per-job iteration statistics are not separated in a batched step;
        // the group's totals are attributed in proportion to the job count
        for (auto& j : group) {
          j->stats.solves += bst.solves / (int)group.size();
          j->stats.iters_total += bst.iters_total / (long long)group.size();
          j->stats.iters_max = std::max(j->stats.iters_max, bst.iters_max);
        }
      });
    }
    s->pool->run_all(tasks);
    for (size_t i = 0; i < act.size(); ++i) {
      auto& j = act[i];
      add_stats(j->stats, stepstats[i]);
      const rk_status st = results[i];
      if (st == RK_ERR_NOT_CONVERGED && j->status == RK_OK) j->status = st;
      const bool failed = st != RK_OK && st != RK_ERR_NOT_CONVERGED;
      if (!failed) j->done_steps += 1;
      if (failed || j->done_steps >= j->nsteps) {
        {
          std::lock_guard<std::mutex> lk(s->mu);
          s->active.erase(std::find(s->active.begin(), s->active.end(), j));
        }
        finish_job(s, j, failed ? st : j->status, failed ? errors[i] : "");
      }
    }
  }
}

}  // namespace rk

extern "C" {

rk_status rk_server_create(size_t hbm_budget_bytes, int max_slots, rk_server** out) {
  if (!out || hbm_budget_bytes == 0 || max_slots < 1 || max_slots > 4096) {
    set_error("rk_server_create: need out != NULL, budget > 0 and 1 <= max_slots <= 4096");
    return RK_ERR_ARG;
  }
  rk_server* s = new rk_server();
  s->budget = hbm_budget_bytes;
  s->max_slots = max_slots;
  s->t0 = std::chrono::steady_clock::now();
  cudaGetDevice(&s->device);
  s->pool.reset(new Pool(8));
  s->worker = std::thread(worker_loop, s);
  *out = s;
  return RK_OK;
}

rk_status rk_submit_job(rk_server* s, const rk_problem_desc* desc, const rk_solver_desc* solver, int q,
                        const double* A_hi, const double* A_lo, const double* b, const double* u0, double dt,
                        int nsteps, uint64_t* job_id) {
  if (!s || !desc || !solver || !A_hi || !A_lo || !b || !u0 || !job_id) {
    set_error("rk_submit_job: NULL argument");
    return RK_ERR_ARG;
  }
  if (q < 1 || q > kMaxStages || !(dt > 0.0) || !std::isfinite(dt) || nsteps < 0) {
    set_error("rk_submit_job: need 1 <= q <= 8, dt > 0 finite, nsteps >= 0");
    return RK_ERR_ARG;
  }
  if (desc->n < 1 || desc->n > 1024 ||
      (desc->op != RK_OP_HEAT7 && desc->op != RK_OP_ADVDIFF_CSR && desc->op != RK_OP_ADV_PERIODIC) ||
      (desc->op == RK_OP_ADVDIFF_CSR && !desc->kappa_field)) {
    set_error("rk_submit_job: invalid problem descriptor");
    return RK_ERR_ARG;
  }
  auto j = std::make_shared<Job>();
  j->desc = *desc;
  const size_t N = (size_t)desc->n * desc->n * desc->n;
  if (desc->kappa_field) j->kappa.assign(desc->kappa_field, desc->kappa_field + N);
  if (desc->source) j->source.assign(desc->source, desc->source + N);
  j->desc.kappa_field = nullptr;
  j->desc.source = nullptr;
  j->sol = *solver;
  j->q = q;
  j->Ah.assign(A_hi, A_hi + q * q);
  j->Al.assign(A_lo, A_lo + q * q);
  j->b.assign(b, b + q);
  j->u0.assign(u0, u0 + N);
  j->dt = dt;
  j->nsteps = nsteps;
  j->est_bytes = job_footprint(*desc, *solver, q, A_lo);
  j->t_submit = std::chrono::steady_clock::now();
  j->stats.true_res = -1.0;
  if (j->est_bytes > s->budget) {
    set_error("rk_submit_job: job needs about %zu bytes, more than the server budget %zu", j->est_bytes, s->budget);
    return RK_ERR_OOM;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stop) {
    set_error("rk_submit_job: server is shutting down");
    return RK_ERR_BUSY;
  }
  j->id = s->next_id++;
  s->jobs[j->id] = j;
  s->pending.push_back(j);
  *job_id = j->id;
  s->cv.notify_all();
  return RK_OK;
}

rk_status rk_poll_job(rk_server* s, uint64_t job_id, int* done) {
  if (!s || !done) {
    set_error("rk_poll_job: NULL argument");
    return RK_ERR_ARG;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->jobs.find(job_id);
  if (it == s->jobs.end()) {
    set_error("rk_poll_job: unknown job %llu", (unsigned long long)job_id);
    return RK_ERR_NOT_FOUND;
  }
  *done = it->second->state == JOB_DONE;
  return RK_OK;
}

rk_status rk_wait_job_info(rk_server* s, uint64_t job_id, double* u_out, rk_stats* stats, rk_job_info* info) {
  if (!s) {
    set_error("rk_wait_job: NULL server");
    return RK_ERR_ARG;
  }
  std::shared_ptr<Job> j;
  {
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) {
      set_error("rk_wait_job: unknown job %llu", (unsigned long long)job_id);
      return RK_ERR_NOT_FOUND;
    }
    j = it->second;
    s->done_cv.wait(lk, [&] { return j->state == JOB_DONE; });
    s->jobs.erase(job_id);
  }
  if (u_out && !j->result.empty()) std::memcpy(u_out, j->result.data(), j->result.size() * sizeof(double));
  if (stats) {
    *stats = j->stats;
    stats->seconds = std::chrono::duration<double>(j->t_done - j->t_admit).count();
  }
  if (info) {
    auto since = [&](std::chrono::steady_clock::time_point t) {
      return std::chrono::duration<double>(t - s->t0).count();
    };
    info->t_submit = since(j->t_submit);
    const bool admitted = j->t_admit.time_since_epoch().count() != 0;
    const bool finished = j->t_done.time_since_epoch().count() != 0;  // cancelled jobs never finish
    info->t_admit = admitted ? since(j->t_admit) : -1.0;
    info->t_first_step = j->first_tick >= 0 ? since(j->t_first) : -1.0;
    info->t_done = finished ? since(j->t_done) : -1.0;
    info->first_tick = j->first_tick;
    info->last_tick = j->last_tick;
    info->steps = j->done_steps;
  }
  if (j->status != RK_OK && j->status != RK_ERR_NOT_CONVERGED) set_error("job %llu failed: %s",
                                                                          (unsigned long long)job_id, j->error.c_str());
  return j->status;
}

rk_status rk_wait_job(rk_server* s, uint64_t job_id, double* u_out, rk_stats* stats, double* latency_s) {
  rk_job_info info{};
  const rk_status st = rk_wait_job_info(s, job_id, u_out, stats, &info);
  if (latency_s) *latency_s = info.t_done >= 0.0 ? info.t_done - info.t_submit : -1.0;
  return st;
}

rk_status rk_server_destroy(rk_server* s) {
  if (!s) {
    set_error("rk_server_destroy: NULL server");
    return RK_ERR_ARG;
  }
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    // jobs never admitted are cancelled
    for (auto& j : s->pending) {
      j->state = JOB_DONE;
      j->status = RK_ERR_BUSY;
      j->error = "server destroyed before the job was admitted";
    }
    s->pending.clear();
    s->cv.notify_all();
    s->done_cv.notify_all();
  }
  s->worker.join();  // resident jobs run to completion first
  s->pool.reset();
  delete s;
  return RK_OK;
}

}  // extern "C"

// Batched stepping (rk_integrate_batch) and the serving loop (rk_server_*).
#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>

#include "rk_batch.cuh"
#include "rk_internal.h"

namespace rk {

// Autotuner cache: (storage, bs, problem-count bucket, log2 of total DOF) ->
// best launch shape.
static std::mutex g_tune_mu;
static std::map<std::tuple<int, int, int, int>, LaunchCfg> g_tune;

static int batch_grid(int storage, int bs, const LaunchCfg& cfg, int count) {
  switch (storage) {
    case RK_F64: return batch_grid_s<double>(bs, cfg, count, device_sms());
    case RK_F32: return batch_grid_s<float>(bs, cfg, count, device_sms());
    case RK_F16: return batch_grid_s<__half>(bs, cfg, count, device_sms());
    default: return batch_grid_s<__nv_bfloat16>(bs, cfg, count, device_sms());
  }
}

static void launch_batch(int storage, int bs, const LaunchCfg& cfg, int grid, BatchItem* items, const int* order,
                         int count, double dt, int* counter, cudaStream_t st) {
  switch (storage) {
    case RK_F64: batch_launch_s<double>(bs, cfg, grid, items, order, count, dt, counter, st); break;
    case RK_F32: batch_launch_s<float>(bs, cfg, grid, items, order, count, dt, counter, st); break;
    case RK_F16: batch_launch_s<__half>(bs, cfg, grid, items, order, count, dt, counter, st); break;
    default: batch_launch_s<__nv_bfloat16>(bs, cfg, grid, items, order, count, dt, counter, st); break;
  }
}

struct Group {
  int storage, bs;
  std::vector<rk_problem*> ps;
  std::vector<BatchItem> h_items;
  BatchItem* d_items = nullptr;
  int* d_order = nullptr;
  int* d_counter = nullptr;
  LaunchCfg cfg;
};

static rk_status fill_item(rk_problem* p, double dt, BatchItem& it) {
  std::memset(&it, 0, sizeof(it));
  it.n = p->n;
  it.q = p->q;
  it.correct = p->sol.correct;
  it.max_iter = p->sol.max_iter;
  it.c = p->c;
  it.tol_rel = p->sol.tol_rel;
  it.tol_abs = p->sol.tol_abs;
  std::memcpy(it.Ah, p->Ah, sizeof(it.Ah));
  std::memcpy(it.Al, p->Al, sizeof(it.Al));
  std::memcpy(it.b, p->b, sizeof(it.b));
  it.u = p->u;
  it.r = p->r;
  it.g64 = p->g64;
  for (int i = 0; i < 8; ++i) {
    it.k[i] = p->k[i];
    it.ke[i] = p->ke[i];
    it.minv[i] = nullptr;
  }
  it.wr = p->wr;
  it.wz = p->wz;
  it.wp[0] = p->wp[0];
  it.wp[1] = p->wp[1];
  it.want_scale = p->sol.storage == RK_F16;
  for (int i = 0; i < p->q; ++i) {
    const double a = p->Al[i * p->q + i];
    if (a != 0.0) {
      const void* m = nullptr;
      RK_TRY(get_minv(p, dt * a, &m));
      it.minv[i] = m;
    }
  }
  it.true_res_max = -1.0;
  return RK_OK;
}

// Pick the launch shape of a group by timing one step of every candidate on
// scratch copies of the states (so tuning never changes a result).
static rk_status autotune(Group& gr, double dt, cudaStream_t st) {
  long long dof = 0;
  for (auto* p : gr.ps) dof += p->N;
  const int cbucket = (int)std::log2((double)gr.ps.size() + 1.0);
  const int dbucket = (int)std::log2((double)dof + 1.0);
  const auto key = std::make_tuple(gr.storage, gr.bs, cbucket, dbucket);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) {
      gr.cfg = it->second;
      return RK_OK;
    }
  }
  // scratch copies of u
  std::vector<double*> copies(gr.ps.size(), nullptr);
  std::vector<BatchItem> trial = gr.h_items;
  rk_status status = RK_OK;
  for (size_t i = 0; i < gr.ps.size() && status == RK_OK; ++i) {
    if (cudaMalloc((void**)&copies[i], (size_t)gr.ps[i]->N * 8) != cudaSuccess) {
      cudaGetLastError();
      copies[i] = nullptr;
      status = RK_ERR_OOM;
      break;
    }
    cudaMemcpyAsync(copies[i], gr.ps[i]->u, (size_t)gr.ps[i]->N * 8, cudaMemcpyDeviceToDevice, st);
    trial[i].u = copies[i];
  }
  BatchItem* d_trial = nullptr;
  if (status == RK_OK && cudaMalloc((void**)&d_trial, trial.size() * sizeof(BatchItem)) != cudaSuccess) {
    cudaGetLastError();
    status = RK_ERR_OOM;
  }
  LaunchCfg best;
  if (status == RK_OK) {
    cudaMemcpyAsync(d_trial, trial.data(), trial.size() * sizeof(BatchItem), cudaMemcpyHostToDevice, st);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best_ms = 1e30f;
    const LaunchCfg cands[] = {{256, 2}, {256, 4}, {512, 1}, {512, 2}};
    for (const auto& c : cands) {
      const int grid = batch_grid(gr.storage, gr.bs, c, (int)gr.ps.size());
      cudaEventRecord(e0, st);
      launch_batch(gr.storage, gr.bs, c, grid, d_trial, gr.d_order, (int)gr.ps.size(), dt, gr.d_counter, st);
      cudaEventRecord(e1, st);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (cudaGetLastError() == cudaSuccess && ms < best_ms) {
        best_ms = ms;
        best = c;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  }
  cudaStreamSynchronize(st);
  for (auto* c : copies)
    if (c) cudaFree(c);
  if (d_trial) cudaFree(d_trial);
  if (status != RK_OK) {
    set_error("batch autotune: out of device memory for scratch copies");
    return status;
  }
  gr.cfg = best;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[key] = best;
  return RK_OK;
}

}  // namespace rk

using namespace rk;

extern "C" rk_status rk_integrate_batch(rk_problem** ps, int count, double dt, int nsteps, rk_stats* stats) {
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
                "which the batched kernel does not; step it with rk_integrate",
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
  auto t0 = std::chrono::steady_clock::now();
  cudaStream_t user = ps[0]->st;
  for (int i = 1; i < count; ++i)
    if (ps[i]->st != user) RK_CUDA(cudaStreamSynchronize(ps[i]->st));
  // group by (storage, block size), largest problems first within a group
  std::map<std::pair<int, int>, Group> groups;
  for (int i = 0; i < count; ++i) {
    auto key = std::make_pair(ps[i]->sol.storage, ps[i]->sol.bj_block);
    Group& g = groups[key];
    g.storage = key.first;
    g.bs = key.second;
    g.ps.push_back(ps[i]);
  }
  cudaStream_t cs = nullptr;
  RK_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  RK_CUDA(cudaStreamSynchronize(user));
  rk_status status = RK_OK;
  auto fail = [&](rk_status s) {
    status = s;
    return s;
  };
  for (auto& kv : groups) {
    Group& g = kv.second;
    std::stable_sort(g.ps.begin(), g.ps.end(), [](rk_problem* a, rk_problem* b) { return a->N > b->N; });
    g.h_items.resize(g.ps.size());
    for (size_t i = 0; i < g.ps.size() && status == RK_OK; ++i) fail(fill_item(g.ps[i], dt, g.h_items[i]));
    if (status != RK_OK) break;
    std::vector<int> order(g.ps.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
    if (cudaMalloc((void**)&g.d_items, g.h_items.size() * sizeof(BatchItem)) != cudaSuccess ||
        cudaMalloc((void**)&g.d_order, order.size() * sizeof(int)) != cudaSuccess ||
        cudaMalloc((void**)&g.d_counter, sizeof(int)) != cudaSuccess) {
      cudaGetLastError();
      set_error("rk_integrate_batch: descriptor allocation failed");
      fail(RK_ERR_OOM);
      break;
    }
    cudaMemcpyAsync(g.d_items, g.h_items.data(), g.h_items.size() * sizeof(BatchItem), cudaMemcpyHostToDevice, cs);
    cudaMemcpyAsync(g.d_order, order.data(), order.size() * sizeof(int), cudaMemcpyHostToDevice, cs);
    if (fail(autotune(g, dt, cs)) != RK_OK) break;
    g.cfg.grid = batch_grid(g.storage, g.bs, g.cfg, (int)g.ps.size());
  }
  if (status == RK_OK && nsteps > 0) {
    // all steps of all groups as one CUDA graph: one persistent launch per
    // group and step, no host involvement between steps
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      for (int s = 0; s < nsteps; ++s)
        for (auto& kv : groups) {
          Group& g = kv.second;
          launch_batch(g.storage, g.bs, g.cfg, g.cfg.grid, g.d_items, g.d_order, (int)g.ps.size(), dt, g.d_counter,
                       cs);
        }
      e = cudaStreamEndCapture(cs, &graph);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    if (e == cudaSuccess) {
      for (auto& kv : groups)
        for (auto* p : kv.second.ps) p->launches += nsteps;
      e = cudaGraphLaunch(exec, cs);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      set_error("rk_integrate_batch: graph capture/launch failed: %s", cudaGetErrorString(e));
      status = RK_ERR_CUDA;
    }
  }
  rk_stats acc{};
  acc.true_res = -1.0;
  bool nonfinite = false;
  if (status == RK_OK) {
    for (auto& kv : groups) {
      Group& g = kv.second;
      std::vector<BatchItem> out(g.h_items.size());
      if (cudaMemcpy(out.data(), g.d_items, out.size() * sizeof(BatchItem), cudaMemcpyDeviceToHost) != cudaSuccess) {
        set_error("rk_integrate_batch: result readback failed");
        status = RK_ERR_CUDA;
        break;
      }
      for (auto& it : out) {
        acc.iters_total += it.iters_total;
        acc.iters_max = std::max(acc.iters_max, it.iters_max);
        acc.solves += it.solves;
        acc.not_converged += it.not_converged;
        acc.true_res = std::max(acc.true_res, it.true_res_max);
        if (it.status == 5) nonfinite = true;
      }
    }
  }
  for (auto& kv : groups) {
    Group& g = kv.second;
    if (g.d_items) cudaFree(g.d_items);
    if (g.d_order) cudaFree(g.d_order);
    if (g.d_counter) cudaFree(g.d_counter);
  }
  cudaStreamDestroy(cs);
  acc.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (stats) *stats = acc;
  if (status != RK_OK) return status;
  if (nonfinite) {
    set_error("rk_integrate_batch: non-finite value or CG breakdown in a problem");
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
        for (auto& j : group) {
          for (size_t i = 0; i < act.size(); ++i)
            if (act[i] == j) {
              results[i] = st;
              errors[i] = err;
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

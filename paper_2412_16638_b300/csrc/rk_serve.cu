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
    if (p->desc.op != RK_OP_HEAT7 || p->sol.krylov != RK_KRYLOV_CG) {
      set_error("rk_integrate_batch: problem %d is not a heat/CG problem", i);
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
extern "C" {
rk_status rk_server_create(size_t, int, rk_server**) { set_error("not built yet"); return RK_ERR_ARG; }
rk_status rk_submit_job(rk_server*, const rk_problem_desc*, const rk_solver_desc*, int, const double*, const double*,
                        const double*, const double*, double, int, uint64_t*) { set_error("not built yet"); return RK_ERR_ARG; }
rk_status rk_poll_job(rk_server*, uint64_t, int*) { set_error("not built yet"); return RK_ERR_ARG; }
rk_status rk_wait_job(rk_server*, uint64_t, double*, rk_stats*, double*) { set_error("not built yet"); return RK_ERR_ARG; }
rk_status rk_server_destroy(rk_server*) { set_error("not built yet"); return RK_ERR_ARG; }
}

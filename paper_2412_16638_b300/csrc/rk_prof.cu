// Launch profiler: CUDA event pairs around kernel launches on a problem's
// stream, harvested into per-kernel totals.
#include "rk_internal.h"

namespace rk {

const char* const kKernelNames[K_COUNT] = {
    "cg_init", "cg_sweep_a", "cg_sweep_b", "op_apply_f64", "correct_f64", "combine_f64", "vec_norms_f64",
    "widen_f64", "true_residual_f64", "add_scaled", "bj_apply", "csr_spmv", "csr_correct_f64", "csr_bj_setup",
    "gmres_init", "gmres_arnoldi", "gmres_orth", "gmres_update", "gmres_precond", "batch_step",
    "fdm_pass", "fdm_pass_scale", "fdm_pass_dot", "cfdm_pass"};

static cudaEvent_t take_event(Prof* pr) {
  if (!pr->pool.empty()) {
    cudaEvent_t e = pr->pool.back();
    pr->pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

static void harvest(rk_problem* p) {
  Prof* pr = p->prof;
  if (!pr || pr->pending.empty()) return;
  cudaStreamSynchronize(p->st);
  for (auto& r : pr->pending) {
    float ms = 0.f;
    if (r.b && cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) ms = 0.f;
    if (r.noop) {
      pr->noop[r.kid] += 1;
    } else {
      pr->n[r.kid] += 1;
      pr->ms[r.kid] += ms;
      pr->bytes[r.kid] += r.bytes;
    }
    pr->pool.push_back(r.a);
    if (r.b) pr->pool.push_back(r.b);
  }
  pr->pending.clear();
  cudaGetLastError();
}

void prof_begin(rk_problem* p, int kid, double bytes, int solve, int idx) {
  p->launches += 1;
  Prof* pr = p->prof;
  if (!pr || !pr->on) return;
  if (pr->pending.size() >= 65536) harvest(p);
  ProfRec r{kid, bytes, take_event(pr), nullptr, solve, idx, false};
  cudaEventRecord(r.a, p->st);
  pr->pending.push_back(r);
}

void prof_end(rk_problem* p) {
  Prof* pr = p->prof;
  if (!pr || !pr->on || pr->pending.empty()) return;
  ProfRec& r = pr->pending.back();
  r.b = take_event(pr);
  cudaEventRecord(r.b, p->st);
}

void prof_finish_solve(rk_problem* p, int solve, int iters) {
  Prof* pr = p->prof;
  if (!pr || !pr->on) return;
  for (auto it = pr->pending.rbegin(); it != pr->pending.rend(); ++it) {
    if (it->solve != solve) {
      if (it->solve >= 0 && it->solve < solve) break;
      continue;
    }
    if (it->idx >= iters) it->noop = true;
  }
}

void prof_mark_noops(rk_problem* p, int solve, int idx_from, int idx_to) {
  Prof* pr = p->prof;
  if (!pr || !pr->on || idx_from >= idx_to) return;
  for (auto it = pr->pending.rbegin(); it != pr->pending.rend(); ++it) {
    if (it->solve != solve) {
      if (it->solve >= 0 && it->solve < solve) break;
      continue;
    }
    if (it->idx >= idx_from && it->idx < idx_to) it->noop = true;
  }
}

void prof_free(rk_problem* p) {
  if (!p->prof) return;
  harvest(p);
  for (auto e : p->prof->pool) cudaEventDestroy(e);
  delete p->prof;
  p->prof = nullptr;
}

}  // namespace rk

using namespace rk;

extern "C" {

rk_status rk_profile(rk_problem* p, int enable) {
  if (!p) {
    set_error("problem is NULL");
    return RK_ERR_ARG;
  }
  if (!p->prof) p->prof = new Prof();
  harvest(p);
  Prof* pr = p->prof;
  for (int k = 0; k < K_COUNT; ++k) {
    pr->n[k] = pr->noop[k] = 0;
    pr->ms[k] = pr->bytes[k] = 0.0;
  }
  pr->on = enable != 0;
  p->launches = 0;
  return RK_OK;
}

rk_status rk_profile_read(rk_problem* p, rk_kernel_stat* out, int max, int* count, long long* launches_total) {
  if (!p || (max > 0 && !out)) {
    set_error("rk_profile_read: NULL argument");
    return RK_ERR_ARG;
  }
  if (launches_total) *launches_total = p->launches;
  int c = 0;
  if (p->prof) {
    harvest(p);
    for (int k = 0; k < K_COUNT && c < max; ++k) {
      if (p->prof->n[k] == 0 && p->prof->noop[k] == 0) continue;
      rk_kernel_stat& s = out[c++];
      std::memset(&s, 0, sizeof(s));
      std::snprintf(s.name, sizeof(s.name), "%s", kKernelNames[k]);
      s.launches = p->prof->n[k];
      s.noop_launches = p->prof->noop[k];
      s.ms_total = p->prof->ms[k];
      s.bytes_total = p->prof->bytes[k];
    }
  }
  if (count) *count = c;
  return RK_OK;
}

}  // extern "C"

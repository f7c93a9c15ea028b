// Host-side definitions shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <cstddef>
#include <atomic>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/rk.h"
#include "rk_device.cuh"
#include "rk_heat.cuh"
#include "rk_vec.cuh"
#include "rk_tiled.cuh"
#include "rk_fdm_geo.h"

namespace rk {

void set_error(const char* fmt, ...);

#define RK_CUDA(call)                                                                   \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess) {                                                            \
      ::rk::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                      __LINE__);                                                        \
      return RK_ERR_CUDA;                                                               \
    }                                                                                   \
  } while (0)

#define RK_TRY(expr)            \
  do {                          \
    rk_status s_ = (expr);      \
    if (s_ != RK_OK) return s_; \
  } while (0)

template <typename T> struct Tag { using type = T; };
template <int V> struct IntC { static constexpr int value = V; };

inline size_t dtype_size(int dt) { return dt == RK_F64 ? 8 : dt == RK_F32 ? 4 : 2; }

// dtype of the GMRES basis: the storage type unless a compressed (BF16) basis
// was asked for with FP32 storage.
inline int basis_dtype(const rk_solver_desc& s) {
  return (s.basis == RK_BF16 && s.storage == RK_F32) ? RK_BF16 : s.storage;
}
// bytes per element of the Krylov solution k^eps (FP32 when work vectors are 16-bit)
inline size_t xsize(int dt) { return dt == RK_F64 ? 8 : 4; }

// Line pitch of the heat problems' Krylov vectors and k^eps in the batched
// path: lines padded to a whole number of the thread segments of the problem's
// storage type and block size (seg_of), so every segment of a line is a full,
// 16-byte aligned vector (the single-problem path uses the unpadded n^3 prefix
// of the same buffers).
inline int batch_seg(int storage, int bs) {
  const int v = (storage == RK_F16 || storage == RK_BF16) ? 8 : 4;
  return bs > v ? bs : v;
}
inline int batch_pitch(int n, int storage, int bs) {
  const int s = batch_seg(storage, bs);
  return (n + s - 1) / s * s;
}
inline size_t krylov_elems(int op, int n, int storage, int bs) {
  return op == RK_OP_HEAT7 ? (size_t)n * n * batch_pitch(n, storage, bs) : (size_t)n * n * n;
}

// storage x arithmetic dispatch: (f64,f64), (f32,f32), (f16,f32), (bf16,f32)
template <typename F>
inline void dispatch_st(int storage, F&& f) {
  switch (storage) {
    case RK_F64: f(Tag<double>{}, Tag<double>{}); break;
    case RK_F32: f(Tag<float>{}, Tag<float>{}); break;
    case RK_F16: f(Tag<__half>{}, Tag<float>{}); break;
    default: f(Tag<__nv_bfloat16>{}, Tag<float>{}); break;
  }
}

template <typename F>
inline void dispatch_bs(int bs, F&& f) {
  switch (bs) {
    case 1: f(IntC<1>{}); break;
    case 2: f(IntC<2>{}); break;
    case 4: f(IntC<4>{}); break;
    case 8: f(IntC<8>{}); break;
    case 16: f(IntC<16>{}); break;
    default: f(IntC<32>{}); break;
  }
}

// Type of k^eps: FP64 when the problem refines its stage solves against an
// FP64 true residual (the corrections then accumulate in FP64), else the
// solver's solution type XOf<storage>.  f receives Tag<type>.
template <typename F>
inline void dispatch_ke(bool ke_hi, int storage, F&& f) {
  if (ke_hi) {
    f(Tag<double>{});
    return;
  }
  switch (storage) {
    case RK_F64: f(Tag<double>{}); break;
    default: f(Tag<float>{}); break;  // FP32 storage, and FP32 solutions of 16-bit storage
  }
}

// elements per thread segment for storage S and block size BS
template <typename S, int BS>
constexpr int seg_of() {
  constexpr int v = (sizeof(S) == 2) ? 8 : 4;
  return BS > v ? BS : v;
}

int device_sms();
// cuTensorMapEncodeTiled through the runtime's driver entry point (null if
// the driver does not provide it).
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_fn();
template <typename S>
inline CUtensorMapDataType tma_dtype() {
  if (sizeof(S) == 8) return CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
  if (sizeof(S) == 4) return CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  return std::is_same<S, __half>::value ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
}
int grid_for(const void* kernel, long long work_items, int threads = kThreads);

struct MinvEntry {
  double shift = 0.0;
  void* dev = nullptr;  // heat: 2*BS*BS values of the arithmetic type;
                        // CSR: per-block inverses in the storage type
  std::vector<double> host;  // heat: the same 2*BS*BS values in FP64
  bool valid = false;
};

// Kernel-parameter copy of a heat block-Jacobi inverse.
// LU factors of the constant tridiagonal block tridiag(off, dd, off) of BS
// nodes, formed in FP64 (see BjTri).
template <typename T, int BS>
inline BjTri<T, BS> bj_tri(double dd, double off) {
  BjTri<T, BS> t;
  double piv = dd;
  for (int i = 0; i < BS; ++i) {
    if (i > 0) piv = dd - off * off / piv;
    t.ip[i] = (T)(1.0 / piv);
    t.nu[i] = (T)(-off / piv);
  }
  t.mo = (T)(-off);
  return t;
}

template <typename T, int BS>
inline BjInv<T, BS> bj_param(const std::vector<double>& h) {
  BjInv<T, BS> v;
  for (int i = 0; i < 2 * BS * BS; ++i) v.m[i] = (T)h[i];
  return v;
}

// CSR operator data (advection-diffusion)
struct Csr {
  int* rowptr = nullptr;   // N+1
  int* cols = nullptr;     // nnz
  double* v64 = nullptr;   // nnz FP64 values of L
  void* vS = nullptr;      // nnz values of L * lscale in the storage precision
  double lscale = 1.0;     // storage scale of L (1 / max |L_ij|)
  long long nnz = 0;
};

struct GmresWork;  // defined in rk_csr.cu

// TMA descriptors of the CG work vectors for the tiled sweeps.
struct TiledMaps {
  bool ok = false;       // set up and usable
  bool tried = false;    // eligibility already decided
  TileGeo tg{};
  CUtensorMap r, p[2];   // r and the two p buffers, box (n, ty+2, 1) (sweep B)
  CUtensorMap z;         // z (the fast-diagonalization output), same box
  CUtensorMap ra, pa[2], za;  // the same buffers with box (n, ty+1, 1) (sweep A)
};

// Fast-diagonalization preconditioner state of a heat problem (storage
// float/half/bf16, n <= 256): the sine basis Q and the eigenvalues mu of
// tridiag(-1, 2, -1), one temporary vector, and the 2-D tensor maps of the
// (n^2 x n) views of r, z and the temporary plus the one of Q.
struct FdmState {
  bool ok = false;
  FdmGeo geo{};
  void* q = nullptr;
  float* mu = nullptr;
  void* t = nullptr;
  CUtensorMap in_r, in_z, in_t, qmap;
  int grid = 0;
  size_t smem = 0;
};

// Kernel ids for the launch profiler.
enum Kid {
  K_CG_INIT, K_CG_A, K_CG_B, K_OP, K_CORRECT, K_COMBINE, K_NORMS, K_WIDEN, K_TRUERES, K_ADDSCALED, K_BJ,
  K_CSR_SPMV, K_CSR_CORRECT, K_CSR_BJ_SETUP, K_GM_INIT, K_GM_ARNOLDI, K_GM_ORTH, K_GM_UPDATE,
  K_GM_PREC, K_BATCH, K_FDM, K_FDM_SCALE, K_FDM_DOT, K_CFDM, K_COUNT
};
extern const char* const kKernelNames[K_COUNT];

struct ProfRec {
  int kid;
  double bytes;
  cudaEvent_t a, b;
  int solve, idx;
  bool noop;
};

struct Prof {
  bool on = false;
  std::vector<ProfRec> pending;
  std::vector<cudaEvent_t> pool;
  long long n[K_COUNT]{}, noop[K_COUNT]{};
  double ms[K_COUNT]{}, bytes[K_COUNT]{};
};

}  // namespace rk

struct rk_problem {
  rk_problem_desc desc{};
  rk_solver_desc sol{};
  cudaStream_t st = nullptr;
  int n = 0;
  long long N = 0;
  double h = 0.0, c = 0.0;  // c = kappa/h^2 (heat)
  // tableau
  int q = 0;
  double Ah[64]{}, Al[64]{}, b[8]{};
  // state
  double* u = nullptr;
  double* r = nullptr;
  double* g64 = nullptr;
  double* src = nullptr;  // forcing f of du/dt = L u + f (FP64), nullptr = none
  double* res64 = nullptr;
  double* k[8]{};
  void* ke[8]{};
  bool ke_alias[8]{};
  // Krylov workspace (storage precision)
  void* wr = nullptr;
  void* wz = nullptr;
  void* wp[2]{};
  void* wdelta = nullptr;
  // k^eps held in FP64 (stage solves refined against the FP64 true residual):
  // the solver writes its solution into wx (solution type), which is widened
  // into ke[i]
  bool ke_hi = false;
  void* wx = nullptr;
  // block-Jacobi statistics of the last preconditioner set-up (CSR path)
  long long bj_blocks = 0, bj_half_blocks = 0;
  // reductions / device scalars
  double* partials = nullptr;
  rk::CgScalars* sc = nullptr;
  rk::RhsScalars* rs = nullptr;  // [0..7] per stage, [8] scratch solve, [9] refinement
  rk::CgScalars* h_sc = nullptr; // pinned mirror
  rk::RhsScalars* h_rs = nullptr;
  // preconditioner cache
  rk::MinvEntry minv[8];
  int minv_next = 0;
  int last_iters[10]{};
  unsigned wait_spins = 0;  // bound of the sweeps' main-loop TMA waits (0 = default)
  bool warm_valid[10]{};  // slot holds a solution usable as the next initial guess
  rk_status batch_status = RK_OK;  // this problem's outcome in its last batched call
  // guard bands (RK_GUARD_BYTES > 0 at allocation): per block the cudaMalloc
  // base, the pointer handed out, its size and the guard size on each side
  struct Guard {
    void* base;
    void* user;
    size_t bytes, guard;
  };
  std::vector<Guard> guards;
  bool has_state = false;
  // CSR path
  rk::Csr csr;
  rk::GmresWork* gw = nullptr;
  rk::TiledMaps* tiled = nullptr;
  rk::FdmState* fdm = nullptr;
  size_t bytes = 0;  // device footprint
  // launch accounting / profiler
  long long launches = 0;
  rk::Prof* prof = nullptr;
  int solve_seq = 0;
};

namespace rk {
rk_status alloc_dev(rk_problem* p, void** ptr, size_t bytes);
// Free a block from alloc_dev (its guard bands too, when it has them).
void free_dev(rk_problem* p, void* ptr);

// NVTX range for the lifetime of the object (steps, stage solves, batched
// calls, server ticks): visible to profilers, a few nanoseconds without one.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};
rk_status get_minv(rk_problem* p, double shift, const void** out);
// Heat path: the cache entry (host and device copies) for this shift.
rk_status get_minv_entry(rk_problem* p, double shift, const MinvEntry** out);
// Solve (I - shift L) x = sigma*g with RHS stats in *rs (device).  Result in x
// (storage precision, scaled by sigma).  Returns iterations in *iters.
rk_status krylov_solve(rk_problem* p, double shift, const double* g64, RhsScalars* rs, void* x,
                       int slot, int* iters, int* status);
// FP64 operator: y = L x + f (f: forcing, nullptr = none); if rs != null also
// the RHS statistics.
rk_status op_apply_f64(rk_problem* p, const double* x, double* y, RhsScalars* rs, const double* f = nullptr);
// FP64 correction k = g + shift * L(ke/sigma) and true-residual norm into rs->res2.
rk_status op_correct_f64(rk_problem* p, double shift, const double* g, const void* ke, double* kout,
                         RhsScalars* rs);
rk_status step_impl(rk_problem* p, double dt, rk_stats* acc);
// Launch accounting: count the launch and, when profiling, bracket it with
// CUDA events.  solve/idx tag Krylov sweeps so launches issued after their
// solve converged can be marked as no-ops (prof_finish_solve).
void prof_begin(rk_problem* p, int kid, double bytes, int solve = -1, int idx = -1);
void prof_end(rk_problem* p);
void prof_finish_solve(rk_problem* p, int solve, int iters);
void prof_mark_noops(rk_problem* p, int solve, int idx_from, int idx_to);
void prof_free(rk_problem* p);
template <typename F>
inline void launch(rk_problem* p, int kid, double bytes, F&& f) {
  prof_begin(p, kid, bytes);
  f();
  prof_end(p);
}
// CSR path
// Fast-diagonalization preconditioner (heat, CG): set up once per problem;
// z = P^-1 r on the problem's wr -> wz (6 tensor-core passes).  With cg the
// last pass also forms r.z and updates the CG scalars; solve/idx tag the
// launches for the profiler.
rk_status fdm_setup(rk_problem* p);
rk_status fdm_apply(rk_problem* p, double shift, bool cg, int solve, int idx);
rk_status fdm_precond_f64(rk_problem* p, double shift, const double* r, double* z);
void fdm_free(rk_problem* p);
rk_status csr_setup(rk_problem* p);
rk_status csr_free(rk_problem* p);
rk_status gmres_solve(rk_problem* p, double shift, const double* g64, RhsScalars* rs, void* x, int slot,
                      int* iters, int* status);
rk_status csr_precond_f64(rk_problem* p, double shift, const double* r, double* z);
rk_status csr_apply_f64(rk_problem* p, const double* x, double* y, RhsScalars* rs, const double* f = nullptr);
rk_status csr_correct_f64(rk_problem* p, double shift, const double* g, const void* ke, double* kout,
                          RhsScalars* rs);
}  // namespace rk

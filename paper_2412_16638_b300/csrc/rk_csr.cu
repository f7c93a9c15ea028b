// Advection-diffusion path: CSR assembly, FP64 operator and correction,
// block-Jacobi with per-block inverses, and the GMRES(m) driver.
#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <utility>
#include <vector>

#include "rk_cfdm.cuh"
#include "rk_csr.cuh"
#include "rk_gmres.cuh"
#include "rk_internal.h"

namespace rk {

__global__ void __launch_bounds__(kThreads) csr_apply_f64_kernel(CsrView A, const double* __restrict__ vals,
                                                                 long long N, const double* __restrict__ x,
                                                                 const double* __restrict__ f,
                                                                 double* __restrict__ y, RhsScalars* rs,
                                                                 double* partials) {
  double acc[2] = {0.0, 0.0};
  const bool wmax = rs != nullptr && rs->want_scale;  // the max norm only sets the FP16 scale
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < N;
       r += (long long)gridDim.x * blockDim.x) {
    double s = f ? f[r] : 0.0;
    for (int e = A.rowptr[r]; e < A.rowptr[r + 1]; ++e) s = fma(vals[e], x[A.cols[e]], s);
    y[r] = s;
    acc[0] = fma(s, s, acc[0]);
    if (wmax) acc[1] = fmax(acc[1], fabs(s));
  }
  if (rs == nullptr) return;
  double tot[2];
  if (grid_reduce<2, 2u>(acc, partials, &rs->ticket, tot)) {
    rs->gg = tot[0];
    rs->gmax = tot[1];
    rs->sigma = rhs_scale(rs, tot[0], tot[1], N);
  }
}

struct CsrMinv {
  double shift = 0.0;
  void* dev = nullptr;
  unsigned char* flags = nullptr;  // adaptive precision: 1 = block stored in FP16
  bool valid = false;
  long long half_blocks = 0;       // blocks stored in FP16 (adaptive precision)
};

struct GmresWork {
  void* V = nullptr;          // (m+1) basis vectors of ldv elements (zero padded), basis type
  void* wbuf = nullptr;       // w = (I - shift L) z of the current step, ldv elements, basis type
  void* z = nullptr;          // preconditioned vector
  int* scol = nullptr;        // sliced-ELL copy of L: columns (ldv * kSellW) ...
  void* sval = nullptr;       // ... and values lscale * L in the storage type
  unsigned* smask = nullptr;  // per 32-row slice: slots whose columns follow `pat`
  SellPattern pat{};          // the operator's column offsets by slot
  double scol_bytes = 0.0;    // column bytes the product still loads (irregular slots + masks)
  long long ldv = 0;          // leading dimension: N rounded up to a whole tile
  // complex fast diagonalization (periodic advection): twiddles, two complex
  // work arrays, one real work vector in the storage type
  void* cf_tw = nullptr;
  void* cf_c[2] = {nullptr, nullptr};
  void* cf_tmp = nullptr;
  double* partials = nullptr; // per-CTA multi-dot partials
  GmScalars* sc = nullptr;
  GmScalars* h_sc = nullptr;  // pinned header mirror
  CsrMinv minv[4];
  int minv_next = 0;
  long long npart = 0;
};

static constexpr size_t kGmHeader = offsetof(GmScalars, h1);

// L u = div(kappa grad u) - v.grad u on the n^3 interior nodes (h = 1/(n+1),
// homogeneous Dirichlet): face diffusivity = mean of the two nodes (kappa_P on
// a boundary face), first-order upwind advection.  Columns of a row ascending.
static void assemble(int n, const double* kap, const double vel[3], std::vector<int>& rowptr,
                     std::vector<int>& cols, std::vector<double>& vals) {
  const long long N = (long long)n * n * n;
  const double h = 1.0 / (n + 1), ih2 = 1.0 / (h * h);
  rowptr.assign(N + 1, 0);
  cols.clear();
  vals.clear();
  cols.reserve(N * 7);
  vals.reserve(N * 7);
  const long long stride[3] = {1, n, (long long)n * n};
  for (int k = 0; k < n; ++k)
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < n; ++i) {
        const long long P = i + (long long)j * n + (long long)k * n * n;
        const int idx[3] = {i, j, k};
        double diag = 0.0;
        double nbv[6] = {0, 0, 0, 0, 0, 0};
        bool nbin[6] = {false, false, false, false, false, false};
        for (int d = 0; d < 3; ++d) {
          for (int s = 0; s < 2; ++s) {  // s = 0: minus side, 1: plus side
            const bool inside = s == 0 ? idx[d] > 0 : idx[d] < n - 1;
            const int slot = d * 2 + s;
            if (inside) {
              const long long Q = s == 0 ? P - stride[d] : P + stride[d];
              const double kf = 0.5 * (kap[P] + kap[Q]);
              nbv[slot] += kf * ih2;
              diag -= kf * ih2;
              nbin[slot] = true;
            } else {
              diag -= kap[P] * ih2;
            }
          }
          const double v = vel[d];
          diag -= std::fabs(v) / h;
          const int up = v >= 0.0 ? d * 2 : d * 2 + 1;  // upstream neighbour
          if (nbin[up]) nbv[up] += std::fabs(v) / h;
        }
        // ascending column order: z-, y-, x-, P, x+, y+, z+
        const int order[6] = {4, 2, 0, 1, 3, 5};
        for (int o = 0; o < 3; ++o) {
          const int slot = order[o];
          if (nbin[slot]) {
            cols.push_back((int)(P - stride[slot / 2]));
            vals.push_back(nbv[slot]);
          }
        }
        cols.push_back((int)P);
        vals.push_back(diag);
        for (int o = 3; o < 6; ++o) {
          const int slot = order[o];
          if (nbin[slot]) {
            cols.push_back((int)(P + stride[slot / 2]));
            vals.push_back(nbv[slot]);
          }
        }
        rowptr[P + 1] = (int)cols.size();
      }
}

template <typename S>
__global__ void to_storage(const double* __restrict__ v, double scale, S* __restrict__ out, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = nar<S>(v[i] * scale);
}

static int gm_seg(int storage, int bs) {
  const int v = dtype_size(storage) == 2 ? 8 : 4;
  return bs > v ? bs : v;
}

// L u = -sum_d beta_d (u(x + h e_d) - u(x - h e_d)) / (2h) on the periodic
// grid x_i = i h, h = 1/n (second-order central differences of Sec. 5.2.2,
// the 1-D matrix Tridiag(-1, 0, 1) + K^(B) per direction).  n >= 3, so the two
// neighbours of a node differ; columns of a row ascending, the diagonal (zero)
// is not stored.
static void assemble_periodic(int n, const double beta[3], std::vector<int>& rowptr, std::vector<int>& cols,
                              std::vector<double>& vals) {
  const long long N = (long long)n * n * n;
  const double ih2 = 0.5 * n;  // 1 / (2h)
  rowptr.assign(N + 1, 0);
  cols.clear();
  vals.clear();
  cols.reserve(N * 6);
  vals.reserve(N * 6);
  const long long stride[3] = {1, n, (long long)n * n};
  std::vector<std::pair<long long, double>> row;
  for (int k = 0; k < n; ++k)
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < n; ++i) {
        const long long P = i + (long long)j * n + (long long)k * n * n;
        const int idx[3] = {i, j, k};
        row.clear();
        for (int d = 0; d < 3; ++d) {
          if (beta[d] == 0.0) continue;
          const long long base = P - idx[d] * stride[d];
          const long long plus = base + ((idx[d] + 1) % n) * stride[d];
          const long long minus = base + ((idx[d] + n - 1) % n) * stride[d];
          row.emplace_back(plus, -beta[d] * ih2);
          row.emplace_back(minus, beta[d] * ih2);
        }
        std::sort(row.begin(), row.end());
        for (const auto& e : row) {
          cols.push_back((int)e.first);
          vals.push_back(e.second);
        }
        rowptr[P + 1] = (int)cols.size();
      }
}

rk_status csr_setup(rk_problem* p) {
  std::vector<int> rowptr, cols;
  std::vector<double> vals;
  if (p->desc.op == RK_OP_ADV_PERIODIC)
    assemble_periodic(p->n, p->desc.vel, rowptr, cols, vals);
  else
    assemble(p->n, p->desc.kappa_field, p->desc.vel, rowptr, cols, vals);
  Csr& c = p->csr;
  c.nnz = (long long)vals.size();
  for (size_t r = 0; r + 1 < rowptr.size(); ++r)
    if (rowptr[r + 1] - rowptr[r] > kSellW) {
      set_error("CSR row %zu has %d entries; the sliced-ELL copy holds at most %d", r, rowptr[r + 1] - rowptr[r],
                kSellW);
      return RK_ERR_ARG;
    }
  double vmax = 0.0;
  for (double v : vals) vmax = std::max(vmax, std::fabs(v));
  if (!(vmax > 0.0) || !std::isfinite(vmax)) {
    set_error("CSR operator has no finite nonzero entries (check kappa_field / vel)");
    return RK_ERR_ARG;
  }
  c.lscale = 1.0 / vmax;
  RK_TRY(alloc_dev(p, (void**)&c.rowptr, rowptr.size() * sizeof(int)));
  RK_TRY(alloc_dev(p, (void**)&c.cols, cols.size() * sizeof(int)));
  RK_TRY(alloc_dev(p, (void**)&c.v64, vals.size() * sizeof(double)));
  RK_TRY(alloc_dev(p, &c.vS, vals.size() * dtype_size(p->sol.storage)));
  RK_CUDA(cudaMemcpy(c.rowptr, rowptr.data(), rowptr.size() * sizeof(int), cudaMemcpyHostToDevice));
  RK_CUDA(cudaMemcpy(c.cols, cols.data(), cols.size() * sizeof(int), cudaMemcpyHostToDevice));
  RK_CUDA(cudaMemcpy(c.v64, vals.data(), vals.size() * sizeof(double), cudaMemcpyHostToDevice));
  rk_status st = RK_OK;
  dispatch_st(p->sol.storage, [&](auto ts, auto) {
    using S = typename decltype(ts)::type;
    auto kern = to_storage<S>;
    kern<<<grid_for((const void*)kern, c.nnz), kThreads, 0, p->st>>>(c.v64, c.lscale, static_cast<S*>(c.vS), c.nnz);
    if (cudaGetLastError() != cudaSuccess) st = RK_ERR_CUDA;
  });
  RK_TRY(st);
  if (p->sol.krylov == RK_KRYLOV_GMRES) {
    GmresWork* w = new GmresWork();
    p->gw = w;
    const size_t s = dtype_size(p->sol.storage);
    const int m = p->sol.restart;
    const size_t bsz = dtype_size(basis_dtype(p->sol));
    w->ldv = (p->N + kGmTile - 1) / kGmTile * kGmTile;
    RK_TRY(alloc_dev(p, &w->V, (size_t)(m + 1) * w->ldv * bsz));
    RK_TRY(alloc_dev(p, &w->wbuf, (size_t)w->ldv * bsz));
    RK_CUDA(cudaMemsetAsync(w->V, 0, (size_t)(m + 1) * w->ldv * bsz, p->st));  // padding stays zero
    RK_CUDA(cudaMemsetAsync(w->wbuf, 0, (size_t)w->ldv * bsz, p->st));
    RK_TRY(alloc_dev(p, &w->z, (size_t)p->N * s));
    RK_TRY(alloc_dev(p, (void**)&w->scol, (size_t)w->ldv * kSellW * sizeof(int)));
    RK_TRY(alloc_dev(p, &w->sval, (size_t)w->ldv * kSellW * s));
    const long long nslices = w->ldv / 32;
    RK_TRY(alloc_dev(p, (void**)&w->smask, (size_t)nslices * sizeof(unsigned)));
    {
      // the kSellW most common column offsets, ascending
      std::map<long long, long long> hist;
      for (size_t r = 0; r + 1 < rowptr.size(); ++r)
        for (int e = rowptr[r]; e < rowptr[r + 1]; ++e) ++hist[(long long)cols[e] - (long long)r];
      std::vector<std::pair<long long, long long>> byc(hist.begin(), hist.end());
      std::stable_sort(byc.begin(), byc.end(), [](const auto& a, const auto& b) { return a.second > b.second; });
      std::vector<long long> ds;
      for (size_t i = 0; i < byc.size() && (int)ds.size() < kSellW; ++i) ds.push_back(byc[i].first);
      while ((int)ds.size() < kSellW) ds.push_back(0);
      std::sort(ds.begin(), ds.end());
      for (int k = 0; k < kSellW; ++k) w->pat.d[k] = (int)ds[k];
    }
    dispatch_st(p->sol.storage, [&](auto ts, auto) {
      using S = typename decltype(ts)::type;
      auto kern = sell_from_csr<S>;
      kern<<<grid_for((const void*)kern, w->ldv), kThreads, 0, p->st>>>(
          CsrView{c.rowptr, c.cols}, c.v64, c.lscale, p->N, w->ldv, w->pat, w->scol, static_cast<S*>(w->sval));
      if (cudaGetLastError() != cudaSuccess) st = RK_ERR_CUDA;
    });
    RK_TRY(st);
    {
      auto km = sell_mask;
      km<<<grid_for((const void*)km, nslices), kThreads, 0, p->st>>>(w->scol, nslices, w->pat, w->smask);
      RK_CUDA(cudaGetLastError());
      std::vector<unsigned> hm((size_t)nslices);
      RK_CUDA(cudaMemcpyAsync(hm.data(), w->smask, hm.size() * sizeof(unsigned), cudaMemcpyDeviceToHost, p->st));
      RK_CUDA(cudaStreamSynchronize(p->st));
      long long loaded = 0;  // (slice, slot) pairs whose columns are still loaded
      for (unsigned m : hm) loaded += kSellW - __builtin_popcount(m & ((1u << kSellW) - 1u));
      w->scol_bytes = (double)loaded * 32.0 * sizeof(int) + (double)nslices * sizeof(unsigned);
    }
    const int seg = gm_seg(p->sol.storage, p->sol.bj_block);
    const long long nsegs = (long long)p->n * p->n * ((p->n + seg - 1) / seg);
    const long long ctas = (nsegs + kThreads - 1) / kThreads;
    w->npart = std::max<long long>(ctas * kGmMax, (long long)device_sms() * 8 * kGmDots);
    RK_TRY(alloc_dev(p, (void**)&w->partials, (size_t)w->npart * sizeof(double)));
    RK_TRY(alloc_dev(p, (void**)&w->sc, sizeof(GmScalars)));
    RK_CUDA(cudaMemset(w->sc, 0, sizeof(GmScalars)));
    if (p->sol.precond == RK_PREC_FDM) {
      // twiddles e^{-2 pi i m / n} in the arithmetic type, formed in FP64
      const int n = p->n;
      const size_t cs = (p->sol.storage == RK_F64) ? 16 : 8;  // complex element
      RK_TRY(alloc_dev(p, &w->cf_tw, (size_t)n * cs));
      RK_TRY(alloc_dev(p, &w->cf_c[0], (size_t)p->N * cs));
      RK_TRY(alloc_dev(p, &w->cf_c[1], (size_t)p->N * cs));
      RK_TRY(alloc_dev(p, &w->cf_tmp, (size_t)p->N * s));
      std::vector<double> t64(2 * (size_t)n);
      for (int m = 0; m < n; ++m) {
        const double ang = -2.0 * 3.14159265358979323846 * (double)m / (double)n;
        t64[2 * m] = std::cos(ang);
        t64[2 * m + 1] = std::sin(ang);
      }
      if (cs == 16) {
        RK_CUDA(cudaMemcpy(w->cf_tw, t64.data(), t64.size() * 8, cudaMemcpyHostToDevice));
      } else {
        std::vector<float> t32(t64.begin(), t64.end());
        RK_CUDA(cudaMemcpy(w->cf_tw, t32.data(), t32.size() * 4, cudaMemcpyHostToDevice));
      }
    }
    RK_CUDA(cudaMallocHost((void**)&w->h_sc, sizeof(GmScalars)));
  }
  RK_CUDA(cudaStreamSynchronize(p->st));
  return RK_OK;
}

rk_status csr_free(rk_problem* p) {
  Csr& c = p->csr;
  if (c.rowptr) free_dev(p, c.rowptr);
  if (c.cols) free_dev(p, c.cols);
  if (c.v64) free_dev(p, c.v64);
  if (c.vS) free_dev(p, c.vS);
  c = Csr{};
  if (p->gw) {
    GmresWork* w = p->gw;
    if (w->V) free_dev(p, w->V);
    if (w->wbuf) free_dev(p, w->wbuf);
    if (w->z) free_dev(p, w->z);
    if (w->scol) free_dev(p, w->scol);
    if (w->smask) free_dev(p, w->smask);
    if (w->sval) free_dev(p, w->sval);
    if (w->cf_tw) free_dev(p, w->cf_tw);
    if (w->cf_c[0]) free_dev(p, w->cf_c[0]);
    if (w->cf_c[1]) free_dev(p, w->cf_c[1]);
    if (w->cf_tmp) free_dev(p, w->cf_tmp);
    if (w->partials) free_dev(p, w->partials);
    if (w->sc) free_dev(p, w->sc);
    if (w->h_sc) cudaFreeHost(w->h_sc);
    for (auto& e : w->minv) {
      if (e.dev) free_dev(p, e.dev);
      if (e.flags) free_dev(p, e.flags);
    }
    delete w;
    p->gw = nullptr;
  }
  return RK_OK;
}

static CsrView view(const rk_problem* p) { return CsrView{p->csr.rowptr, p->csr.cols}; }

rk_status csr_apply_f64(rk_problem* p, const double* x, double* y, RhsScalars* rs, const double* f) {
  auto kern = csr_apply_f64_kernel;
  const int grid = grid_for((const void*)kern, p->N);
  const double bytes = (double)p->csr.nnz * 12.0 + 4.0 * (p->N + 1) + (f ? 24.0 : 16.0) * p->N;
  launch(p, K_CSR_SPMV, bytes,
         [&] { kern<<<grid, kThreads, 0, p->st>>>(view(p), p->csr.v64, p->N, x, f, y, rs, p->partials); });
  RK_CUDA(cudaGetLastError());
  return RK_OK;
}

rk_status csr_correct_f64(rk_problem* p, double shift, const double* gv, const void* ke, double* kout,
                          RhsScalars* rs) {
  rk_status st = RK_OK;
  dispatch_ke(p->ke_hi, p->sol.storage, [&](auto tx) {
    using X = typename decltype(tx)::type;
    auto kern = csr_correct_f64_kernel<X>;
    const int grid = grid_for((const void*)kern, p->N);
    const double bytes = (double)p->csr.nnz * 12.0 + 4.0 * (p->N + 1) + (16.0 + sizeof(X)) * p->N;
    launch(p, K_CSR_CORRECT, bytes, [&] {
      kern<<<grid, kThreads, 0, p->st>>>(view(p), p->csr.v64, p->N, gv, static_cast<const X*>(ke), shift, kout, rs,
                                         p->partials);
    });
    if (cudaGetLastError() != cudaSuccess) st = RK_ERR_CUDA;
  });
  if (st != RK_OK) set_error("csr_correct_f64 launch failed");
  return st;
}

// The six passes with the compile-time kernel for n = N1 N2 (rk_cfdm.cuh).
template <typename SI, typename S, typename T, int N1, int N2>
static rk_status cfdm_apply_ct(rk_problem* p, const SI* in, long long in_jstride, S* out, const GmScalars* sc,
                               int solve, int idx, const Cplx<T>* tw, const CfScale& sp) {
  constexpr int n = N1 * N2;
  using C = Cplx<T>;
  GmresWork* w = p->gw;
  const int grid = n * ((n + kCfTile - 1) / kCfTile);
  const size_t smem = (size_t)kCfTile * (n + 1) * sizeof(C) + (size_t)n * sizeof(C);
  auto k_first = cfdm_pass_ct<SI, S, T, true, false, N1, N2>;
  auto k_mid = cfdm_pass_ct<SI, S, T, false, false, N1, N2>;
  auto k_last = cfdm_pass_ct<SI, S, T, false, true, N1, N2>;
  static std::once_flag once;
  static cudaError_t attr = cudaSuccess;
  std::call_once(once, [&] {
    for (const void* k : {(const void*)k_first, (const void*)k_mid, (const void*)k_last})
      if (attr == cudaSuccess) attr = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaGetLastError();
  });
  if (attr != cudaSuccess) {
    set_error("periodic fast diagonalization: shared-memory attribute refused");
    return RK_ERR_CUDA;
  }
  constexpr int threads = 32 * N1;
  const double Nc = (double)p->N * sizeof(C);
  void* c0 = w->cf_c[0];
  void* c1 = w->cf_c[1];
  prof_begin(p, K_CFDM, (double)p->N * sizeof(SI) + Nc, solve, idx);
  k_first<<<grid, threads, smem, p->st>>>(in, c0, tw, 0, 0, sp, sc, in_jstride);
  prof_end(p);
  prof_begin(p, K_CFDM, 2.0 * Nc, solve, idx);
  k_mid<<<grid, threads, smem, p->st>>>(c0, c1, tw, 0, 0, sp, sc, 0);
  prof_end(p);
  prof_begin(p, K_CFDM, 2.0 * Nc, solve, idx);
  k_mid<<<grid, threads, smem, p->st>>>(c1, c0, tw, 0, 1, sp, sc, 0);
  prof_end(p);
  prof_begin(p, K_CFDM, 2.0 * Nc, solve, idx);
  k_mid<<<grid, threads, smem, p->st>>>(c0, c1, tw, 1, 0, sp, sc, 0);
  prof_end(p);
  prof_begin(p, K_CFDM, 2.0 * Nc, solve, idx);
  k_mid<<<grid, threads, smem, p->st>>>(c1, c0, tw, 1, 0, sp, sc, 0);
  prof_end(p);
  prof_begin(p, K_CFDM, Nc + (double)p->N * sizeof(S), solve, idx);
  k_last<<<grid, threads, smem, p->st>>>(c0, out, tw, 1, 0, sp, sc, 0);
  prof_end(p);
  if (cudaGetLastError() != cudaSuccess) {
    set_error("periodic fast-diagonalization launch failed");
    return RK_ERR_CUDA;
  }
  return RK_OK;
}

// z = P^-1 u for the periodic advection stage matrix by the six complex
// passes (rk_cfdm.cuh).  u: basis slot sc->j when sc != null (a GMRES step,
// skipped on the device when none is due), else the vector `in`.
template <typename SI, typename S, typename T>
static rk_status cfdm_apply(rk_problem* p, double shift, const SI* in, long long in_jstride, S* out,
                            const GmScalars* sc, int solve, int idx) {
  GmresWork* w = p->gw;
  const int n = p->n;
  const int nbt = (n + kCfTile - 1) / kCfTile;
  const int grid = n * nbt;
  using C = Cplx<T>;
  static int smem_optin = 0;
  if (smem_optin == 0) {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess || v <= 0) {
      cudaGetLastError();
      set_error("periodic fast diagonalization: shared-memory limit query failed");
      return RK_ERR_CUDA;
    }
    smem_optin = v;
  }
  const int n1 = cfdm_factor(n);
  const size_t smem = cfdm_smem<T>(n);
  if (smem > (size_t)smem_optin) {
    set_error("periodic fast diagonalization: n = %d needs %zu bytes of shared memory (limit %d)", n, smem,
              smem_optin);
    return RK_ERR_ARG;
  }
  const C* tw = static_cast<const C*>(w->cf_tw);
  CfScale sp{};
  sp.s = shift;
  sp.beta[0] = p->desc.vel[0];
  sp.beta[1] = p->desc.vel[1];
  sp.beta[2] = p->desc.vel[2];
  sp.inv_h = (double)n;
  sp.norm = 1.0 / ((double)n * n * n);
  // the grids with a compile-time pass (cfdm_has_ct), for FP32 and FP64
  // throughout; 16-bit storage and compressed bases take the table pass
  if constexpr (std::is_same<SI, S>::value && std::is_same<S, T>::value) {
    switch (n) {
      case 200: return cfdm_apply_ct<SI, S, T, 10, 20>(p, in, in_jstride, out, sc, solve, idx, tw, sp);
      case 64: return cfdm_apply_ct<SI, S, T, 8, 8>(p, in, in_jstride, out, sc, solve, idx, tw, sp);
      case 32: return cfdm_apply_ct<SI, S, T, 4, 8>(p, in, in_jstride, out, sc, solve, idx, tw, sp);
      case 20: return cfdm_apply_ct<SI, S, T, 4, 5>(p, in, in_jstride, out, sc, solve, idx, tw, sp);
      default: break;
    }
  }
  auto k_first = cfdm_pass<SI, S, T, true, false>;
  auto k_mid = cfdm_pass<SI, S, T, false, false>;
  auto k_last = cfdm_pass<SI, S, T, false, true>;
  static bool attr_done[3] = {false, false, false};
  const int slot = sizeof(T) == 8 ? 2 : (sizeof(SI) == 2 ? 1 : 0);
  if (!attr_done[slot]) {
    const int lim = smem_optin;
    if (cudaFuncSetAttribute((const void*)k_first, cudaFuncAttributeMaxDynamicSharedMemorySize, lim) != cudaSuccess ||
        cudaFuncSetAttribute((const void*)k_mid, cudaFuncAttributeMaxDynamicSharedMemorySize, lim) != cudaSuccess ||
        cudaFuncSetAttribute((const void*)k_last, cudaFuncAttributeMaxDynamicSharedMemorySize, lim) != cudaSuccess) {
      cudaGetLastError();
      set_error("periodic fast diagonalization: shared-memory attribute refused");
      return RK_ERR_CUDA;
    }
    attr_done[slot] = true;
  }
  const double Nc = (double)p->N * sizeof(C);
  void* c0 = w->cf_c[0];
  void* c1 = w->cf_c[1];
  prof_begin(p, K_CFDM, (double)p->N * sizeof(SI) + Nc, solve, idx);
  k_first<<<grid, kCfThreads, smem, p->st>>>(in, c0, n, n1, tw, 0, 0, sp, sc, in_jstride);
  prof_end(p);
  prof_begin(p, K_CFDM, 2.0 * Nc, solve, idx);
  k_mid<<<grid, kCfThreads, smem, p->st>>>(c0, c1, n, n1, tw, 0, 0, sp, sc, 0);
  prof_end(p);
  prof_begin(p, K_CFDM, 2.0 * Nc, solve, idx);
  k_mid<<<grid, kCfThreads, smem, p->st>>>(c1, c0, n, n1, tw, 0, 1, sp, sc, 0);
  prof_end(p);
  prof_begin(p, K_CFDM, 2.0 * Nc, solve, idx);
  k_mid<<<grid, kCfThreads, smem, p->st>>>(c0, c1, n, n1, tw, 1, 0, sp, sc, 0);
  prof_end(p);
  prof_begin(p, K_CFDM, 2.0 * Nc, solve, idx);
  k_mid<<<grid, kCfThreads, smem, p->st>>>(c1, c0, n, n1, tw, 1, 0, sp, sc, 0);
  prof_end(p);
  prof_begin(p, K_CFDM, Nc + (double)p->N * sizeof(S), solve, idx);
  k_last<<<grid, kCfThreads, smem, p->st>>>(c0, out, n, n1, tw, 1, 0, sp, sc, 0);
  prof_end(p);
  if (cudaGetLastError() != cudaSuccess) {
    set_error("periodic fast-diagonalization launch failed");
    return RK_ERR_CUDA;
  }
  return RK_OK;
}

// Per-block inverses of I - shift L for this shift (cached, 4 shifts); with
// adaptive precision also the per-block FP16 flags.
static rk_status csr_minv(rk_problem* p, double shift, const void** out, const unsigned char** flags_out = nullptr) {
  if (!p->gw) {
    GmresWork* w = new GmresWork();
    p->gw = w;
  }
  GmresWork* w = p->gw;
  for (auto& e : w->minv)
    if (e.valid && e.shift == shift) {
      *out = e.dev;
      if (flags_out) *flags_out = e.flags;
      return RK_OK;
    }
  CsrMinv& e = w->minv[w->minv_next];
  w->minv_next = (w->minv_next + 1) % 4;
  const int bs = p->sol.bj_block;
  const long long nbl = (p->n + bs - 1) / bs;
  const long long nblocks = (long long)p->n * p->n * nbl;
  const double tau = p->sol.bj_adapt_tau;
  // Thomas factors (3 values per row) without adaptive precision, else the
  // dense inverses (see csr_bj_setup)
  const long long slot = tau > 0.0 ? (long long)bs * bs : 3LL * bs;
  if (!e.dev) RK_TRY(alloc_dev(p, &e.dev, (size_t)(nblocks * slot) * dtype_size(p->sol.storage)));
  if (tau > 0.0 && !e.flags) RK_TRY(alloc_dev(p, (void**)&e.flags, (size_t)nblocks));
  rk_status st = RK_OK;
  dispatch_st(p->sol.storage, [&](auto ts, auto) {
    using S = typename decltype(ts)::type;
    dispatch_bs(bs, [&](auto bsc) {
      constexpr int BS = decltype(bsc)::value;
      auto kern = csr_bj_setup<S, BS>;
      launch(p, K_CSR_BJ_SETUP, (double)p->csr.nnz * 12.0 + (double)(nblocks * slot) * sizeof(S), [&] {
        kern<<<grid_for((const void*)kern, nblocks), kThreads, 0, p->st>>>(view(p), p->csr.v64, p->n, shift,
                                                                          static_cast<S*>(e.dev), tau, e.flags);
      });
      if (cudaGetLastError() != cudaSuccess) st = RK_ERR_CUDA;
    });
  });
  if (st != RK_OK) {
    set_error("csr_bj_setup launch failed");
    return st;
  }
  e.half_blocks = 0;
  if (e.flags) {  // count the FP16 blocks (statistics of the adaptive choice)
    std::vector<unsigned char> f((size_t)nblocks);
    RK_CUDA(cudaMemcpyAsync(f.data(), e.flags, f.size(), cudaMemcpyDeviceToHost, p->st));
    RK_CUDA(cudaStreamSynchronize(p->st));
    for (unsigned char v : f) e.half_blocks += v;
  }
  p->bj_half_blocks = e.half_blocks;
  p->bj_blocks = nblocks;
  e.shift = shift;
  e.valid = true;
  *out = e.dev;
  if (flags_out) *flags_out = e.flags;
  return RK_OK;
}

rk_status csr_precond_f64(rk_problem* p, double shift, const double* r, double* z) {
  if (p->sol.precond == RK_PREC_FDM) {
    if (!p->gw || !p->gw->cf_tw) {
      set_error("periodic fast diagonalization: not set up");
      return RK_ERR_ARG;
    }
    rk_status st = RK_OK;
    dispatch_st(p->sol.storage, [&](auto ts, auto tt) {
      using S = typename decltype(ts)::type;
      using T = typename decltype(tt)::type;
      if constexpr (sizeof(S) >= 4) {
        S* tmp = static_cast<S*>(p->gw->cf_tmp);
        S* zs = static_cast<S*>(p->gw->z);
        auto kin = convert_vec<double, S>;
        auto kout = convert_vec<S, double>;
        kin<<<grid_for((const void*)kin, p->N), kThreads, 0, p->st>>>(r, tmp, p->N);
        st = cfdm_apply<S, S, T>(p, shift, tmp, 0, zs, nullptr, -1, -1);
        if (st == RK_OK) kout<<<grid_for((const void*)kout, p->N), kThreads, 0, p->st>>>(zs, z, p->N);
      } else {
        st = RK_ERR_ARG;
      }
    });
    if (st == RK_OK && cudaGetLastError() != cudaSuccess) st = RK_ERR_CUDA;
    return st;
  }
  const void* minv = nullptr;
  const unsigned char* flags = nullptr;
  RK_TRY(csr_minv(p, shift, &minv, &flags));
  rk_status st = RK_OK;
  dispatch_st(p->sol.storage, [&](auto ts, auto tt) {
    using S = typename decltype(ts)::type;
    using T = typename decltype(tt)::type;
    dispatch_bs(p->sol.bj_block, [&](auto bsc) {
      constexpr int BS = decltype(bsc)::value;
      constexpr int SEG = seg_of<S, BS>();
      HeatGeo g{p->n, (p->n + SEG - 1) / SEG, (long long)p->n * p->n, p->N};
      auto kern = csr_bj_apply_f64io<S, T, BS, SEG>;
      launch(p, K_BJ, (16.0 + (flags ? BS : 3) * sizeof(S)) * p->N, [&] {
        kern<<<grid_for((const void*)kern, g.n2 * g.nseg), kThreads, 0, p->st>>>(g, static_cast<const S*>(minv), flags,
                                                                                r, z);
      });
      if (cudaGetLastError() != cudaSuccess) st = RK_ERR_CUDA;
    });
  });
  if (st != RK_OK) set_error("csr block-Jacobi launch failed");
  return st;
}

// Right-preconditioned restarted GMRES(m) on (I - shift L) x = sigma g, x0 = 0.
// Each Arnoldi step launches three kernels (preconditioner; product on the
// sliced-ELL copy + the step's one reduction + Hessenberg/Givens; basis
// update with the delayed reorthogonalisation, rk_gmres.cuh); they return at
// once when the device state says the cycle or the solve has ended.  The host
// polls the state once per chunk of steps and launches the cycle-end update
// and the restart.
rk_status gmres_solve(rk_problem* p, double shift, const double* g64, RhsScalars* rs, void* x, int slot, int* iters,
                      int* status) {
  if (p->desc.op == RK_OP_HEAT7 || !p->gw || !p->gw->V) {
    set_error("GMRES is implemented for the CSR operators");
    return RK_ERR_ARG;
  }
  GmresWork* w = p->gw;
  const void* minv = nullptr;
  const unsigned char* mflags = nullptr;
  const bool cfdm = p->sol.precond == RK_PREC_FDM;  // periodic complex fast diagonalization
  if (!cfdm) RK_TRY(csr_minv(p, shift, &minv, &mflags));
  const int m = p->sol.restart;
  GmScalars* hs = w->h_sc;
  std::memset(hs, 0, kGmHeader);
  hs->max_iter = p->sol.max_iter;
  hs->m = m;
  hs->tol_rel = p->sol.tol_rel;
  hs->tol_abs = p->sol.tol_abs;
  hs->verify = basis_dtype(p->sol) != p->sol.storage ? 1 : 0;
  RK_CUDA(cudaMemcpyAsync(w->sc, hs, kGmHeader, cudaMemcpyHostToDevice, p->st));
  RK_CUDA(cudaMemsetAsync(&w->sc->ticket2, 0, sizeof(unsigned), p->st));
  const int solve = ++p->solve_seq;
  rk_status st = RK_OK;
  // basis type: the storage type, or BF16 with FP32 storage (compressed basis)
  auto with_basis = [&](auto ts, auto tt, auto fn) {
    using S = typename decltype(ts)::type;
    if constexpr (std::is_same<S, float>::value) {
      if (basis_dtype(p->sol) == RK_BF16) return fn(ts, tt, Tag<__nv_bfloat16>{});
    }
    return fn(ts, tt, ts);
  };
  dispatch_st(p->sol.storage, [&](auto ts0, auto tt0) { with_basis(ts0, tt0, [&](auto ts, auto tt, auto tb) {
    using S = typename decltype(ts)::type;
    using T = typename decltype(tt)::type;
    using B = typename decltype(tb)::type;
    using X = typename XOf<S>::type;
    dispatch_bs(p->sol.bj_block, [&](auto bsc) {
      constexpr int BS = decltype(bsc)::value;
      constexpr int SEG = seg_of<S, BS>();
      HeatGeo g{p->n, (p->n + SEG - 1) / SEG, (long long)p->n * p->n, p->N};
      const long long nsegs = g.n2 * g.nseg;
      B* V = static_cast<B*>(w->V);
      B* wb = static_cast<B*>(w->wbuf);
      S* z = static_cast<S*>(w->z);
      X* xs = static_cast<X*>(x);
      const S* lv = static_cast<const S*>(p->csr.vS);
      const S* M = static_cast<const S*>(minv);
      const T cs = (T)(shift / p->csr.lscale);
      const long long ldv = w->ldv;
      const double Ns = (double)p->N * sizeof(S), Nx = (double)p->N * sizeof(X);
      const double Nb = (double)p->N * sizeof(B);
      const double mat = (double)p->csr.nnz * (4.0 + sizeof(S)) + 4.0 * (p->N + 1);
      // the slot values, plus the columns of the slots off the pattern
      const double sell = (double)p->N * kSellW * sizeof(S) + w->scol_bytes;
      // block inverses read per apply: BS entries per row, FP16 for the
      // adaptively stored blocks, plus one flag byte per block
      const double fhalf = p->bj_blocks > 0 ? (double)p->bj_half_blocks / (double)p->bj_blocks : 0.0;
      // the block-Jacobi data read per application: Thomas factors (3 per
      // row), or dense inverse rows (BS per row, FP16 rows at 2 bytes) and flags
      const double minv_bytes = mflags ? (double)BS * p->N * (sizeof(S) * (1.0 - fhalf) + 2.0 * fhalf) +
                                             (double)p->bj_blocks
                                       : 3.0 * p->N * sizeof(S);
      auto k_start = gm_start<S, B, T, SEG>;
      auto k_restart = gm_restart<S, B, T, SEG>;
      auto k_prec = gm_dc_prec<S, B, T, BS, SEG>;
      auto k_arn = gm_dc_arnoldi<S, B, T>;
      auto k_upd_basis = gm_dc_update<S, B, T>;
      auto k_upd = gm_update<S, B, T, BS, SEG>;
      const int gs = grid_for((const void*)k_start, nsegs), gp = grid_for((const void*)k_prec, nsegs);
      // persistent grids of the two streaming kernels (ring in dynamic shared memory)
      const size_t smem = gm_dc_smem<B>();
      if (cudaFuncSetAttribute((const void*)k_arn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
              cudaSuccess ||
          cudaFuncSetAttribute((const void*)k_upd_basis, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
              cudaSuccess) {
        cudaGetLastError();
        st = RK_ERR_CUDA;
        set_error("GMRES: shared-memory attribute of the Arnoldi kernels refused");
        return;
      }
      int occ_a = 0, occ_u = 0;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_a, k_arn, kGmThreads, smem);
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_u, k_upd_basis, kGmThreads, smem);
      cudaGetLastError();
      const long long ntiles = ldv / kGmTile;
      const int ga = (int)std::max(1LL, std::min<long long>(ntiles, (long long)device_sms() * std::max(1, occ_a)));
      const int gu = (int)std::max(1LL, std::min<long long>(ntiles, (long long)device_sms() * std::max(1, occ_u)));
      if ((long long)ga * kGmDots > w->npart) {
        st = RK_ERR_ARG;
        set_error("GMRES: reduction workspace too small for %d CTAs", ga);
        return;
      }
      launch(p, K_GM_INIT, 8.0 * p->N + Nb + Nx,
             [&] { k_start<<<gs, kThreads, 0, p->st>>>(g, g64, rs, V, xs, w->sc, w->partials); });
      // Arnoldi steps in chunks; each kernel returns at once when the device
      // state says the cycle or the solve has ended.  Step j of a cycle moves
      // j + 1 basis vectors in gm_dc_arnoldi and j + 2 (plus two written) in
      // gm_dc_update; a cycle has m + 1 steps (the last one only finishes
      // column m - 1), so the host's step count modulo m + 1 is j.
      int launched = 0, worked = 0, rounds = 0;
      const int maxlaunch = p->sol.max_iter + 4 * (m + 1) + 64;
      const int maxrounds = 2 * (maxlaunch / 8) + 16;  // every round advances the device state
      while (true) {
        if (++rounds > maxrounds) {
          st = RK_ERR_TIMEOUT;
          set_error("GMRES made no progress after %d polling rounds", rounds);
          return;
        }
        const int chunk = 8;
        for (int c = 0; c < chunk; ++c) {
          const int idx = launched + c;
          const double jb = (double)(idx % (m + 1));
          if (cfdm) {
            if ((st = cfdm_apply<B, S, T>(p, shift, V, ldv, z, w->sc, solve, idx)) != RK_OK) return;
          } else {
            prof_begin(p, K_GM_PREC, Nb + Ns + minv_bytes, solve, idx);
            k_prec<<<gp, kThreads, 0, p->st>>>(g, V, ldv, M, mflags, z, w->sc);
            prof_end(p);
          }
          prof_begin(p, K_GM_ARNOLDI, sell + Ns + Nb + (jb + 1.0) * Nb, solve, idx);
          k_arn<<<ga, kGmThreads, smem, p->st>>>(w->scol, w->smask, w->pat, static_cast<const S*>(w->sval), cs, z, V,
                                                 ldv, wb, p->N, w->sc, w->partials);
          prof_end(p);
          prof_begin(p, K_GM_ORTH, (jb + 2.0) * Nb + 2.0 * Nb, solve, idx);
          k_upd_basis<<<gu, kGmThreads, smem, p->st>>>(V, ldv, wb, p->N, w->sc);
          prof_end(p);
        }
        launched += chunk;
        if (cudaGetLastError() != cudaSuccess) {
          st = RK_ERR_CUDA;
          set_error("GMRES launch failed");
          return;
        }
        if (cudaMemcpyAsync(hs, w->sc, kGmHeader, cudaMemcpyDeviceToHost, p->st) != cudaSuccess ||
            cudaStreamSynchronize(p->st) != cudaSuccess) {
          st = RK_ERR_CUDA;
          set_error("GMRES status readback failed");
          return;
        }
        const int did = hs->steps - worked;
        prof_mark_noops(p, solve, launched - chunk + did, launched);
        worked = hs->steps;
        launched = worked;  // launch indices continue from the device step count
        if (hs->status == 6) {
          st = RK_ERR_TIMEOUT;
          set_error("GMRES: a bounded wait for a streamed basis tile gave up");
          return;
        }
        if (hs->cycle_end) {
          if (cfdm) {
            // x += P^-1 (V y): the combination, the six passes, the sum
            S* tmp = static_cast<S*>(w->cf_tmp);
            auto kc = gm_basis_combine<S, B, T>;
            auto ka = add_into<S, X>;
            launch(p, K_GM_UPDATE, (double)hs->jused * Nb + Ns, [&] {
              kc<<<grid_for((const void*)kc, p->N), kThreads, 0, p->st>>>(V, ldv, p->N, w->sc->y, &w->sc->jused, tmp);
            });
            if ((st = cfdm_apply<S, S, T>(p, shift, tmp, 0, z, nullptr, -1, -1)) != RK_OK) return;
            launch(p, K_GM_UPDATE, Ns + 2.0 * Nx,
                   [&] { ka<<<grid_for((const void*)ka, p->N), kThreads, 0, p->st>>>(xs, z, p->N); });
          } else {
            launch(p, K_GM_UPDATE, (double)hs->jused * Nb + 2.0 * Nx + minv_bytes,
                   [&] { k_upd<<<gp, kThreads, 0, p->st>>>(g, V, ldv, M, mflags, xs, w->sc); });
          }
          if (hs->done) break;
          launch(p, K_GM_INIT, mat + Nx + 8.0 * p->N + Nb, [&] {
            k_restart<<<gs, kThreads, 0, p->st>>>(g, view(p), lv, cs, g64, rs, xs, V, w->sc, w->partials);
          });
        } else if (hs->done) {
          break;
        }
        if (launched > maxlaunch || hs->iter > p->sol.max_iter + 1) {
          st = RK_ERR_TIMEOUT;
          set_error("GMRES did not stop after %d steps", launched);
          return;
        }
      }
      if (cudaStreamSynchronize(p->st) != cudaSuccess) {
        st = RK_ERR_CUDA;
        set_error("GMRES final synchronisation failed");
      }
    });
  }); });
  if (st != RK_OK) return st;
  *iters = hs->iter;
  *status = hs->status;
  p->last_iters[slot] = hs->iter;
  return RK_OK;
}

}  // namespace rk

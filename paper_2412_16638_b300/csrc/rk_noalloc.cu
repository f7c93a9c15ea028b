// rk_heat_solve_noalloc: the heat-operator block-Jacobi CG stage solve for
// callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at all: code running inside a memory
// pool or arena that owns the whole device budget, plug-ins of host programs
// whose allocator policy forbids it, and sections that must not synchronise
// the device (cudaMalloc/cudaFree can).  This entry point runs the same CG
// kernels as rk_solve, but its workspace (Krylov vectors, reduction partials,
// solver scalars) lives in one file-scope device array of fixed size, and the
// block-Jacobi inverse travels as a kernel parameter, so the call allocates
// nothing.
//
// Properties a caller must know:
//  - The array g_noalloc_scratch (RK_NOALLOC_BYTES, about 5.3 MB) bounds the
//    problem size: n <= RK_NOALLOC_MAX_N (64).
//  - The CUDA runtime loads a library's device code and its __device__ arrays
//    onto a device lazily, at their first use there.  So the FIRST call on a
//    device places the array (and the CG kernels' code) in that device's
//    memory; that one call can fail with an out-of-memory error if the device
//    is already full.  Make it before a pool or arena claims the device's
//    memory (or run with CUDA_MODULE_LOADING=EAGER, which loads everything
//    when the context is created).  From then on the array stays on that
//    device until the process exits and later calls allocate nothing.
//  - Every call looks up the array's device address with
//    cudaGetSymbolAddress, with the caller's device current.  The address is
//    not cached: after a cudaDeviceReset the module is loaded again and the
//    array may sit elsewhere.
//  - The call is synchronous (it reads the CG status back to the host between
//    chunks of sweeps): never call it while a stream is being captured.
//  - Every call uses the same array and leaves its contents behind; each call
//    re-initialises everything that must start from a known value.  Calls
//    that overlap on the GPU (different streams, threads or processes sharing
//    the context) race on the array and give wrong results: serialise them.
#include <cmath>

#include "rk_internal.h"

namespace {

constexpr int RK_NOALLOC_MAX_N = 64;
constexpr long long kMaxDof = (long long)RK_NOALLOC_MAX_N * RK_NOALLOC_MAX_N * RK_NOALLOC_MAX_N;
constexpr int kMaxBs = 32;
constexpr int kMaxCtas = 4096;  // grid cap; partials hold 2 doubles per CTA

// byte offsets inside the scratch array (each 256-byte aligned)
constexpr size_t align256(size_t v) { return (v + 255) / 256 * 256; }
constexpr size_t kOffCg = 0;
constexpr size_t kOffRhs = align256(kOffCg + sizeof(rk::CgScalars));
constexpr size_t kOffPart = align256(kOffRhs + sizeof(rk::RhsScalars));
constexpr size_t kOffVec = align256(kOffPart + sizeof(double) * 2 * kMaxCtas);
constexpr size_t kVecBytes = align256(sizeof(float) * kMaxDof);
constexpr size_t RK_NOALLOC_BYTES = kOffVec + 5 * kVecBytes;  // r, z, p0, p1, x

static __device__ __align__(256) unsigned char g_noalloc_scratch[RK_NOALLOC_BYTES];

// Device address of g_noalloc_scratch on the current device.  In host code
// the symbol itself is only a stand-in.  Looked up on every call (a cheap host
// lookup once the module is loaded), never cached: a cudaDeviceReset reloads
// the module and may move the array.
rk_status scratch_address(unsigned char** out) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || !p) {
    cudaGetLastError();
    rk::set_error("rk_heat_solve_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
    return RK_ERR_CUDA;
  }
  *out = static_cast<unsigned char*>(p);
  return RK_OK;
}

// Tridiagonal m x m block (diag dd, off-diagonals off) inverted by Gauss-Jordan
// with partial pivoting in FP64 into the top-left of a zeroed BS x BS array.
// Uses only stack storage.
void block_inverse(int m, double dd, double off, int BS, float* inv) {
  double a[kMaxBs][2 * kMaxBs];
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < 2 * m; ++j) a[i][j] = 0.0;
  for (int i = 0; i < m; ++i) {
    a[i][i] = dd;
    if (i > 0) a[i][i - 1] = off;
    if (i + 1 < m) a[i][i + 1] = off;
    a[i][m + i] = 1.0;
  }
  for (int c = 0; c < m; ++c) {
    int piv = c;
    for (int i = c + 1; i < m; ++i)
      if (std::fabs(a[i][c]) > std::fabs(a[piv][c])) piv = i;
    if (piv != c)
      for (int j = 0; j < 2 * m; ++j) std::swap(a[c][j], a[piv][j]);
    const double d = a[c][c];
    for (int j = 0; j < 2 * m; ++j) a[c][j] /= d;
    for (int i = 0; i < m; ++i) {
      if (i == c || a[i][c] == 0.0) continue;
      const double f = a[i][c];
      for (int j = 0; j < 2 * m; ++j) a[i][j] -= f * a[c][j];
    }
  }
  for (int i = 0; i < BS * BS; ++i) inv[i] = 0.f;
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) inv[i * BS + j] = (float)a[i][m + j];
}

int grid_of(const void* kern, long long work) {
  int occ = 0, dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, rk::kThreads, 0) != cudaSuccess || occ < 1) occ = 1;
  long long need = (work + rk::kThreads - 1) / rk::kThreads;
  long long cap = (long long)(sms > 0 ? sms : 1) * occ;
  long long g = need < cap ? need : cap;
  if (g > kMaxCtas) g = kMaxCtas;
  return (int)(g < 1 ? 1 : g);
}

template <int BS>
rk_status solve_bs(int n, double c, double shift, double tol_rel, double tol_abs, int max_iter, const double* g_dev,
                   double* k_dev, cudaStream_t st, unsigned char* base, int* iters_out) {
  using S = float;
  using T = float;
  constexpr int SEG = rk::seg_of<S, BS>();
  rk::HeatGeo g;
  g.n = n;
  g.nseg = (n + SEG - 1) / SEG;
  g.n2 = (long long)n * n;
  g.N = g.n2 * n;
  const long long work = g.n2 * g.nseg;

  auto* sc = reinterpret_cast<rk::CgScalars*>(base + kOffCg);
  auto* rs = reinterpret_cast<rk::RhsScalars*>(base + kOffRhs);
  auto* partials = reinterpret_cast<double*>(base + kOffPart);
  rk::BjInv<T, BS> minv;  // block-Jacobi inverse, passed by value as a kernel parameter
  S* r = reinterpret_cast<S*>(base + kOffVec);
  S* z = reinterpret_cast<S*>(base + kOffVec + kVecBytes);
  S* p[2] = {reinterpret_cast<S*>(base + kOffVec + 2 * kVecBytes), reinterpret_cast<S*>(base + kOffVec + 3 * kVecBytes)};
  float* x = reinterpret_cast<float*>(base + kOffVec + 4 * kVecBytes);

  // everything that must start from a known value: solver scalars (ticket 0,
  // done 0) and right-hand-side scalars (sigma 1, ticket 0)
  float inv[2 * BS * BS];
  const double dd = 1.0 + 6.0 * shift * c, off = -shift * c;
  block_inverse(BS < n ? BS : n, dd, off, BS, inv);
  for (int i = 0; i < BS * BS; ++i) inv[BS * BS + i] = 0.f;
  if (n % BS) block_inverse(n % BS, dd, off, BS, inv + BS * BS);
  rk::CgScalars sc0{};
  sc0.tol_rel = tol_rel;
  sc0.tol_abs = tol_abs;
  sc0.max_iter = max_iter;
  rk::RhsScalars rs0{};
  rs0.sigma = 1.0;
  RK_CUDA(cudaMemcpyAsync(sc, &sc0, sizeof(sc0), cudaMemcpyHostToDevice, st));
  RK_CUDA(cudaMemcpyAsync(rs, &rs0, sizeof(rs0), cudaMemcpyHostToDevice, st));

  for (int i = 0; i < 2 * BS * BS; ++i) minv.m[i] = inv[i];
  const T d = (T)dd, o = (T)off;
  auto ki = rk::cg_init<S, T, BS, SEG>;
  auto ka = rk::cg_sweep_a<S, T, SEG>;
  auto kb = rk::cg_sweep_b<S, T, BS, SEG>;
  const int gi = grid_of((const void*)ki, work), ga = grid_of((const void*)ka, work), gb = grid_of((const void*)kb, work);
  ki<<<gi, rk::kThreads, 0, st>>>(g, g_dev, rs, minv, r, z, x, sc, partials, 1);
  RK_CUDA(cudaGetLastError());
  rk::CgScalars hs{};
  int launched = 0, cur = 0, chunk = 8;
  while (true) {
    for (int i = 0; i < chunk; ++i) {
      ka<<<ga, rk::kThreads, 0, st>>>(g, d, o, z, p[cur ^ 1], p[cur], sc, partials);
      kb<<<gb, rk::kThreads, 0, st>>>(g, d, o, p[cur], x, r, z, minv, sc, partials);
      cur ^= 1;
    }
    launched += chunk;
    RK_CUDA(cudaGetLastError());
    RK_CUDA(cudaMemcpyAsync(&hs, sc, sizeof(hs), cudaMemcpyDeviceToHost, st));
    RK_CUDA(cudaStreamSynchronize(st));
    if (hs.done) break;
    if (launched > max_iter + 16) {
      rk::set_error("rk_heat_solve_noalloc: CG did not stop after %d sweeps", launched);
      return RK_ERR_TIMEOUT;
    }
    chunk = launched / 2 > 8 ? (launched / 2 < 64 ? launched / 2 : 64) : 8;
    cur = hs.iter & 1;
  }
  auto kw = rk::widen_f64<float>;
  kw<<<grid_of((const void*)kw, g.N), rk::kThreads, 0, st>>>(x, rs, k_dev, g.N);
  RK_CUDA(cudaGetLastError());
  RK_CUDA(cudaStreamSynchronize(st));
  if (iters_out) *iters_out = hs.iter;
  if (hs.status == 5) {
    rk::set_error("rk_heat_solve_noalloc: non-finite value or CG breakdown");
    return RK_ERR_NONFINITE;
  }
  return hs.status == 4 ? RK_ERR_NOT_CONVERGED : RK_OK;
}

}  // namespace

extern "C" rk_status rk_heat_solve_noalloc(int n, double kappa, double shift, int bj_block, double tol_rel,
                                           double tol_abs, int max_iter, const double* g_dev, double* k_dev,
                                           void* cuda_stream, int* iters) {
  if (n < 1 || n > RK_NOALLOC_MAX_N) {
    rk::set_error("rk_heat_solve_noalloc: n = %d is outside 1..%d, the size its fixed %zu-byte device "
                  "workspace holds; use rk_solve for larger grids",
                  n, RK_NOALLOC_MAX_N, (size_t)RK_NOALLOC_BYTES);
    return RK_ERR_ARG;
  }
  if (!(kappa > 0.0) || !std::isfinite(kappa) || !(shift >= 0.0) || !std::isfinite(shift)) {
    rk::set_error("rk_heat_solve_noalloc: kappa must be > 0 and shift >= 0, both finite");
    return RK_ERR_ARG;
  }
  if (!(bj_block == 1 || bj_block == 2 || bj_block == 4 || bj_block == 8 || bj_block == 16 || bj_block == 32)) {
    rk::set_error("rk_heat_solve_noalloc: bj_block must be 1, 2, 4, 8, 16 or 32");
    return RK_ERR_ARG;
  }
  if (!(tol_rel >= 0.0) || !(tol_abs >= 0.0) || max_iter < 1 || max_iter > 1000000) {
    rk::set_error("rk_heat_solve_noalloc: tolerances must be >= 0 and 1 <= max_iter <= 1e6");
    return RK_ERR_ARG;
  }
  if (!g_dev || !k_dev) {
    rk::set_error("rk_heat_solve_noalloc: g and k must be device pointers");
    return RK_ERR_ARG;
  }
  unsigned char* base = nullptr;
  RK_TRY(scratch_address(&base));
  const double h = 1.0 / (n + 1);
  const double c = kappa / (h * h);
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  switch (bj_block) {
    case 1: return solve_bs<1>(n, c, shift, tol_rel, tol_abs, max_iter, g_dev, k_dev, st, base, iters);
    case 2: return solve_bs<2>(n, c, shift, tol_rel, tol_abs, max_iter, g_dev, k_dev, st, base, iters);
    case 4: return solve_bs<4>(n, c, shift, tol_rel, tol_abs, max_iter, g_dev, k_dev, st, base, iters);
    case 8: return solve_bs<8>(n, c, shift, tol_rel, tol_abs, max_iter, g_dev, k_dev, st, base, iters);
    case 16: return solve_bs<16>(n, c, shift, tol_rel, tol_abs, max_iter, g_dev, k_dev, st, base, iters);
    default: return solve_bs<32>(n, c, shift, tol_rel, tol_abs, max_iter, g_dev, k_dev, st, base, iters);
  }
}

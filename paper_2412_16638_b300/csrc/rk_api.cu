// C ABI implementation: problem lifecycle, the DIRK stage loop, the heat CG
// driver and the kernel-level test entry points.
#include <cmath>
#include <cstdarg>
#include <cstdlib>
#include <mutex>
#include <type_traits>
#include <unordered_map>

#include "rk_internal.h"

namespace rk {

static thread_local std::string g_last_error;

void set_error(const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
}

int device_sms() {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 148;
  }
  return sms;
}

// Grid size for a grid-stride kernel: enough CTAs for the work, at most the
// number that can be resident at once (SMs x occupancy).
int grid_for(const void* kernel, long long work_items, int threads) {
  static std::mutex mu;
  static std::unordered_map<const void*, int> occ;
  int o;
  {
    std::lock_guard<std::mutex> lk(mu);
    auto it = occ.find(kernel);
    if (it == occ.end()) {
      int v = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, kernel, threads, 0) != cudaSuccess || v <= 0) v = 1;
      occ[kernel] = v;
      o = v;
    } else {
      o = it->second;
    }
  }
  long long need = (work_items + threads - 1) / threads;
  long long cap = (long long)device_sms() * o;
  long long g = need < cap ? need : cap;
  return (int)(g < 1 ? 1 : g);
}

// Guard bands: with the environment variable RK_GUARD_BYTES = G > 0 when a
// block is allocated, the block gets G bytes (rounded up to 256, so alignment
// is kept) of the pattern kGuardByte on each side; rk_check_guards counts the
// pattern bytes that changed, which catches out-of-bounds writes of the
// kernels near their buffers (the substitute for a memory checker).
static const unsigned char kGuardByte = 0xA5;

static size_t guard_bytes() {
  const char* env = std::getenv("RK_GUARD_BYTES");
  if (!env) return 0;
  char* end = nullptr;
  const long long v = std::strtoll(env, &end, 10);
  if (end == env || v <= 0) return 0;
  const long long capped = v < (1LL << 24) ? v : (1LL << 24);
  return ((size_t)capped + 255) / 256 * 256;
}

rk_status alloc_dev(rk_problem* p, void** ptr, size_t bytes) {
  *ptr = nullptr;
  if (bytes == 0) return RK_OK;
  const size_t g = guard_bytes();
  void* base = nullptr;
  cudaError_t e = cudaMalloc(&base, bytes + 2 * g);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error("cudaMalloc(%zu) failed: %s", bytes + 2 * g, cudaGetErrorString(e));
    return RK_ERR_OOM;
  }
  if (g > 0) {
    unsigned char* b = static_cast<unsigned char*>(base);
    if (cudaMemset(b, kGuardByte, g) != cudaSuccess || cudaMemset(b + g + bytes, kGuardByte, g) != cudaSuccess) {
      cudaGetLastError();
      cudaFree(base);
      set_error("guard band initialisation failed");
      return RK_ERR_CUDA;
    }
    *ptr = b + g;
    p->guards.push_back(rk_problem::Guard{base, *ptr, bytes, g});
  } else {
    *ptr = base;
  }
  p->bytes += bytes;
  return RK_OK;
}

void free_dev(rk_problem* p, void* ptr) {
  if (!ptr) return;
  for (size_t i = 0; i < p->guards.size(); ++i)
    if (p->guards[i].user == ptr) {
      cudaFree(p->guards[i].base);
      p->guards.erase(p->guards.begin() + (long)i);
      return;
    }
  cudaFree(ptr);
}

// Dense inverse of a tridiagonal m x m block (diag dd, off-diagonals off) by
// Gauss-Jordan elimination with partial pivoting in FP64, written into the
// top-left corner of a zeroed BS x BS array.
static void tridiag_block_inverse(int m, double dd, double off, int BS, double* inv) {
  std::vector<double> a((size_t)m * 2 * m, 0.0);
  for (int i = 0; i < m; ++i) {
    a[(size_t)i * 2 * m + i] = dd;
    if (i > 0) a[(size_t)i * 2 * m + i - 1] = off;
    if (i + 1 < m) a[(size_t)i * 2 * m + i + 1] = off;
    a[(size_t)i * 2 * m + m + i] = 1.0;
  }
  for (int c = 0; c < m; ++c) {
    int piv = c;
    for (int i = c + 1; i < m; ++i)
      if (std::fabs(a[(size_t)i * 2 * m + c]) > std::fabs(a[(size_t)piv * 2 * m + c])) piv = i;
    if (piv != c)
      for (int jj = 0; jj < 2 * m; ++jj) std::swap(a[(size_t)c * 2 * m + jj], a[(size_t)piv * 2 * m + jj]);
    const double d = a[(size_t)c * 2 * m + c];
    for (int jj = 0; jj < 2 * m; ++jj) a[(size_t)c * 2 * m + jj] /= d;
    for (int i = 0; i < m; ++i) {
      if (i == c) continue;
      const double f = a[(size_t)i * 2 * m + c];
      if (f == 0.0) continue;
      for (int jj = 0; jj < 2 * m; ++jj) a[(size_t)i * 2 * m + jj] -= f * a[(size_t)c * 2 * m + jj];
    }
  }
  for (int i = 0; i < BS * BS; ++i) inv[i] = 0.0;
  for (int i = 0; i < m; ++i)
    for (int jj = 0; jj < m; ++jj) inv[i * BS + jj] = a[(size_t)i * 2 * m + m + jj];
}

// Block-Jacobi inverses of (I - shift L) for the heat operator: blocks are
// x-line segments of bs nodes, so every full block is the same tridiagonal
// matrix (diag 1 + 6 shift c, off -shift c) and the line's tail block is the
// same matrix of size n mod bs.  Cached per shift value.
static rk_status heat_minv(rk_problem* p, double shift, const void** out) {
  const int bs = p->sol.bj_block;
  for (auto& e : p->minv)
    if (e.valid && e.shift == shift) {
      *out = e.dev;
      return RK_OK;
    }
  MinvEntry& e = p->minv[p->minv_next];
  p->minv_next = (p->minv_next + 1) % 8;
  const size_t tsize = (p->sol.arith == RK_F64) ? 8 : 4;
  if (!e.dev) RK_TRY(alloc_dev(p, &e.dev, 2 * (size_t)bs * bs * tsize));
  std::vector<double> inv(2 * (size_t)bs * bs, 0.0);
  const double dd = 1.0 + 6.0 * shift * p->c, off = -shift * p->c;
  tridiag_block_inverse(std::min(bs, p->n), dd, off, bs, inv.data());
  const int tail = p->n % bs;
  if (tail) tridiag_block_inverse(tail, dd, off, bs, inv.data() + (size_t)bs * bs);
  if (tsize == 8) {
    RK_CUDA(cudaMemcpyAsync(e.dev, inv.data(), inv.size() * 8, cudaMemcpyHostToDevice, p->st));
    RK_CUDA(cudaStreamSynchronize(p->st));  // the host vector goes out of scope
  } else {
    std::vector<float> f(inv.begin(), inv.end());
    RK_CUDA(cudaMemcpyAsync(e.dev, f.data(), f.size() * 4, cudaMemcpyHostToDevice, p->st));
    RK_CUDA(cudaStreamSynchronize(p->st));
  }
  e.host = inv;
  e.shift = shift;
  e.valid = true;
  *out = e.dev;
  return RK_OK;
}

rk_status get_minv_entry(rk_problem* p, double shift, const MinvEntry** out) {
  const void* d = nullptr;
  RK_TRY(heat_minv(p, shift, &d));
  for (auto& e : p->minv)
    if (e.valid && e.dev == d) {
      *out = &e;
      return RK_OK;
    }
  set_error("block-Jacobi cache lookup failed");
  return RK_ERR_ARG;
}

rk_status get_minv(rk_problem* p, double shift, const void** out) {
  if (p->desc.op == RK_OP_HEAT7) return heat_minv(p, shift, out);
  set_error("get_minv: the CSR preconditioner is set up by the GMRES path");
  return RK_ERR_ARG;
}

static HeatGeo heat_geo(const rk_problem* p, int seg) {
  HeatGeo g;
  g.n = p->n;
  g.nseg = (p->n + seg - 1) / seg;
  g.n2 = (long long)p->n * p->n;
  g.N = p->N;
  return g;
}

rk_status op_apply_f64(rk_problem* p, const double* x, double* y, RhsScalars* rs, const double* f) {
  if (p->desc.op != RK_OP_HEAT7) return csr_apply_f64(p, x, y, rs, f);
  constexpr int SEG = 4;
  HeatGeo g = heat_geo(p, SEG);
  auto kern = heat_apply_f64<SEG>;
  int grid = grid_for((const void*)kern, g.n2 * g.nseg);
  launch(p, K_OP, (f ? 24.0 : 16.0) * p->N,
         [&] { kern<<<grid, kThreads, 0, p->st>>>(g, x, f, y, -6.0 * p->c, p->c, rs, p->partials); });
  RK_CUDA(cudaGetLastError());
  return RK_OK;
}

rk_status op_correct_f64(rk_problem* p, double shift, const double* gv, const void* ke, double* kout,
                         RhsScalars* rs) {
  if (p->desc.op != RK_OP_HEAT7) return csr_correct_f64(p, shift, gv, ke, kout, rs);
  constexpr int SEG = 4;
  HeatGeo g = heat_geo(p, SEG);
  rk_status st = RK_OK;
  dispatch_ke(p->ke_hi, p->sol.storage, [&](auto tx) {
    using X = typename decltype(tx)::type;
    auto kern = heat_correct_f64<X, SEG>;
    int grid = grid_for((const void*)kern, g.n2 * g.nseg);
    launch(p, K_CORRECT, (16.0 + sizeof(X)) * p->N, [&] {
      kern<<<grid, kThreads, 0, p->st>>>(g, gv, static_cast<const X*>(ke), shift * p->c, kout, rs, p->partials);
    });
    if (cudaGetLastError() != cudaSuccess) st = RK_ERR_CUDA;
  });
  if (st != RK_OK) set_error("heat_correct_f64 launch failed");
  return st;
}

// ------------------------------------------------------------ tiled sweeps
EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  static std::mutex mu;
  std::lock_guard<std::mutex> lk(mu);
  if (!tried) {
    tried = true;
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(f);
    cudaGetLastError();
  }
  return fn;
}

// Decide once per problem whether the tiled sweeps apply (n <= 256, n a
// multiple of the segment, 16-byte row stride, shared memory fits) and build
// the tensor maps of r, p0, p1.  Returns false to keep the per-segment kernels.
template <typename S, typename T, int BS, int SEG>
static bool tiled_setup(rk_problem* p) {
  if (!p->tiled) p->tiled = new TiledMaps();
  TiledMaps& tm = *p->tiled;
  if (tm.tried) return tm.ok;
  tm.tried = true;
  if (std::getenv("RK_NO_TILED")) return false;
  const int n = p->n;
  if (n > 256 || n % SEG != 0 || ((size_t)n * sizeof(S)) % 16 != 0) return false;
  const int tpl = n / SEG;
  if (tpl > 256) return false;
  int ty = 0;  // sweep A runs tpl*(ty+2) threads (<= 320), sweep B tpl*ty (<= 256)
  for (int c = 1; c <= n; ++c)
    if (n % c == 0 && c * tpl <= 256 && (c + 2) * tpl <= 320 && c + 2 <= 256) ty = c;
  if (ty == 0) return false;
  const size_t sa = tiled_smem_a<S, T, BS>(n, ty), sb = tiled_smem_b<S, T, BS>(n, ty);
  if (sa > 200 * 1024 || sb > 200 * 1024) return false;
  EncodeTiledFn enc = encode_fn();
  if (!enc) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)n, (cuuint64_t)n, (cuuint64_t)n};
  const cuuint64_t strides[2] = {(cuuint64_t)n * sizeof(S), (cuuint64_t)n * n * sizeof(S)};
  const cuuint32_t box_b[3] = {(cuuint32_t)n, (cuuint32_t)(ty + 2), 1};  // sweep B: a halo line on each side
  const cuuint32_t box_a[3] = {(cuuint32_t)n, (cuuint32_t)(ty + 1), 1};  // sweep A: the line above
  const cuuint32_t estr[3] = {1, 1, 1};
  void* bufs[8] = {p->wr, p->wp[0], p->wp[1], p->wz, p->wr, p->wp[0], p->wp[1], p->wz};
  CUtensorMap* maps[8] = {&tm.r, &tm.p[0], &tm.p[1], &tm.z, &tm.ra, &tm.pa[0], &tm.pa[1], &tm.za};
  for (int i = 0; i < 8; ++i) {
    if (enc(maps[i], tma_dtype<S>(), 3, bufs[i], dims, strides, i < 4 ? box_b : box_a, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return false;
  }
  auto ka = cg_tiled_a<S, T, BS, SEG>;
  auto kb = cg_tiled_b<S, T, BS, SEG>;
  // The limit is a property of the kernel, shared by every problem: set it
  // once to the largest size any problem may use (never lower it).
  static std::once_flag once;
  static bool attr_ok = false;
  std::call_once(once, [&] {
    attr_ok = cudaFuncSetAttribute((const void*)ka, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024) ==
                  cudaSuccess &&
              cudaFuncSetAttribute((const void*)kb, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024) ==
                  cudaSuccess;
    cudaGetLastError();
  });
  if (!attr_ok) return false;
  int occa = 0, occb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occa, ka, (ty + 1) * tpl, sa) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occb, kb, ty * tpl, sb) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  // with a single resident CTA per SM the plane pipeline cannot hide its
  // latency (measured: FP64 at 256^3 ran 1.5x slower tiled); keep the
  // per-segment sweeps then
  if (occa < 2 || occb < 2) return false;
  const int nyt = n / ty;
  const int slots = device_sms() * std::min(occa, occb);
  tm.tg = TileGeo{n, tpl, ty, nyt, std::max(1, std::min(n, slots / nyt))};
  tm.ok = true;
  return true;
}

// Chunked device-resident CG: after cg_init, sweeps A and B are launched in
// chunks; each sweep returns at once when the device flag `done` is set, and
// the host reads the flag back once per chunk.  The first chunk is sized by
// the iteration count of the previous solve of the same stage slot.
static rk_status heat_cg_solve(rk_problem* p, double shift, const double* g64, RhsScalars* rs, void* x,
                               int slot, int* iters, int* status) {
  // With the fast-diagonalization preconditioner the sweeps run with the
  // identity block (z = r) and z = P^-1 r is formed after cg_init and after
  // every sweep B by the tensor-core passes, which also update r.z and beta.
  const bool fdm = p->sol.precond == RK_PREC_FDM;
  const MinvEntry* me = nullptr;
  if (fdm)
    RK_TRY(fdm_setup(p));
  else
    RK_TRY(get_minv_entry(p, shift, &me));
  CgScalars init{};
  init.tol_rel = p->sol.tol_rel;
  init.tol_abs = p->sol.tol_abs;
  init.max_iter = p->sol.max_iter;
  init.wait_spins = p->wait_spins;
  *p->h_sc = init;
  RK_CUDA(cudaMemcpyAsync(p->sc, p->h_sc, sizeof(CgScalars), cudaMemcpyHostToDevice, p->st));
  const bool warm = p->sol.warm_start && slot < 8 && p->warm_valid[slot];
  rk_status st = RK_OK;
  dispatch_st(p->sol.storage, [&](auto ts, auto tt) {
    using S = typename decltype(ts)::type;
    using T = typename decltype(tt)::type;
    dispatch_bs(fdm ? 1 : p->sol.bj_block, [&](auto bsc) {
      constexpr int BS = decltype(bsc)::value;
      constexpr int SEG = seg_of<S, BS>();
      HeatGeo g = heat_geo(p, SEG);
      const long long work = g.n2 * g.nseg;
      const T d = (T)(1.0 + 6.0 * shift * p->c), o = (T)(-shift * p->c);
      S* r = static_cast<S*>(p->wr);
      S* z = static_cast<S*>(p->wz);
      using X = typename XOf<S>::type;
      X* xs = static_cast<X*>(x);
      BjInv<T, BS> M;
      BjTri<T, BS> tri;
      if (fdm) {
        for (auto& v : M.m) v = T(0);
        for (int i = 0; i < BS; ++i) M.m[i * BS + i] = M.m[BS * BS + i * BS + i] = T(1);
        for (int i = 0; i < BS; ++i) tri.ip[i] = T(1), tri.nu[i] = T(0);
        tri.mo = T(0);
      } else {
        M = bj_param<T, BS>(me->host);
        tri = bj_tri<T, BS>(1.0 + 6.0 * shift * p->c, -shift * p->c);
      }
      auto ki = cg_init<S, T, BS, SEG>;
      auto ka = cg_sweep_a<S, T, SEG>;
      auto kb = cg_sweep_b<S, T, BS, SEG>;
      const int gi = grid_for((const void*)ki, work), ga = grid_for((const void*)ka, work),
                gb = grid_for((const void*)kb, work);
      const double Ns = (double)p->N * sizeof(S);
      const int solve = ++p->solve_seq;
      const double Nx = (double)p->N * sizeof(X);
      if (warm) {
        auto kw = cg_init_warm<S, T, BS, SEG>;
        launch(p, K_CG_INIT, 8.0 * p->N + 2.0 * Ns + Nx, [&] {
          kw<<<grid_for((const void*)kw, work), kThreads, 0, p->st>>>(g, g64, rs, d, o, M, r, z, xs, p->sc,
                                                                     p->partials);
        });
      }
      const bool tiled = tiled_setup<S, T, BS, SEG>(p);
      if (!warm) {
        // z and x are stored only where the first sweeps read them
        const int store_zx = (tiled || fdm) ? 0 : 1;
        launch(p, K_CG_INIT, 8.0 * p->N + (store_zx ? 2.0 * Ns + Nx : Ns), [&] {
          ki<<<gi, kThreads, 0, p->st>>>(g, g64, rs, M, r, z, xs, p->sc, p->partials, store_zx);
        });
      }
      if (fdm && (st = fdm_apply(p, shift, true, solve, 0)) != RK_OK) return;
      const TileGeo tg = tiled ? p->tiled->tg : TileGeo{};
      const int tgrid = tg.nyt * tg.nzc, tthreads = tg.tpl * tg.ty, athreads = tg.tpl * (tg.ty + 1);
      const size_t sma = tiled ? tiled_smem_a<S, T, BS>(tg.n, tg.ty) : 0;
      const size_t smb = tiled ? tiled_smem_b<S, T, BS>(tg.n, tg.ty) : 0;
      int launched = 0, cur = 0;
      const int predicted = p->last_iters[slot] > 0 ? p->last_iters[slot] : 8;
      int chunk = std::max(2, predicted);
      while (true) {
        for (int c = 0; c < chunk; ++c) {
          S* pn = static_cast<S*>(p->wp[cur]);
          const S* po = static_cast<const S*>(p->wp[cur ^ 1]);
          const int idx = launched + c;
          if (tiled) {
            // 8 vectors per iteration: A reads r, p_old, writes p; B reads p, r, x, writes r, x
            prof_begin(p, K_CG_A, (idx == 0 ? 2.0 : 3.0) * Ns, solve, idx);
            cg_tiled_a<S, T, BS, SEG><<<tgrid, athreads, sma, p->st>>>(fdm ? p->tiled->za : p->tiled->ra,
                                                                       p->tiled->pa[cur ^ 1], tg, d, o, tri, pn,
                                                                       p->sc, p->partials);
            prof_end(p);
            prof_begin(p, K_CG_B, (idx == 0 ? 3.0 * Ns + Nx : 3.0 * Ns + 2.0 * Nx), solve, idx);
            cg_tiled_b<S, T, BS, SEG><<<tgrid, tthreads, smb, p->st>>>(p->tiled->p[cur], tg, d, o, tri, xs, r, p->sc,
                                                                       p->partials);
            prof_end(p);
          } else {
            prof_begin(p, K_CG_A, (idx == 0 ? 2.0 : 3.0) * Ns, solve, idx);
            ka<<<ga, kThreads, 0, p->st>>>(g, d, o, z, po, pn, p->sc, p->partials);
            prof_end(p);
            prof_begin(p, K_CG_B, (idx == 0 ? 4.0 * Ns + Nx : 4.0 * Ns + 2.0 * Nx), solve, idx);
            kb<<<gb, kThreads, 0, p->st>>>(g, d, o, pn, xs, r, z, M, p->sc, p->partials);
            prof_end(p);
          }
          if (fdm && (st = fdm_apply(p, shift, true, solve, idx + 1)) != RK_OK) return;
          cur ^= 1;
        }
        launched += chunk;
        if (cudaGetLastError() != cudaSuccess) {
          st = RK_ERR_CUDA;
          set_error("CG sweep launch failed");
          return;
        }
        if (cudaMemcpyAsync(p->h_sc, p->sc, sizeof(CgScalars), cudaMemcpyDeviceToHost, p->st) != cudaSuccess ||
            cudaStreamSynchronize(p->st) != cudaSuccess) {
          st = RK_ERR_CUDA;
          set_error("CG status readback failed: %s", cudaGetErrorString(cudaGetLastError()));
          return;
        }
        if (p->h_sc->done) {
          prof_finish_solve(p, solve, p->h_sc->iter);
          break;
        }
        if (launched > p->sol.max_iter + 4) {  // the device caps iterations itself
          st = RK_ERR_TIMEOUT;
          set_error("CG did not stop after %d sweeps", launched);
          return;
        }
        // past the prediction: 2 more, then about doubling the overshoot
        chunk = std::max(2, std::min(64, launched - predicted + 1));
        // while the solve runs every launched pair advances the device count
        // by one, so the ping-pong parity equals the device iteration parity
        cur = p->h_sc->iter & 1;
      }
    });
  });
  if (st != RK_OK) return st;
  // a solve that stops before its first sweep (zero or non-finite right-hand
  // side) returns x = 0, which cg_init may have left unwritten
  if (p->h_sc->iter == 0 && !warm) RK_CUDA(cudaMemsetAsync(x, 0, (size_t)p->N * xsize(p->sol.storage), p->st));
  *iters = p->h_sc->iter;
  *status = p->h_sc->status;
  p->last_iters[slot] = p->h_sc->iter;
  if (slot < 8) p->warm_valid[slot] = p->sol.warm_start && (*status == 0 || *status == 4);
  return RK_OK;
}

rk_status krylov_solve(rk_problem* p, double shift, const double* g64, RhsScalars* rs, void* x, int slot,
                       int* iters, int* status) {
  if (p->sol.krylov == RK_KRYLOV_GMRES) return gmres_solve(p, shift, g64, rs, x, slot, iters, status);
  if (p->desc.op != RK_OP_HEAT7) {
    set_error("CG is implemented for the heat operator; use GMRES for advection-diffusion");
    return RK_ERR_ARG;
  }
  return heat_cg_solve(p, shift, g64, rs, x, slot, iters, status);
}

static rk_status launch_combine(rk_problem* p, const CombineArgs& a) {
  rk_status st = RK_OK;
  dispatch_ke(p->ke_hi, p->sol.storage, [&](auto tx) {
    using S = typename decltype(tx)::type;
    auto kern = combine_f64<S>;
    int grid = grid_for((const void*)kern, a.N);
    const double bytes = (double)a.N * ((a.u ? 8.0 : 0.0) + 8.0 * a.nh + (double)sizeof(S) * a.ne + 8.0);
    launch(p, K_COMBINE, bytes, [&] { kern<<<grid, kThreads, 0, p->st>>>(a); });
    if (cudaGetLastError() != cudaSuccess) st = RK_ERR_CUDA;
  });
  if (st != RK_OK) set_error("combine launch failed");
  return st;
}

template <typename F>
static rk_status launch_typed(rk_problem* p, F&& f) {
  rk_status st = RK_OK;
  dispatch_st(p->sol.storage, [&](auto ts, auto) {
    using X = typename XOf<typename decltype(ts)::type>::type;
    f(Tag<X>{});
    if (cudaGetLastError() != cudaSuccess) st = RK_ERR_CUDA;
  });
  if (st != RK_OK) set_error("kernel launch failed");
  return st;
}

// The same with the type of k^eps (FP64 when the problem refines its solves).
template <typename F>
static rk_status launch_ke(rk_problem* p, F&& f) {
  rk_status st = RK_OK;
  dispatch_ke(p->ke_hi, p->sol.storage, [&](auto tx) {
    f(tx);
    if (cudaGetLastError() != cudaSuccess) st = RK_ERR_CUDA;
  });
  if (st != RK_OK) set_error("kernel launch failed");
  return st;
}

// One DIRK step (Sec. 2.2; Eqs. mpAstep1-5 and RKstep): the same loop as the
// float64 oracle, with the implicit solves in the storage/arithmetic
// precision and every explicit evaluation and linear combination in FP64.
rk_status step_impl(rk_problem* p, double dt, rk_stats* acc) {
  NvtxRange range_step("rk_step");
  const int q = p->q;
  const bool mixed = p->sol.correct != 0;
  bool implicit[kMaxStages];
  for (int i = 0; i < q; ++i) implicit[i] = p->Al[i * q + i] != 0.0;
  rk_status worst = RK_OK;
  for (int i = 0; i < q; ++i) {
    // stage right-hand side r_i
    CombineArgs ca{};
    ca.u = p->u;
    ca.out = p->r;
    ca.N = p->N;
    for (int j = 0; j < i; ++j) {
      double chj = dt * p->Ah[i * q + j];
      double cej = dt * p->Al[i * q + j];
      if (cej != 0.0 && (!implicit[j] || !mixed)) {
        chj += cej;  // k^eps_j of an explicit stage (or of the plain form) is k_j
        cej = 0.0;
      }
      if (chj != 0.0) {
        ca.kh[ca.nh] = p->k[j];
        ca.ch[ca.nh++] = chj;
      }
      if (cej != 0.0) {
        ca.ke[ca.ne] = p->ke[j];
        ca.ce[ca.ne] = cej;
        ca.rs[ca.ne++] = p->rs + j;
      }
    }
    const double* rp = p->u;
    if (ca.nh + ca.ne > 0) {
      RK_TRY(launch_combine(p, ca));
      rp = p->r;
    }
    if (!implicit[i]) {
      RK_TRY(op_apply_f64(p, rp, p->k[i], nullptr, p->src));  // k_i = L r_i + f
      continue;
    }
    const double shift = dt * p->Al[i * q + i];
    RhsScalars* rs = p->rs + i;
    RK_TRY(op_apply_f64(p, rp, p->g64, rs, p->src));  // g = L r_i + f (FP64) + norms + scale
    int iters = 0, status = 0;
    // with an FP64 k^eps the solver writes its own solution type into wx
    void* xsol = p->ke_hi ? p->wx : p->ke[i];
    {
      NvtxRange range_solve("stage solve");
      RK_TRY(krylov_solve(p, shift, p->g64, rs, xsol, i, &iters, &status));
    }
    if (acc) {
      acc->iters_total += iters;
      acc->iters_max = std::max(acc->iters_max, iters);
      acc->solves += 1;
      if (status == 4) acc->not_converged += 1;
    }
    if (status == 5) {
      set_error("stage %d solve: non-finite value or Krylov breakdown", i);
      return RK_ERR_NONFINITE;
    }
    if (status == 6) {
      set_error("stage %d solve: a bounded device wait for a TMA tile gave up", i);
      return RK_ERR_TIMEOUT;
    }
    if (status == 4) worst = RK_ERR_NOT_CONVERGED;
    if (mixed) {
      if (p->ke_hi) {
        RK_TRY(launch_typed(p, [&](auto ts) {
          using X = typename decltype(ts)::type;
          auto kern = widen_keep_f64<X>;
          launch(p, K_WIDEN, (8.0 + sizeof(X)) * p->N, [&] {
            kern<<<grid_for((const void*)kern, p->N), kThreads, 0, p->st>>>(static_cast<const X*>(p->wx),
                                                                             static_cast<double*>(p->ke[i]), p->N);
          });
        }));
      }
      // k_i = L y_i, y_i = r_i + shift k^eps_i, in FP64; true residual
      RK_TRY(op_correct_f64(p, shift, p->g64, p->ke[i], p->k[i], rs));
      // Refinement against the FP64 true residual res = k_i - k^eps_i of the
      // stage system: solve (I - shift L) delta = res in the solver's
      // precision and add delta to k^eps in FP64, until the relative true
      // residual is at most tol_true; still above it after max_refine
      // refinements: not converged (the state stays valid).
      for (int it = 0; p->sol.tol_true > 0.0; ++it) {
        RK_CUDA(cudaMemcpyAsync(p->h_rs + i, rs, sizeof(RhsScalars), cudaMemcpyDeviceToHost, p->st));
        RK_CUDA(cudaStreamSynchronize(p->st));
        const double rel = std::sqrt(p->h_rs[i].res2 / std::max(p->h_rs[i].gg, 1e-300));
        if (!(rel > p->sol.tol_true)) break;
        if (it >= p->sol.max_refine) {
          set_error("stage %d: FP64 true residual %.3e above tol_true %.3e after %d refinements", i, rel,
                    p->sol.tol_true, it);
          if (acc) acc->not_converged += 1;
          worst = RK_ERR_NOT_CONVERGED;
          break;
        }
        if (!p->res64) RK_TRY(alloc_dev(p, (void**)&p->res64, (size_t)p->N * 8));
        if (!p->wdelta) RK_TRY(alloc_dev(p, &p->wdelta, (size_t)p->N * xsize(p->sol.storage)));
        RhsScalars* rsd = p->rs + 9;
        RK_TRY(launch_ke(p, [&](auto tk) {
          using K = typename decltype(tk)::type;
          auto kern = true_residual_f64<K>;
          launch(p, K_TRUERES, (16.0 + sizeof(K)) * p->N, [&] {
            kern<<<grid_for((const void*)kern, p->N), kThreads, 0, p->st>>>(
                p->k[i], static_cast<const K*>(p->ke[i]), rs, p->res64, p->N);
          });
        }));
        {
          auto kern = vec_norms_f64;
          launch(p, K_NORMS, 8.0 * p->N, [&] {
            kern<<<grid_for((const void*)kern, p->N), kThreads, 0, p->st>>>(p->res64, p->N, rsd, p->partials);
          });
          RK_CUDA(cudaGetLastError());
        }
        int it2 = 0, st2 = 0;
        NvtxRange range_refine("refinement solve");
        RK_TRY(krylov_solve(p, shift, p->res64, rsd, p->wdelta, 8, &it2, &st2));
        if (st2 == 5 || st2 == 6) {
          set_error("stage %d refinement solve failed (status %d)", i, st2);
          return st2 == 5 ? RK_ERR_NONFINITE : RK_ERR_TIMEOUT;
        }
        if (acc) {
          acc->iters_total += it2;
          acc->refinements += 1;
        }
        rk_status ast = RK_OK;
        dispatch_ke(p->ke_hi, p->sol.storage, [&](auto tk) {
          using K = typename decltype(tk)::type;
          ast = launch_typed(p, [&](auto ts) {
            using D = typename decltype(ts)::type;
            auto kern = add_scaled_inplace<K, D>;
            launch(p, K_ADDSCALED, (2.0 * sizeof(K) + sizeof(D)) * p->N, [&] {
              kern<<<grid_for((const void*)kern, p->N), kThreads, 0, p->st>>>(
                  static_cast<K*>(p->ke[i]), static_cast<const D*>(p->wdelta), rs, rsd, p->N);
            });
          });
        });
        RK_TRY(ast);
        RK_TRY(op_correct_f64(p, shift, p->g64, p->ke[i], p->k[i], rs));
      }
    } else if (!p->ke_alias[i]) {
      RK_TRY(launch_typed(p, [&](auto ts) {
        using S = typename decltype(ts)::type;
        auto kern = widen_f64<S>;
        launch(p, K_WIDEN, (8.0 + sizeof(S)) * p->N, [&] {
          kern<<<grid_for((const void*)kern, p->N), kThreads, 0, p->st>>>(static_cast<const S*>(p->ke[i]), rs,
                                                                           p->k[i], p->N);
        });
      }));
    }
  }
  // u_{n+1} = u_n + dt sum_j b_j k_j
  CombineArgs ca{};
  ca.u = p->u;
  ca.out = p->u;
  ca.N = p->N;
  for (int j = 0; j < q; ++j)
    if (p->b[j] != 0.0) {
      ca.kh[ca.nh] = p->k[j];
      ca.ch[ca.nh++] = dt * p->b[j];
    }
  RK_TRY(launch_combine(p, ca));
  if (mixed && acc) {
    RK_CUDA(cudaMemcpyAsync(p->h_rs, p->rs, sizeof(RhsScalars) * q, cudaMemcpyDeviceToHost, p->st));
    RK_CUDA(cudaStreamSynchronize(p->st));
    for (int i = 0; i < q; ++i)
      if (implicit[i]) {
        const double rel = std::sqrt(p->h_rs[i].res2 / std::max(p->h_rs[i].gg, 1e-300));
        acc->true_res = std::max(acc->true_res, rel);
      }
  }
  return worst;
}

}  // namespace rk

using namespace rk;

// ------------------------------------------------------------------ helpers
static rk_status check_solver(const rk_solver_desc* s, const rk_problem_desc* d) {
  if (!s) {
    set_error("solver descriptor is NULL");
    return RK_ERR_ARG;
  }
  if (s->krylov != RK_KRYLOV_CG && s->krylov != RK_KRYLOV_GMRES) {
    set_error("unknown krylov %d", s->krylov);
    return RK_ERR_ARG;
  }
  const int bs = s->bj_block;
  if (!(bs == 1 || bs == 2 || bs == 4 || bs == 8 || bs == 16 || bs == 32)) {
    set_error("bj_block must be 1, 2, 4, 8, 16 or 32 (got %d)", bs);
    return RK_ERR_ARG;
  }
  if (s->storage < RK_F64 || s->storage > RK_BF16) {
    set_error("unknown storage dtype %d", s->storage);
    return RK_ERR_ARG;
  }
  if (!((s->arith == RK_F64 && s->storage == RK_F64) || (s->arith == RK_F32 && s->storage != RK_F64))) {
    set_error("supported precision pairs: storage F64 / arith F64, storage F32|F16|BF16 / arith F32");
    return RK_ERR_ARG;
  }
  if (!(s->tol_rel >= 0.0) || !(s->tol_abs >= 0.0) || s->max_iter < 1 || s->max_iter > 1000000) {
    set_error("tolerances must be >= 0 and 1 <= max_iter <= 1e6");
    return RK_ERR_ARG;
  }
  if (s->krylov == RK_KRYLOV_GMRES && (s->restart < 1 || s->restart > 64)) {
    set_error("GMRES restart must be in 1..64");
    return RK_ERR_ARG;
  }
  if (s->krylov == RK_KRYLOV_CG && d && d->op != RK_OP_HEAT7) {
    set_error("CG needs the symmetric heat operator");
    return RK_ERR_ARG;
  }
  if (s->krylov == RK_KRYLOV_GMRES && d && d->op == RK_OP_HEAT7) {
    set_error("GMRES is implemented for the CSR operators (advection-diffusion, periodic advection)");
    return RK_ERR_ARG;
  }
  if (s->max_refine < 0 || s->max_refine > 10) {
    set_error("max_refine must be in 0..10");
    return RK_ERR_ARG;
  }
  if (!(s->basis == 0 || s->basis == s->storage || (s->basis == RK_BF16 && s->storage == RK_F32))) {
    set_error("GMRES basis: 0 or the storage dtype, or RK_BF16 with RK_F32 storage (got %d)", s->basis);
    return RK_ERR_ARG;
  }
  if (s->basis == RK_BF16 && s->storage == RK_F32 && s->krylov != RK_KRYLOV_GMRES) {
    set_error("a compressed basis applies to GMRES only");
    return RK_ERR_ARG;
  }
  if (s->warm_start != 0 && s->warm_start != 1) {
    set_error("warm_start must be 0 or 1");
    return RK_ERR_ARG;
  }
  if (s->warm_start && s->correct && s->storage != RK_F64 && s->max_refine > 0 && s->tol_true > 0.0) {
    set_error("warm_start is not combined with refinement (max_refine > 0, tol_true > 0)");
    return RK_ERR_ARG;
  }
  if (s->warm_start && (s->krylov != RK_KRYLOV_CG || s->storage == RK_F16)) {
    set_error("warm_start is implemented for CG with FP64, FP32 or BF16 storage");
    return RK_ERR_ARG;
  }
  if (!(s->bj_adapt_tau >= 0.0) || !std::isfinite(s->bj_adapt_tau)) {
    set_error("bj_adapt_tau must be finite and >= 0");
    return RK_ERR_ARG;
  }
  if (s->bj_adapt_tau > 0.0 &&
      (s->storage != RK_F32 || s->precond != RK_PREC_BLOCK_JACOBI || (d && d->op == RK_OP_HEAT7))) {
    set_error("adaptive-precision block-Jacobi (bj_adapt_tau > 0) is built for the CSR operators with FP32 storage");
    return RK_ERR_ARG;
  }
  if (s->precond != RK_PREC_BLOCK_JACOBI && s->precond != RK_PREC_FDM) {
    set_error("unknown preconditioner %d", s->precond);
    return RK_ERR_ARG;
  }
  if (s->precond == RK_PREC_FDM && d && d->op == RK_OP_ADV_PERIODIC) {
    // complex fast diagonalization of the periodic advection stage matrix
    if (s->krylov != RK_KRYLOV_GMRES || (s->storage != RK_F32 && s->storage != RK_F64)) {
      set_error("the periodic fast-diagonalization preconditioner runs with GMRES and FP32 or FP64 storage");
      return RK_ERR_ARG;
    }
    if (d->n > 400) {
      set_error("the periodic fast-diagonalization preconditioner needs n <= 400 (n = %d)", d->n);
      return RK_ERR_ARG;
    }
    return RK_OK;
  }
  if (s->precond == RK_PREC_FDM) {
    if (s->krylov != RK_KRYLOV_CG || (d && d->op != RK_OP_HEAT7)) {
      set_error("the fast-diagonalization preconditioner is built for CG on the heat operator and GMRES on the "
                "periodic advection operator");
      return RK_ERR_ARG;
    }
    if (s->storage == RK_F64) {
      set_error("the fast-diagonalization preconditioner runs on the tensor cores: FP32, FP16 or BF16 storage");
      return RK_ERR_ARG;
    }
    const size_t es = s->storage == RK_F32 ? 4 : 2;
    if (d && (d->n > 256 || ((size_t)d->n * es) % 16 != 0)) {
      set_error("the fast-diagonalization preconditioner needs n <= 256 and 16-byte rows (n = %d)", d->n);
      return RK_ERR_ARG;
    }
  }
  return RK_OK;
}

static void free_problem(rk_problem* p) {
  if (!p) return;
  auto f = [p](void* ptr) { free_dev(p, ptr); };
  f(p->u);
  f(p->r);
  f(p->g64);
  f(p->src);
  f(p->res64);
  for (int i = 0; i < 8; ++i) {
    f(p->k[i]);
    if (!p->ke_alias[i]) f(p->ke[i]);
  }
  f(p->wr);
  f(p->wz);
  f(p->wp[0]);
  f(p->wp[1]);
  f(p->wdelta);
  f(p->wx);
  f(p->partials);
  f(p->sc);
  f(p->rs);
  for (auto& e : p->minv) f(e.dev);
  if (p->h_sc) cudaFreeHost(p->h_sc);
  if (p->h_rs) cudaFreeHost(p->h_rs);
  csr_free(p);
  fdm_free(p);
  prof_free(p);
  delete p->tiled;
  delete p;
}

extern "C" {

const char* rk_last_error(void) { return g_last_error.c_str(); }

const char* rk_version(void) { return "rk-b300 0.1 (sm_103a)"; }

rk_status rk_create_problem(const rk_problem_desc* desc, const rk_solver_desc* solver, void* cuda_stream,
                            rk_problem** out) {
  if (!out) {
    set_error("out is NULL");
    return RK_ERR_ARG;
  }
  *out = nullptr;
  if (!desc) {
    set_error("problem descriptor is NULL");
    return RK_ERR_ARG;
  }
  if (desc->op != RK_OP_HEAT7 && desc->op != RK_OP_ADVDIFF_CSR && desc->op != RK_OP_ADV_PERIODIC) {
    set_error("unknown operator %d", desc->op);
    return RK_ERR_ARG;
  }
  if (desc->n < 1 || desc->n > 1024) {
    set_error("n must be in 1..1024 (got %d)", desc->n);
    return RK_ERR_ARG;
  }
  if (desc->op == RK_OP_HEAT7 && !(desc->kappa > 0.0 && std::isfinite(desc->kappa))) {
    set_error("kappa must be positive and finite");
    return RK_ERR_ARG;
  }
  if (desc->op == RK_OP_ADVDIFF_CSR) {
    if (!desc->kappa_field) {
      set_error("RK_OP_ADVDIFF_CSR needs kappa_field");
      return RK_ERR_ARG;
    }
    if ((long long)desc->n * desc->n * desc->n * 7 > 2000000000LL) {
      set_error("CSR with int32 indices supports n^3*7 < 2e9");
      return RK_ERR_ARG;
    }
  }
  if (desc->op == RK_OP_ADV_PERIODIC) {
    if (desc->n < 3) {
      set_error("RK_OP_ADV_PERIODIC needs n >= 3 (distinct neighbours on the periodic grid)");
      return RK_ERR_ARG;
    }
    if ((long long)desc->n * desc->n * desc->n * 6 > 2000000000LL) {
      set_error("CSR with int32 indices supports n^3*6 < 2e9");
      return RK_ERR_ARG;
    }
    for (int d = 0; d < 3; ++d)
      if (!std::isfinite(desc->vel[d])) {
        set_error("vel must be finite");
        return RK_ERR_ARG;
      }
  }
  RK_TRY(check_solver(solver, desc));
  rk_problem* p = new rk_problem();
  p->desc = *desc;
  p->desc.kappa_field = nullptr;
  p->desc.source = nullptr;
  p->sol = *solver;
  p->st = static_cast<cudaStream_t>(cuda_stream);
  p->n = desc->n;
  p->N = (long long)desc->n * desc->n * desc->n;
  p->h = desc->op == RK_OP_ADV_PERIODIC ? 1.0 / desc->n : 1.0 / (desc->n + 1);
  p->c = desc->kappa / (p->h * p->h);
  // refined stage solves keep k^eps in FP64 (the FP32 rounding of k^eps would
  // otherwise bound the refinement)
  p->ke_hi = solver->correct && solver->storage != RK_F64 && solver->max_refine > 0 && solver->tol_true > 0.0;
  const size_t N = (size_t)p->N, s = dtype_size(solver->storage);
  rk_status st = RK_OK;
  auto A = [&](void** ptr, size_t bytes) {
    if (st == RK_OK) st = alloc_dev(p, ptr, bytes);
  };
  A((void**)&p->u, N * 8);
  A((void**)&p->r, N * 8);
  A((void**)&p->g64, N * 8);
  // padded lines for the batched path (heat)
  const size_t NK = krylov_elems(desc->op, desc->n, solver->storage, solver->bj_block);
  A(&p->wr, NK * s);
  A(&p->wz, NK * s);
  A(&p->wp[0], NK * s);
  A(&p->wp[1], NK * s);
  A((void**)&p->partials, (size_t)device_sms() * 32 * 4 * 8);
  A((void**)&p->sc, sizeof(CgScalars));
  A((void**)&p->rs, 10 * sizeof(RhsScalars));
  if (st == RK_OK && cudaMallocHost((void**)&p->h_sc, sizeof(CgScalars)) != cudaSuccess) st = RK_ERR_OOM;
  if (st == RK_OK && cudaMallocHost((void**)&p->h_rs, 10 * sizeof(RhsScalars)) != cudaSuccess) st = RK_ERR_OOM;
  if (st == RK_OK) {
    std::vector<RhsScalars> z(10);
    for (auto& r : z) {
      r = RhsScalars{};
      r.sigma = 1.0;
      r.want_scale = (solver->storage == RK_F16);
      // (not with warm starts: the previous solution is kept at scale 1)
      r.want_range = (solver->storage == RK_F32 || solver->storage == RK_BF16) && !solver->warm_start;
    }
    if (cudaMemcpy(p->rs, z.data(), sizeof(RhsScalars) * 10, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(p->sc, 0, sizeof(CgScalars)) != cudaSuccess || cudaMemset(p->u, 0, N * 8) != cudaSuccess) {
      set_error("initial device copies failed");
      st = RK_ERR_CUDA;
    }
  }
  if (st == RK_OK && desc->op != RK_OP_HEAT7) {
    // csr_setup reads the kappa field from the caller's descriptor
    p->desc.kappa_field = desc->kappa_field;
    st = csr_setup(p);
    p->desc.kappa_field = nullptr;
  }
  if (st == RK_OK && desc->source) {
    A((void**)&p->src, N * 8);
    if (st == RK_OK && cudaMemcpy(p->src, desc->source, N * 8, cudaMemcpyHostToDevice) != cudaSuccess) {
      set_error("copy of the forcing term failed");
      st = RK_ERR_CUDA;
    }
  }
  if (st != RK_OK) {
    free_problem(p);
    return st;
  }
  *out = p;
  return RK_OK;
}

rk_status rk_get_problem_info(const rk_problem* p, rk_problem_info* info) {
  if (!p || !info) {
    set_error("rk_get_problem_info: NULL argument");
    return RK_ERR_ARG;
  }
  info->device_bytes = p->bytes;
  info->launches = p->launches;
  info->bj_blocks = p->bj_blocks;
  info->bj_half_blocks = p->bj_half_blocks;
  info->batch_status = p->batch_status;
  return RK_OK;
}

rk_status rk_check_guards(rk_problem* p, long long* corrupted_bytes, int* guarded_blocks) {
  if (!p || !corrupted_bytes) {
    set_error("rk_check_guards: NULL argument");
    return RK_ERR_ARG;
  }
  RK_CUDA(cudaStreamSynchronize(p->st));
  long long bad = 0;
  std::vector<unsigned char> h;
  for (const auto& gd : p->guards) {
    h.resize(gd.guard);
    const unsigned char* b = static_cast<const unsigned char*>(gd.base);
    for (const unsigned char* src : {b, b + gd.guard + gd.bytes}) {
      RK_CUDA(cudaMemcpy(h.data(), src, gd.guard, cudaMemcpyDeviceToHost));
      for (unsigned char c : h) bad += (c != kGuardByte);
    }
  }
  *corrupted_bytes = bad;
  if (guarded_blocks) *guarded_blocks = (int)p->guards.size();
  return RK_OK;
}

rk_status rk_guard_poke(rk_problem* p, int block, long long offset) {
  if (!p || block < 0 || block >= (int)p->guards.size() || offset < 0 ||
      offset >= (long long)p->guards[block].guard) {
    set_error("rk_guard_poke: no guarded block %d with a byte %lld", block, offset);
    return RK_ERR_ARG;
  }
  RK_CUDA(cudaStreamSynchronize(p->st));
  RK_CUDA(cudaMemset(static_cast<unsigned char*>(p->guards[block].base) + offset, (unsigned char)~kGuardByte, 1));
  return RK_OK;
}

rk_status rk_set_wait_limit(rk_problem* p, unsigned long long spins) {
  if (!p) {
    set_error("problem is NULL");
    return RK_ERR_ARG;
  }
  if (spins > 0xffffffffull) {
    set_error("rk_set_wait_limit: at most 2^32 - 1 polls");
    return RK_ERR_ARG;
  }
  p->wait_spins = (unsigned)spins;
  return RK_OK;
}

rk_status rk_destroy_problem(rk_problem* p) {
  if (!p) {
    set_error("problem is NULL");
    return RK_ERR_ARG;
  }
  if (p->st)
    cudaStreamSynchronize(p->st);
  else
    cudaDeviceSynchronize();
  free_problem(p);
  return RK_OK;
}

rk_status rk_set_tableau(rk_problem* p, int q, const double* A_hi, const double* A_lo, const double* b) {
  if (!p || !A_hi || !A_lo || !b) {
    set_error("rk_set_tableau: NULL argument");
    return RK_ERR_ARG;
  }
  if (q < 1 || q > kMaxStages) {
    set_error("q must be in 1..%d", kMaxStages);
    return RK_ERR_ARG;
  }
  for (int i = 0; i < q; ++i) {
    if (!std::isfinite(b[i])) {
      set_error("b must be finite");
      return RK_ERR_ARG;
    }
    for (int j = 0; j < q; ++j) {
      if (!std::isfinite(A_hi[i * q + j]) || !std::isfinite(A_lo[i * q + j])) {
        set_error("tableau entries must be finite");
        return RK_ERR_ARG;
      }
      if (j >= i && A_hi[i * q + j] != 0.0) {
        set_error("A_hi must be strictly lower triangular (entry %d,%d)", i, j);
        return RK_ERR_ARG;
      }
      if (j > i && A_lo[i * q + j] != 0.0) {
        set_error("A_lo must be lower triangular (entry %d,%d)", i, j);
        return RK_ERR_ARG;
      }
    }
    if (A_lo[i * q + i] < 0.0) {
      set_error("implicit diagonal entries must be >= 0");
      return RK_ERR_ARG;
    }
  }
  const size_t N = (size_t)p->N, s = dtype_size(p->sol.storage);
  for (int i = 0; i < q; ++i) {
    if (!p->k[i]) RK_TRY(alloc_dev(p, (void**)&p->k[i], N * 8));
    const bool implicit = A_lo[i * q + i] != 0.0;
    const bool alias = (p->sol.storage == RK_F64 && !p->sol.correct);
    if (implicit && !p->ke[i]) {
      if (alias) {
        p->ke[i] = p->k[i];
        p->ke_alias[i] = true;
      } else {
        RK_TRY(alloc_dev(p, &p->ke[i], krylov_elems(p->desc.op, p->n, p->sol.storage, p->sol.bj_block) *
                                             (p->ke_hi ? 8 : xsize(p->sol.storage))));
      }
    }
  }
  if (p->ke_hi && !p->wx) RK_TRY(alloc_dev(p, &p->wx, N * xsize(p->sol.storage)));
  p->q = q;
  for (auto& v : p->warm_valid) v = false;  // stage slots change meaning
  std::memcpy(p->Ah, A_hi, sizeof(double) * q * q);
  std::memcpy(p->Al, A_lo, sizeof(double) * q * q);
  std::memcpy(p->b, b, sizeof(double) * q);
  return RK_OK;
}

rk_status rk_set_state(rk_problem* p, const double* u, int is_device_ptr) {
  if (!p || !u) {
    set_error("rk_set_state: NULL argument");
    return RK_ERR_ARG;
  }
  RK_CUDA(cudaMemcpyAsync(p->u, u, (size_t)p->N * 8,
                          is_device_ptr ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, p->st));
  RK_CUDA(cudaStreamSynchronize(p->st));
  p->has_state = true;
  return RK_OK;
}

rk_status rk_get_state(const rk_problem* p, double* u, int is_device_ptr) {
  if (!p || !u) {
    set_error("rk_get_state: NULL argument");
    return RK_ERR_ARG;
  }
  RK_CUDA(cudaMemcpyAsync(u, p->u, (size_t)p->N * 8,
                          is_device_ptr ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, p->st));
  RK_CUDA(cudaStreamSynchronize(p->st));
  return RK_OK;
}

rk_status rk_step(rk_problem* p, double dt, rk_stats* stats) { return rk_integrate(p, dt, 1, stats); }

rk_status rk_integrate(rk_problem* p, double dt, int nsteps, rk_stats* stats) {
  if (!p) {
    set_error("problem is NULL");
    return RK_ERR_ARG;
  }
  if (p->q == 0) {
    set_error("no tableau set");
    return RK_ERR_ARG;
  }
  if (!(dt > 0.0) || !std::isfinite(dt) || nsteps < 0) {
    set_error("dt must be positive and finite, nsteps >= 0");
    return RK_ERR_ARG;
  }
  auto t0 = std::chrono::steady_clock::now();
  rk_stats acc{};
  acc.true_res = -1.0;
  rk_status worst = RK_OK;
  for (int s = 0; s < nsteps; ++s) {
    rk_status st = step_impl(p, dt, &acc);
    if (st == RK_ERR_NOT_CONVERGED) {
      worst = st;
      continue;
    }
    if (st != RK_OK) {
      if (stats) *stats = acc;
      return st;
    }
  }
  RK_CUDA(cudaStreamSynchronize(p->st));
  acc.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (stats) *stats = acc;
  return worst;
}

rk_status rk_apply_op(rk_problem* p, const double* x, double* y, int is_device_ptr) {
  if (!p || !x || !y) {
    set_error("rk_apply_op: NULL argument");
    return RK_ERR_ARG;
  }
  const size_t bytes = (size_t)p->N * 8;
  const double* xin = x;
  double* yout = y;
  if (!is_device_ptr) {
    RK_CUDA(cudaMemcpyAsync(p->r, x, bytes, cudaMemcpyHostToDevice, p->st));
    xin = p->r;
    yout = p->g64;
  }
  RK_TRY(op_apply_f64(p, xin, yout, nullptr));
  if (!is_device_ptr) RK_CUDA(cudaMemcpyAsync(y, yout, bytes, cudaMemcpyDeviceToHost, p->st));
  RK_CUDA(cudaStreamSynchronize(p->st));
  return RK_OK;
}

rk_status rk_solve(rk_problem* p, double shift, const double* g, double* k, int is_device_ptr, rk_stats* stats) {
  if (!p || !g || !k) {
    set_error("rk_solve: NULL argument");
    return RK_ERR_ARG;
  }
  if (!(shift >= 0.0) || !std::isfinite(shift)) {
    set_error("shift must be finite and >= 0");
    return RK_ERR_ARG;
  }
  auto t0 = std::chrono::steady_clock::now();
  const size_t bytes = (size_t)p->N * 8;
  RK_CUDA(cudaMemcpyAsync(p->g64, g, bytes, is_device_ptr ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                          p->st));
  RhsScalars* rs = p->rs + 8;
  {
    auto kern = vec_norms_f64;
    launch(p, K_NORMS, 8.0 * p->N,
           [&] { kern<<<grid_for((const void*)kern, p->N), kThreads, 0, p->st>>>(p->g64, p->N, rs, p->partials); });
    RK_CUDA(cudaGetLastError());
  }
  // solve into the delta workspace (storage precision), then widen
  if (!p->wdelta) RK_TRY(alloc_dev(p, &p->wdelta, (size_t)p->N * xsize(p->sol.storage)));
  int iters = 0, status = 0;
  RK_TRY(krylov_solve(p, shift, p->g64, rs, p->wdelta, 8, &iters, &status));
  double* kout = is_device_ptr ? k : p->r;
  RK_TRY(launch_typed(p, [&](auto ts) {
    using S = typename decltype(ts)::type;
    auto kern = widen_f64<S>;
    launch(p, K_WIDEN, (8.0 + sizeof(S)) * p->N, [&] {
      kern<<<grid_for((const void*)kern, p->N), kThreads, 0, p->st>>>(static_cast<const S*>(p->wdelta), rs, kout,
                                                                       p->N);
    });
  }));
  if (!is_device_ptr) RK_CUDA(cudaMemcpyAsync(k, kout, bytes, cudaMemcpyDeviceToHost, p->st));
  RK_CUDA(cudaStreamSynchronize(p->st));
  if (stats) {
    *stats = rk_stats{};
    stats->iters_total = iters;
    stats->iters_max = iters;
    stats->solves = 1;
    stats->not_converged = (status == 4);
    stats->true_res = -1.0;
    stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  if (status == 5) {
    set_error("solve: non-finite value or Krylov breakdown");
    return RK_ERR_NONFINITE;
  }
  if (status == 6) {
    set_error("solve: a bounded device wait for a TMA tile gave up");
    return RK_ERR_TIMEOUT;
  }
  return status == 4 ? RK_ERR_NOT_CONVERGED : RK_OK;
}

rk_status rk_apply_precond(rk_problem* p, double shift, const double* r, double* z, int is_device_ptr) {
  if (!p || !r || !z) {
    set_error("rk_apply_precond: NULL argument");
    return RK_ERR_ARG;
  }
  const size_t bytes = (size_t)p->N * 8;
  const double* rin = r;
  double* zout = z;
  if (!is_device_ptr) {
    RK_CUDA(cudaMemcpyAsync(p->r, r, bytes, cudaMemcpyHostToDevice, p->st));
    rin = p->r;
    zout = p->g64;
  }
  if (p->desc.op != RK_OP_HEAT7) {
    RK_TRY(csr_precond_f64(p, shift, rin, zout));
  } else if (p->sol.precond == RK_PREC_FDM) {
    RK_TRY(fdm_precond_f64(p, shift, rin, zout));
  } else {
    const MinvEntry* me = nullptr;
    RK_TRY(get_minv_entry(p, shift, &me));
    rk_status lst = RK_OK;
    dispatch_st(p->sol.storage, [&](auto ts, auto tt) {
      using S = typename decltype(ts)::type;
      using T = typename decltype(tt)::type;
      dispatch_bs(p->sol.bj_block, [&](auto bsc) {
        constexpr int BS = decltype(bsc)::value;
        constexpr int SEG = seg_of<S, BS>();
        HeatGeo g = heat_geo(p, SEG);
        auto kern = bj_apply_f64io<S, T, BS, SEG>;
        const BjInv<T, BS> M = bj_param<T, BS>(me->host);
        launch(p, K_BJ, 16.0 * p->N, [&] {
          kern<<<grid_for((const void*)kern, g.n2 * g.nseg), kThreads, 0, p->st>>>(g, rin, M, zout);
        });
        if (cudaGetLastError() != cudaSuccess) lst = RK_ERR_CUDA;
      });
    });
    RK_TRY(lst);
  }
  if (!is_device_ptr) RK_CUDA(cudaMemcpyAsync(z, zout, bytes, cudaMemcpyDeviceToHost, p->st));
  RK_CUDA(cudaStreamSynchronize(p->st));
  return RK_OK;
}

}  // extern "C"

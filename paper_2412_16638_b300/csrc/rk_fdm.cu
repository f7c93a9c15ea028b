// Host side of the fast-diagonalization preconditioner (Sec. 3, Eq. Pinvform):
// one-time set-up per problem (sine basis, eigenvalues, temporary, tensor
// maps) and the six-pass application z = P^-1 r.
#include <cmath>
#include <mutex>

#include "rk_fdm.cuh"
#include "rk_internal.h"

namespace rk {

namespace {

// r (FP64) -> storage type, no scaling (the caller's values must fit it).
template <typename S>
__global__ void __launch_bounds__(kThreads) narrow_kernel(const double* __restrict__ in, S* __restrict__ out,
                                                          long long N) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
    out[i] = nar<S>(in[i]);
}

template <typename S>
__global__ void __launch_bounds__(kThreads) widen_kernel(const S* __restrict__ in, double* __restrict__ out,
                                                         long long N) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
    out[i] = wid<double>(in[i]);
}

// Host-side rounding of a double to the storage type.
template <typename S>
S host_round(double v) {
  if constexpr (std::is_same<S, float>::value)
    return (float)v;
  else if constexpr (std::is_same<S, __half>::value)
    return __double2half(v);
  else
    return __double2bfloat16(v);
}

// Largest dynamic shared memory a block of `kern` may use on this device:
// the opt-in limit minus the kernel's static shared memory.
int smem_dynamic_max(const void* kern) {
  int dev = 0, optin = 0;
  cudaFuncAttributes fa{};
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess || optin <= 0)
    optin = 227 * 1024;
  if (cudaFuncGetAttributes(&fa, kern) != cudaSuccess) fa.sharedSizeBytes = 4096;
  cudaGetLastError();
  return optin - (int)fa.sharedSizeBytes;
}

template <typename S>
rk_status setup_typed(rk_problem* p) {
  FdmState& f = *p->fdm;
  const int n = p->n;
  if (n > 256 || ((size_t)n * sizeof(S)) % 16 != 0) {
    set_error("fast diagonalization needs n <= 256 and n * %zu bytes a multiple of 16 (n = %d)", sizeof(S), n);
    return RK_ERR_ARG;
  }
  EncodeTiledFn enc = encode_fn();
  if (!enc) {
    set_error("cuTensorMapEncodeTiled is not available");
    return RK_ERR_CUDA;
  }
  // n <= 128: one CTA per 128-row tile with all N columns; n > 128: CTA
  // pairs on 256-row tiles, each CTA holding one N half of Q
  FdmGeo g{};
  g.n = n;
  g.rows = n * n;
  g.pair = n > 128 ? 1 : 0;
  g.nt = (n + 15) / 16 * 16;
  g.kblocks = (int)((n * sizeof(S) + 127) / 128);
  g.mtiles = g.pair ? (g.rows + kFdmPairRows - 1) / kFdmPairRows : (g.rows + kFdmRows - 1) / kFdmRows;
  const void* kern = g.pair ? (const void*)fdm_pass_pair<S> : (const void*)fdm_pass<S>;
  const int qrows = g.pair ? g.nt / 2 : g.nt;  // Q rows held by one CTA
  const size_t budget = (size_t)smem_dynamic_max(kern);
  const size_t fixed = fdm_smem_bytes(qrows, g.kblocks, 0);
  g.stages = budget > fixed ? (int)std::min<size_t>(kFdmMaxStages, (budget - fixed) / kFdmStageBytes) : 0;
  if (g.stages < 2) {
    set_error("fast diagonalization: shared memory too small for n = %d", n);
    return RK_ERR_ARG;
  }
  f.geo = g;
  f.smem = fdm_smem_bytes(qrows, g.kblocks, g.stages);

  // Q_jk = sqrt(2/(n+1)) sin((j+1)(k+1) pi/(n+1)); mu_k = 4 sin^2((k+1) pi/(2(n+1)))
  std::vector<S> qh((size_t)n * n);
  std::vector<float> muh(n);
  const double sc = std::sqrt(2.0 / (n + 1));
  for (int j = 0; j < n; ++j) {
    for (int k = 0; k < n; ++k) {
      // reduce (j+1)(k+1) modulo 2(n+1) so the sine argument stays in [0, 2 pi)
      const long long a = ((long long)(j + 1) * (k + 1)) % (2LL * (n + 1));
      qh[(size_t)j * n + k] = host_round<S>(sc * std::sin(M_PI * (double)a / (n + 1)));
    }
    const double s = std::sin(M_PI * (j + 1) / (2.0 * (n + 1)));
    muh[j] = (float)(4.0 * s * s);
  }
  RK_TRY(alloc_dev(p, &f.q, qh.size() * sizeof(S)));
  RK_TRY(alloc_dev(p, reinterpret_cast<void**>(&f.mu), muh.size() * sizeof(float)));
  RK_TRY(alloc_dev(p, &f.t, (size_t)p->N * sizeof(S)));
  RK_CUDA(cudaMemcpy(f.q, qh.data(), qh.size() * sizeof(S), cudaMemcpyHostToDevice));
  RK_CUDA(cudaMemcpy(f.mu, muh.data(), muh.size() * sizeof(float), cudaMemcpyHostToDevice));

  const cuuint32_t kb_elems = (cuuint32_t)(128 / sizeof(S));
  const cuuint32_t estr[2] = {1, 1};
  {
    const cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)n * n};
    const cuuint64_t strides[1] = {(cuuint64_t)n * sizeof(S)};
    const cuuint32_t box[2] = {kb_elems, (cuuint32_t)kFdmRows};
    void* bufs[3] = {p->wr, p->wz, f.t};
    CUtensorMap* maps[3] = {&f.in_r, &f.in_z, &f.in_t};
    for (int i = 0; i < 3; ++i)
      if (enc(maps[i], tma_dtype<S>(), 2, bufs[i], dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS) {
        set_error("tensor map of the fast-diagonalization input failed");
        return RK_ERR_CUDA;
      }
  }
  {
    const cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)n};
    const cuuint64_t strides[1] = {(cuuint64_t)n * sizeof(S)};
    const cuuint32_t box[2] = {kb_elems, (cuuint32_t)qrows};
    if (enc(&f.qmap, tma_dtype<S>(), 2, f.q, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS) {
      set_error("tensor map of the sine basis failed");
      return RK_ERR_CUDA;
    }
  }
  // Set once per kernel to the largest size any problem uses.  At least
  // 120 KB is requested so one CTA is resident per SM: its tensor memory
  // columns (256, or all 512 for a pair) are then always free at allocation.
  static std::once_flag once;
  static cudaError_t attr = cudaSuccess;
  std::call_once(once, [] {
    const void* k1 = (const void*)fdm_pass<S>;
    const void* k2 = (const void*)fdm_pass_pair<S>;
    attr = cudaFuncSetAttribute(k1, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_dynamic_max(k1));
    if (attr == cudaSuccess)
      attr = cudaFuncSetAttribute(k2, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_dynamic_max(k2));
    cudaGetLastError();
  });
  if (attr != cudaSuccess) {
    set_error("fdm_pass shared-memory attribute: %s", cudaGetErrorString(attr));
    return RK_ERR_CUDA;
  }
  f.smem = std::max<size_t>(f.smem, 120 * 1024);
  if (g.pair) {
    // persistent pairs: as many as can be resident at once (a cluster's two
    // CTAs must share a GPC, so this can be below half the SM count)
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2 * std::max(1, device_sms() / 2));
    cfg.blockDim = dim3(kFdmPairThreads);
    cfg.dynamicSmemBytes = f.smem;
    int clusters = 0;
    if (cudaOccupancyMaxActiveClusters(&clusters, (const void*)fdm_pass_pair<S>, &cfg) != cudaSuccess || clusters < 1) {
      cudaGetLastError();
      clusters = std::max(1, device_sms() / 2);
    }
    f.grid = 2 * std::min(g.mtiles, clusters);
  } else {
    f.grid = std::max(1, std::min(g.mtiles, device_sms()));
  }
  f.ok = true;
  return RK_OK;
}

template <typename S>
rk_status apply_typed(rk_problem* p, double shift, bool cg, int solve, int idx) {
  FdmState& f = *p->fdm;
  const FdmGeo g = f.geo;
  S* r = static_cast<S*>(p->wr);
  S* z = static_cast<S*>(p->wz);
  S* t = static_cast<S*>(f.t);
  const float c = (float)(shift * p->c);
  const double Ns = (double)p->N * sizeof(S);
  // r -> t -> z -> t (scaled by P_D^-1) -> z -> t -> z (with r.z)
  struct Pass {
    const CUtensorMap* in;
    S* out;
    int mode;
  } const passes[6] = {{&f.in_r, t, kFdmPlain}, {&f.in_t, z, kFdmPlain}, {&f.in_z, t, kFdmScale},
                       {&f.in_t, z, kFdmPlain}, {&f.in_z, t, kFdmPlain}, {&f.in_t, z, cg ? kFdmDot : kFdmPlain}};
  for (const Pass& ps : passes) {
    const int kid = ps.mode == kFdmDot ? K_FDM_DOT : (ps.mode == kFdmScale ? K_FDM_SCALE : K_FDM);
    prof_begin(p, kid, (ps.mode == kFdmDot ? 3.0 : 2.0) * Ns, cg ? solve : -1, cg ? idx : -1);
    if (g.pair)
      fdm_pass_pair<S><<<f.grid, kFdmPairThreads, f.smem, p->st>>>(*ps.in, f.qmap, g, ps.mode, c, f.mu, ps.out, r,
                                                                cg ? 1 : 0, p->sc, p->partials);
    else
      fdm_pass<S><<<f.grid, kFdmThreads, f.smem, p->st>>>(*ps.in, f.qmap, g, ps.mode, c, f.mu, ps.out, r, cg ? 1 : 0,
                                                           p->sc, p->partials);
    prof_end(p);
  }
  if (cudaGetLastError() != cudaSuccess) {
    set_error("fdm_pass launch failed");
    return RK_ERR_CUDA;
  }
  return RK_OK;
}

template <typename F>
rk_status dispatch_low(rk_problem* p, F&& f) {
  switch (p->sol.storage) {
    case RK_F32: return f(Tag<float>{});
    case RK_F16: return f(Tag<__half>{});
    case RK_BF16: return f(Tag<__nv_bfloat16>{});
    default:
      set_error("fast diagonalization needs FP32, FP16 or BF16 storage");
      return RK_ERR_ARG;
  }
}

}  // namespace

rk_status fdm_setup(rk_problem* p) {
  if (p->fdm && p->fdm->ok) return RK_OK;
  if (p->desc.op != RK_OP_HEAT7) {
    set_error("fast diagonalization is implemented for the constant-coefficient heat operator");
    return RK_ERR_ARG;
  }
  if (!p->fdm) p->fdm = new FdmState();
  return dispatch_low(p, [&](auto ts) {
    using S = typename decltype(ts)::type;
    return setup_typed<S>(p);
  });
}

rk_status fdm_apply(rk_problem* p, double shift, bool cg, int solve, int idx) {
  RK_TRY(fdm_setup(p));
  return dispatch_low(p, [&](auto ts) {
    using S = typename decltype(ts)::type;
    return apply_typed<S>(p, shift, cg, solve, idx);
  });
}

rk_status fdm_precond_f64(rk_problem* p, double shift, const double* r, double* z) {
  RK_TRY(fdm_setup(p));
  return dispatch_low(p, [&](auto ts) {
    using S = typename decltype(ts)::type;
    auto kn = narrow_kernel<S>;
    auto kw = widen_kernel<S>;
    // the passes report a timed-out wait in the CG scalars
    RK_CUDA(cudaMemsetAsync(p->sc, 0, sizeof(CgScalars), p->st));
    kn<<<grid_for((const void*)kn, p->N), kThreads, 0, p->st>>>(r, static_cast<S*>(p->wr), p->N);
    rk_status st = apply_typed<S>(p, shift, false, -1, -1);
    if (st != RK_OK) return st;
    kw<<<grid_for((const void*)kw, p->N), kThreads, 0, p->st>>>(static_cast<const S*>(p->wz), z, p->N);
    if (cudaGetLastError() != cudaSuccess) {
      set_error("fast-diagonalization conversion launch failed");
      return RK_ERR_CUDA;
    }
    RK_CUDA(cudaMemcpyAsync(p->h_sc, p->sc, sizeof(CgScalars), cudaMemcpyDeviceToHost, p->st));
    RK_CUDA(cudaStreamSynchronize(p->st));
    if (p->h_sc->status == 6) {
      set_error("fast-diagonalization pass: a bounded wait timed out");
      return RK_ERR_TIMEOUT;
    }
    return RK_OK;
  });
}

void fdm_free(rk_problem* p) {
  if (!p->fdm) return;
  if (p->fdm->q) free_dev(p, p->fdm->q);
  if (p->fdm->mu) free_dev(p, p->fdm->mu);
  if (p->fdm->t) free_dev(p, p->fdm->t);
  delete p->fdm;
  p->fdm = nullptr;
}

}  // namespace rk

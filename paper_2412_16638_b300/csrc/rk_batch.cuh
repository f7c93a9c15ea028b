// Batched stepping: many independent heat problems advanced by one
// persistent launch per step.  Each CTA takes the next problem from a work
// list (largest first, atomic counter) and performs the whole DIRK step for
// it -- stage right-hand sides, FP64 operator, block-Jacobi CG, FP64
// correction, update -- with CTA-wide reductions only, so the problems never
// wait on one another and no grid-wide barrier exists.
#pragma once
#include "rk_device.cuh"
#include "rk_heat.cuh"
#include "rk_vec.cuh"

namespace rk {

struct BatchItem {
  // problem
  int n, q, correct, max_iter;
  double c;                 // kappa / h^2
  double tol_rel, tol_abs;
  double Ah[64], Al[64], b[8];
  // device buffers of the problem
  double* u;
  double* r;
  double* g64;
  double* k[8];
  void* ke[8];              // solution type X (FP32 for 16-bit storage)
  void* wr;
  void* wz;
  void* wp[2];
  const void* minv[8];      // block-Jacobi inverse per stage (arithmetic type), null for explicit stages
  int want_scale;
  // outputs, accumulated over the steps of one call
  long long iters_total;
  int iters_max, solves, not_converged, status;
  double true_res_max;
};

#define RK_CTA_SEG_LOOP(g, SEG)                                                  \
  for (long long t_ = threadIdx.x; t_ < (long long)(g).n2 * (g).nseg; t_ += blockDim.x) { \
    const long long line = t_ / (g).nseg;                                        \
    const int sidx = (int)(t_ - line * (g).nseg);                                \
    const int i0 = sidx * (SEG);                                                 \
    const int m = min((SEG), (g).n - i0);                                        \
    const int j = (int)(line % (g).n);                                           \
    const int k = (int)(line / (g).n);                                           \
    const long long base = line * (g).n + i0;

// CTA-wide reduction of NV doubles, result broadcast to every thread.
template <int NV, unsigned MAXMASK>
__device__ __forceinline__ void cta_allreduce(double (&v)[NV], double* sred, double* sbc) {
  block_reduce<NV, MAXMASK>(v, sred);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int c = 0; c < NV; ++c) sbc[c] = v[c];
  }
  __syncthreads();
#pragma unroll
  for (int c = 0; c < NV; ++c) v[c] = sbc[c];
  __syncthreads();
}

template <typename S, typename T, int BS>
struct BatchStep {
  using X = typename XOf<S>::type;
  static constexpr int SEG = (BS > ((sizeof(S) == 2) ? 8 : 4)) ? BS : ((sizeof(S) == 2) ? 8 : 4);
  static constexpr int SEG64 = 4;

  // y = d x + o * (neighbour sum) in FP64; optional norms.
  static __device__ void apply64(const HeatGeo& g, const double* x, double* y, double d, double o, double (&nrm)[2],
                                 double* sred, double* sbc) {
    double acc[2] = {0.0, 0.0};
    RK_CTA_SEG_LOOP(g, SEG64)
      double xv[SEG64], nb[SEG64], yv[SEG64];
      load_seg<double, double, SEG64>(x + base, m, xv);
      nb_sum<double, SEG64>(
          g, i0, m, j, k, base, xv,
          [&](long long off, int mm, double (&v)[SEG64]) { load_seg<double, double, SEG64>(x + off, mm, v); },
          [&](long long idx) { return x[idx]; }, nb);
#pragma unroll
      for (int e = 0; e < SEG64; ++e) {
        yv[e] = fma(d, xv[e], o * nb[e]);
        if (e < m) {
          acc[0] = fma(yv[e], yv[e], acc[0]);
          acc[1] = fmax(acc[1], fabs(yv[e]));
        }
      }
      store_seg<double, double, SEG64>(y + base, m, yv);
    }
    __syncthreads();
    cta_allreduce<2, 2u>(acc, sred, sbc);
    nrm[0] = acc[0];
    nrm[1] = acc[1];
  }

  // k = g + cs * lap(ke) / sigma (FP64), returns sum (k - ke/sigma)^2.
  static __device__ double correct64(const HeatGeo& g, const double* gv, const X* ke, double cs, double inv_sigma,
                                     double* kout, double* sred, double* sbc) {
    double acc[1] = {0.0};
    RK_CTA_SEG_LOOP(g, SEG64)
      double v[SEG64], nb[SEG64], gs[SEG64], kv[SEG64];
      load_seg<double, X, SEG64>(ke + base, m, v);
      nb_sum<double, SEG64>(
          g, i0, m, j, k, base, v,
          [&](long long off, int mm, double (&w)[SEG64]) { load_seg<double, X, SEG64>(ke + off, mm, w); },
          [&](long long idx) { return wid<double>(ke[idx]); }, nb);
      load_seg<double, double, SEG64>(gv + base, m, gs);
#pragma unroll
      for (int e = 0; e < SEG64; ++e) {
        kv[e] = fma(cs * inv_sigma, fma(-6.0, v[e], nb[e]), gs[e]);
        const double res = kv[e] - v[e] * inv_sigma;
        if (e < m) acc[0] = fma(res, res, acc[0]);
      }
      store_seg<double, double, SEG64>(kout + base, m, kv);
    }
    __syncthreads();
    cta_allreduce<1, 0u>(acc, sred, sbc);
    return acc[0];
  }

  // CG on (d I + o * neighbour sum) x = sigma g, all vectors of the problem.
  static __device__ int cg(const HeatGeo& g, T d, T o, const double* gv, double sigma, double tol_rel,
                           double tol_abs, int max_iter, const T* sM, S* r, S* z, S* p0, S* p1, X* x, int* status,
                           double* sred, double* sbc) {
    // init
    double acc2[2] = {0.0, 0.0};
    RK_CTA_SEG_LOOP(g, SEG)
      (void)j;
      (void)k;
      (void)line;
      double gd[SEG];
      load_seg<double, double, SEG>(gv + base, m, gd);
      T rv[SEG], zv[SEG], zero[SEG];
#pragma unroll
      for (int e = 0; e < SEG; ++e) {
        rv[e] = (e < m) ? rnd<S, T>((T)(gd[e] * sigma)) : T(0);
        zero[e] = T(0);
      }
      bj_apply<T, BS, SEG>(sM, g.n, i0, rv, zv);
#pragma unroll
      for (int e = 0; e < SEG; ++e) {
        zv[e] = rnd<S, T>(zv[e]);
        if (e < m) {
          acc2[0] += (double)(rv[e] * zv[e]);
          acc2[1] += (double)(rv[e] * rv[e]);
        }
      }
      store_seg<S, T, SEG>(r + base, m, rv);
      store_seg<S, T, SEG>(z + base, m, zv);
      store_seg<X, T, SEG>(x + base, m, zero);
    }
    __syncthreads();
    cta_allreduce<2, 0u>(acc2, sred, sbc);
    double rz = acc2[0];
    const double ta = tol_abs * sigma;
    const double thresh2 = fmax(tol_rel * tol_rel * acc2[1], ta * ta);
    *status = 0;
    if (!isfinite(acc2[0]) || !isfinite(acc2[1])) {
      *status = 5;
      return 0;
    }
    if (acc2[1] <= thresh2 || acc2[1] == 0.0) return 0;
    double beta = 0.0;
    int it = 0;
    S* pbuf[2] = {p0, p1};
    while (true) {
      S* pn = pbuf[it & 1];
      const S* po = pbuf[(it & 1) ^ 1];
      const bool first = (it == 0);
      // sweep A
      double acc1[1] = {0.0};
      const T tb = (T)beta;
      RK_CTA_SEG_LOOP(g, SEG)
        auto pseg = [&](long long off, int mm, T (&v)[SEG]) {
          load_seg<T, S, SEG>(z + off, mm, v);
          if (!first) {
            T qv[SEG];
            load_seg<T, S, SEG>(po + off, mm, qv);
#pragma unroll
            for (int e = 0; e < SEG; ++e) v[e] = rnd<S, T>(fma(tb, qv[e], v[e]));
          }
        };
        auto ppt = [&](long long idx) {
          T v = wid<T>(z[idx]);
          if (!first) v = rnd<S, T>(fma(tb, wid<T>(po[idx]), v));
          return v;
        };
        T pv[SEG], nb[SEG];
        pseg(base, m, pv);
        nb_sum<T, SEG>(g, i0, m, j, k, base, pv, pseg, ppt, nb);
        T pw = T(0);
#pragma unroll
        for (int e = 0; e < SEG; ++e) {
          const T w = fma(d, pv[e], o * nb[e]);
          if (e < m) pw = fma(pv[e], w, pw);
        }
        acc1[0] += (double)pw;
        store_seg<S, T, SEG>(pn + base, m, pv);
      }
      __syncthreads();
      cta_allreduce<1, 0u>(acc1, sred, sbc);
      const double pAp = acc1[0];
      const double alpha = rz / pAp;
      if (!isfinite(pAp) || !isfinite(rz)) {
        *status = 5;
        return it;
      }
      if (!(pAp > 0.0) || !isfinite(alpha)) {  // attainable accuracy reached
        *status = 4;
        return it;
      }
      // sweep B
      const T ta_ = (T)alpha;
      double accb[2] = {0.0, 0.0};
      RK_CTA_SEG_LOOP(g, SEG)
        T pv[SEG], nb[SEG], rv[SEG], xv[SEG], zv[SEG];
        load_seg<T, S, SEG>(pn + base, m, pv);
        nb_sum<T, SEG>(
            g, i0, m, j, k, base, pv, [&](long long off, int mm, T (&v)[SEG]) { load_seg<T, S, SEG>(pn + off, mm, v); },
            [&](long long idx) { return wid<T>(pn[idx]); }, nb);
        load_seg<T, S, SEG>(r + base, m, rv);
        if (!first) {
          load_seg<T, X, SEG>(x + base, m, xv);
        } else {
#pragma unroll
          for (int e = 0; e < SEG; ++e) xv[e] = T(0);
        }
#pragma unroll
        for (int e = 0; e < SEG; ++e) {
          const T w = fma(d, pv[e], o * nb[e]);
          rv[e] = (e < m) ? rnd<S, T>(fma(-ta_, w, rv[e])) : T(0);
          xv[e] = fma(ta_, pv[e], xv[e]);
        }
        bj_apply<T, BS, SEG>(sM, g.n, i0, rv, zv);
        T rzl = T(0), rrl = T(0);
#pragma unroll
        for (int e = 0; e < SEG; ++e) {
          zv[e] = rnd<S, T>(zv[e]);
          if (e < m) {
            rzl = fma(rv[e], zv[e], rzl);
            rrl = fma(rv[e], rv[e], rrl);
          }
        }
        accb[0] += (double)rzl;
        accb[1] += (double)rrl;
        store_seg<X, T, SEG>(x + base, m, xv);
        store_seg<S, T, SEG>(r + base, m, rv);
        store_seg<S, T, SEG>(z + base, m, zv);
      }
      __syncthreads();
      cta_allreduce<2, 0u>(accb, sred, sbc);
      ++it;
      beta = accb[0] / rz;
      rz = accb[0];
      if (!isfinite(accb[0]) || !isfinite(accb[1])) {
        *status = 5;
        return it;
      }
      if (accb[1] <= thresh2) return it;
      if (it >= max_iter) {
        *status = 4;
        return it;
      }
    }
  }

  // u-combination r = u + sum ch k + sum ce ke/sigma (FP64), element-wise.
  static __device__ void combine(long long N, const double* u, double* out, const double* const* kh, const double* ch,
                                 int nh, const X* const* ke, const double* ce, int ne) {
    for (long long i = threadIdx.x; i < N; i += blockDim.x) {
      double v = u[i];
      for (int jj = 0; jj < nh; ++jj) v = fma(ch[jj], kh[jj][i], v);
      for (int jj = 0; jj < ne; ++jj) v = fma(ce[jj], wid<double>(ke[jj][i]), v);
      out[i] = v;
    }
    __syncthreads();
  }

  // One DIRK step of one problem (same stage loop as step_impl).
  static __device__ void step(BatchItem& it, double dt, T* sM, double* sred, double* sbc, double* ssig) {
    const int n = it.n, q = it.q;
    HeatGeo g64{n, (n + SEG64 - 1) / SEG64, (long long)n * n, (long long)n * n * n};
    HeatGeo gs{n, (n + SEG - 1) / SEG, (long long)n * n, (long long)n * n * n};
    const long long N = g64.N;
    const bool mixed = it.correct != 0;
    __shared__ const double* s_kh[kMaxStages];
    __shared__ double s_ch[kMaxStages];
    __shared__ const X* s_ke[kMaxStages];
    __shared__ double s_ce[kMaxStages];
    __shared__ int s_nh, s_ne;
    for (int i = 0; i < q; ++i) {
      if (threadIdx.x == 0) {
        int nh = 0, ne = 0;
        for (int jj = 0; jj < i; ++jj) {
          double chj = dt * it.Ah[i * q + jj], cej = dt * it.Al[i * q + jj];
          const bool impl_j = it.Al[jj * q + jj] != 0.0;
          if (cej != 0.0 && (!impl_j || !mixed)) {
            chj += cej;
            cej = 0.0;
          }
          if (chj != 0.0) {
            s_kh[nh] = it.k[jj];
            s_ch[nh++] = chj;
          }
          if (cej != 0.0) {
            s_ke[ne] = static_cast<const X*>(it.ke[jj]);
            s_ce[ne++] = cej / ssig[jj];
          }
        }
        s_nh = nh;
        s_ne = ne;
      }
      __syncthreads();
      const double* rp = it.u;
      if (s_nh + s_ne > 0) {
        combine(N, it.u, it.r, s_kh, s_ch, s_nh, s_ke, s_ce, s_ne);
        rp = it.r;
      }
      const double a = it.Al[i * q + i];
      if (a == 0.0) {
        double nrm[2];
        apply64(g64, rp, it.k[i], -6.0 * it.c, it.c, nrm, sred, sbc);
        if (threadIdx.x == 0) ssig[i] = 1.0;
        __syncthreads();
        continue;
      }
      const double shift = dt * a;
      double nrm[2];
      apply64(g64, rp, it.g64, -6.0 * it.c, it.c, nrm, sred, sbc);
      const double sigma = (it.want_scale && nrm[1] > 0.0 && isfinite(nrm[1])) ? 1.0 / nrm[1] : 1.0;
      if (threadIdx.x == 0) ssig[i] = mixed ? sigma : 1.0;
      // block-Jacobi inverse of this stage into shared memory
      const T* Mi = static_cast<const T*>(it.minv[i]);
      for (int e = threadIdx.x; e < 2 * BS * BS; e += blockDim.x) sM[e] = Mi[e];
      __syncthreads();
      int status = 0;
      X* xk = static_cast<X*>(it.ke[i]);
      const int iters = cg(gs, (T)(1.0 + 6.0 * shift * it.c), (T)(-shift * it.c), it.g64, sigma, it.tol_rel,
                           it.tol_abs, it.max_iter, sM, static_cast<S*>(it.wr), static_cast<S*>(it.wz),
                           static_cast<S*>(it.wp[0]), static_cast<S*>(it.wp[1]), xk, &status, sred, sbc);
      if (threadIdx.x == 0) {
        it.iters_total += iters;
        it.iters_max = max(it.iters_max, iters);
        it.solves += 1;
        if (status == 4) it.not_converged += 1;
        if (status == 5) it.status = 5;
      }
      if (mixed) {
        const double res2 = correct64(g64, it.g64, xk, shift * it.c, 1.0 / sigma, it.k[i], sred, sbc);
        if (threadIdx.x == 0 && nrm[0] > 0.0) it.true_res_max = fmax(it.true_res_max, sqrt(res2 / nrm[0]));
      } else if ((void*)it.ke[i] != (void*)it.k[i]) {
        for (long long e = threadIdx.x; e < N; e += blockDim.x) it.k[i][e] = wid<double>(xk[e]) / sigma;
        __syncthreads();
      }
    }
    // update u += dt sum b_j k_j
    for (long long e = threadIdx.x; e < N; e += blockDim.x) {
      double v = it.u[e];
      for (int jj = 0; jj < q; ++jj)
        if (it.b[jj] != 0.0) v = fma(dt * it.b[jj], it.k[jj][e], v);
      it.u[e] = v;
    }
    __syncthreads();
  }
};

// Persistent batched step: CTAs take problems from order[] through *counter.
template <typename S, typename T, int BS>
__global__ void __launch_bounds__(512, 1) batch_step_kernel(BatchItem* items, const int* order, int count, double dt, int* counter) {
  __shared__ T sM[2 * BS * BS];
  __shared__ double sred[64];
  __shared__ double sbc[4];
  __shared__ double ssig[kMaxStages];
  __shared__ int s_idx;
  while (true) {
    if (threadIdx.x == 0) s_idx = atomicAdd(counter, 1);
    __syncthreads();
    const int w = s_idx;
    __syncthreads();
    if (w >= count) return;
    BatchStep<S, T, BS>::step(items[order[w]], dt, sM, sred, sbc, ssig);
  }
}

struct LaunchCfg {
  int threads = 512;
  int ctas_per_sm = 2;
  int grid = 0;  // filled in for a given group
};

// Host helpers, explicitly instantiated per storage type in rk_batch_*.cu
// (the arithmetic type is FP64 for FP64 storage, FP32 otherwise).
template <typename S>
int batch_grid_s(int bs, const LaunchCfg& cfg, int count, int sms);
template <typename S>
void batch_launch_s(int bs, const LaunchCfg& cfg, int grid, BatchItem* items, const int* order, int count, double dt,
                    int* counter, cudaStream_t st);

#ifdef RK_BATCH_INSTANTIATE
template <typename S>
struct ArithOf { using type = float; };
template <>
struct ArithOf<double> { using type = double; };

template <typename S, typename F>
static void batch_dispatch_bs(int bs, F&& f) {
  switch (bs) {
    case 1: f(batch_step_kernel<S, typename ArithOf<S>::type, 1>); break;
    case 2: f(batch_step_kernel<S, typename ArithOf<S>::type, 2>); break;
    case 4: f(batch_step_kernel<S, typename ArithOf<S>::type, 4>); break;
    case 8: f(batch_step_kernel<S, typename ArithOf<S>::type, 8>); break;
    case 16: f(batch_step_kernel<S, typename ArithOf<S>::type, 16>); break;
    default: f(batch_step_kernel<S, typename ArithOf<S>::type, 32>); break;
  }
}

template <typename S>
int batch_grid_s(int bs, const LaunchCfg& cfg, int count, int sms) {
  int grid = 1;
  batch_dispatch_bs<S>(bs, [&](auto kern) {
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, cfg.threads, 0) != cudaSuccess || occ < 1) occ = 1;
    const int per_sm = cfg.ctas_per_sm < occ ? cfg.ctas_per_sm : occ;
    grid = count < sms * per_sm ? count : sms * per_sm;
    if (grid < 1) grid = 1;
  });
  return grid;
}

template <typename S>
void batch_launch_s(int bs, const LaunchCfg& cfg, int grid, BatchItem* items, const int* order, int count, double dt,
                    int* counter, cudaStream_t st) {
  cudaMemsetAsync(counter, 0, sizeof(int), st);
  batch_dispatch_bs<S>(bs, [&](auto kern) { kern<<<grid, cfg.threads, 0, st>>>(items, order, count, dt, counter); });
}
#endif

}  // namespace rk

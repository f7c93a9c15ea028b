// Kernels of the advection-diffusion path: CSR operator (FP64 and storage
// precision), block-Jacobi with per-block inverses, and right-preconditioned
// restarted GMRES(m) with classical Gram-Schmidt applied twice (CGS2).  The
// Arnoldi/Hessenberg/Givens state lives on the device; the last CTA of each
// reduction updates it, so the host only polls a status word.
//
// Thread mapping of the vector kernels is the x-line segment mapping of the
// heat path (RK_SEG_LOOP): block-Jacobi blocks (x-line segments of BS nodes)
// lie inside one thread's segment.
#pragma once
#include "rk_device.cuh"
#include "rk_heat.cuh"

namespace rk {

constexpr int kGmMax = 64;  // largest restart length

struct CsrView {
  const int* rowptr;
  const int* cols;
};

// Device-resident GMRES state.  The header (up to `ticket`) is what the host
// polls.
struct GmScalars {
  int j;          // Arnoldi index within the current cycle
  int iter;       // total Arnoldi steps
  int max_iter;
  int m;          // restart length
  int cycle_end;  // 1: the cycle has finished, x must be updated
  int done;       // 1: stop (converged, max_iter or breakdown)
  int status;     // 0 ok, 4 not converged, 5 non-finite
  int jused;      // basis vectors used by the finished cycle
  unsigned ticket;
  int verify;     // 1: a converged cycle is confirmed by the true residual of
                  // the restart (compressed basis: x is assembled from it)
  int conv_est;   // verify mode: the cycle that just ended converged by its estimate
  int pad2;
  double beta;    // residual norm at the start of the cycle
  double bnorm;   // ||sigma g||
  double thresh;  // stopping threshold on the residual norm
  double tol_rel, tol_abs;
  double hnext;   // ||w|| of the last Arnoldi step before rotation
  double res;     // current residual estimate |g_{j+1}|
  double h1[kGmMax + 1], h2[kGmMax + 1];
  double H[(kGmMax + 1) * kGmMax];  // column-major (m+1) x m
  double cs[kGmMax], sn[kGmMax], gv[kGmMax + 1], y[kGmMax];
};

// ------------------------------------------------------------- FP64 CSR ops
// y = L x + f (FP64; f the optional forcing, nullptr = none); with rs != null
// also ||y||^2, ||y||_inf and the storage scale.
__global__ void __launch_bounds__(kThreads) csr_apply_f64_kernel(CsrView A, const double* __restrict__ vals,
                                                                 long long N, const double* __restrict__ x,
                                                                 const double* __restrict__ f,
                                                                 double* __restrict__ y, RhsScalars* rs,
                                                                 double* partials);

// k = g + shift * L (ke/sigma) in FP64, true residual ||k - ke/sigma||^2 -> rs->res2.
template <typename X>
__global__ void __launch_bounds__(kThreads) csr_correct_f64_kernel(CsrView A, const double* __restrict__ vals,
                                                                   long long N, const double* __restrict__ gv,
                                                                   const X* __restrict__ ke, double shift,
                                                                   double* __restrict__ kout, RhsScalars* rs,
                                                                   double* partials) {
  const double inv_sigma = 1.0 / rs->sigma;
  double acc[1] = {0.0};
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < N;
       r += (long long)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int e = A.rowptr[r]; e < A.rowptr[r + 1]; ++e) s = fma(vals[e], wid<double>(ke[A.cols[e]]), s);
    const double v = wid<double>(ke[r]) * inv_sigma;
    const double k = fma(shift * inv_sigma, s, gv[r]);
    kout[r] = k;
    const double res = k - v;
    acc[0] = fma(res, res, acc[0]);
  }
  double tot[1];
  if (grid_reduce<1, 0u>(acc, partials, &rs->ticket, tot)) rs->res2 = tot[0];
}

// ------------------------------------------------------------- block-Jacobi
// Per-block inverses of the x-line-segment blocks of I - shift L.  One thread
// per block: the block of a 7-point operator restricted to an x-line segment
// is tridiagonal; its inverse is formed column by column with the Thomas
// recurrences in FP64 (the blocks are diagonally dominant M-matrices, so no
// pivoting is needed) and stored row-major, zero padded to BS x BS.
template <typename S, int BS>
__global__ void __launch_bounds__(kThreads) csr_bj_setup(CsrView A, const double* __restrict__ vals, int n,
                                                         double shift, S* __restrict__ minv) {
  const int nbl = (n + BS - 1) / BS;
  const long long nblocks = (long long)n * n * nbl;
  for (long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x; b < nblocks;
       b += (long long)gridDim.x * blockDim.x) {
    const long long line = b / nbl;
    const int i0 = (int)(b - line * nbl) * BS;
    const int m = min(BS, n - i0);
    const long long r0 = line * n + i0;
    double lo[BS], di[BS], up[BS];
    for (int i = 0; i < m; ++i) {
      const long long r = r0 + i;
      double a = 0.0, d = 0.0, c = 0.0;
      for (int e = A.rowptr[r]; e < A.rowptr[r + 1]; ++e) {
        const long long col = A.cols[e];
        if (col == r) d = vals[e];
        else if (col == r - 1 && i > 0) a = vals[e];
        else if (col == r + 1 && i + 1 < m) c = vals[e];
      }
      lo[i] = -shift * a;
      di[i] = 1.0 - shift * d;
      up[i] = -shift * c;
    }
    // Thomas forward elimination of the matrix (independent of the rhs)
    double cp[BS], den[BS];
    for (int i = 0; i < m; ++i) {
      den[i] = di[i] - (i > 0 ? lo[i] * cp[i - 1] : 0.0);
      cp[i] = (i + 1 < m) ? up[i] / den[i] : 0.0;
    }
    S* out = minv + b * BS * BS;
    for (int jcol = 0; jcol < BS; ++jcol) {
      double xcol[BS];
      if (jcol < m) {
        double dp[BS];
        for (int i = 0; i < m; ++i) {
          const double rhs = (i == jcol) ? 1.0 : 0.0;
          dp[i] = (rhs - (i > 0 ? lo[i] * dp[i - 1] : 0.0)) / den[i];
        }
        for (int i = m - 1; i >= 0; --i) xcol[i] = dp[i] - (i + 1 < m ? cp[i] * xcol[i + 1] : 0.0);
      }
      for (int i = 0; i < BS; ++i)
        out[i * BS + jcol] = nar<S>((i < m && jcol < m) ? xcol[i] : 0.0);
    }
  }
}

// z = D^{-1} r for the blocks of one segment (per-block inverses in S).
template <typename T, typename S, int BS, int SEG>
__device__ __forceinline__ void bj_apply_blocks(const S* __restrict__ minv, long long line, int nbl, int i0,
                                                const T (&r)[SEG], T (&z)[SEG]) {
#pragma unroll
  for (int cb = 0; cb < SEG / BS; ++cb) {
    const int bi = i0 / BS + cb;
    if (bi >= nbl) {
#pragma unroll
      for (int i = 0; i < BS; ++i) z[cb * BS + i] = T(0);
      continue;
    }
    const S* M = minv + (line * nbl + bi) * (long long)(BS * BS);
#pragma unroll
    for (int i = 0; i < BS; ++i) {
      T row[BS];
      load_seg<T, S, BS>(M + i * BS, BS, row);
      T a = T(0);
#pragma unroll
      for (int jj = 0; jj < BS; ++jj) a = fma(row[jj], r[cb * BS + jj], a);
      z[cb * BS + i] = a;
    }
  }
}

template <typename S, typename T, int BS, int SEG>
__global__ void __launch_bounds__(kThreads) csr_bj_apply_f64io(HeatGeo g, const S* __restrict__ minv,
                                                               const double* __restrict__ r, double* __restrict__ z) {
  const int nbl = (g.n + BS - 1) / BS;
  RK_SEG_LOOP(g, SEG)
    (void)j;
    (void)k;
    double rd[SEG];
    load_seg<double, double, SEG>(r + base, m, rd);
    T rv[SEG], zv[SEG];
#pragma unroll
    for (int e = 0; e < SEG; ++e) rv[e] = (e < m) ? rnd<S, T>((T)rd[e]) : T(0);
    bj_apply_blocks<T, S, BS, SEG>(minv, line, nbl, i0, rv, zv);
    double zd[SEG];
#pragma unroll
    for (int e = 0; e < SEG; ++e) zd[e] = (double)rnd<S, T>(zv[e]);
    store_seg<double, double, SEG>(z + base, m, zd);
  RK_SEG_LOOP_END
}

// (I - shift L) applied to the m <= SEG consecutive rows base .. base+m-1 of
// a storage-precision vector: x_r - (shift/lscale) sum_e Lhat_re x_c, with
// Lhat = lscale * L stored in S.  The k-th entries of all rows are loaded together (k = 0 .. 6: the
// operators assembled here have at most 7 entries per row; longer rows finish
// in a plain loop), so the gathers of a segment are in flight at once instead
// of one dependent row-pointer -> column -> x chain per row.  Per row the
// entries are summed in column order.
template <typename T, typename S, typename V, int SEG>
__device__ __forceinline__ void shifted_seg(CsrView A, const S* __restrict__ lv, long long base, int m,
                                            const V* __restrict__ x, T cs, T (&out)[SEG]) {
  constexpr int kNnz = 7;
  int rp[SEG + 1];
#pragma unroll
  for (int i = 0; i <= SEG; ++i) rp[i] = (i <= m) ? A.rowptr[base + i] : 0;
  T s[SEG];
#pragma unroll
  for (int i = 0; i < SEG; ++i) s[i] = T(0);
#pragma unroll
  for (int k = 0; k < kNnz; ++k) {
#pragma unroll
    for (int i = 0; i < SEG; ++i) {
      const int e = rp[i] + k;
      if (i < m && e < rp[i + 1]) s[i] = fma(wid<T>(lv[e]), wid<T>(x[A.cols[e]]), s[i]);
    }
  }
#pragma unroll
  for (int i = 0; i < SEG; ++i) {
    if (i < m)
      for (int e = rp[i] + kNnz; e < rp[i + 1]; ++e) s[i] = fma(wid<T>(lv[e]), wid<T>(x[A.cols[e]]), s[i]);
    out[i] = (i < m) ? fma(-cs, s[i], wid<T>(x[base + i])) : T(0);
  }
}

// ------------------------------------------------------------- GMRES kernels
// Per-thread multi-segment layout of the reduction kernels: thread t of T
// handles segments t, t+T, ..., t+(R-1)T.
#define RK_GM_SEGS(g, SEG, R)                                                    \
  const long long nsegs_ = (long long)(g).n2 * (g).nseg;                         \
  const long long tthreads_ = (long long)gridDim.x * blockDim.x;                 \
  const long long tid_ = (long long)blockIdx.x * blockDim.x + threadIdx.x;

struct SegPos {
  long long base;
  int m;
  int i0;
  long long line;
  bool valid;
};

__device__ __forceinline__ SegPos seg_pos(const HeatGeo& g, long long sidx, int SEG) {
  SegPos p;
  p.valid = sidx < (long long)g.n2 * g.nseg;
  if (!p.valid) {
    p.base = 0;
    p.m = 0;
    p.i0 = 0;
    p.line = 0;
    return p;
  }
  p.line = sidx / g.nseg;
  p.i0 = (int)(sidx - p.line * g.nseg) * SEG;
  p.m = min(SEG, g.n - p.i0);
  p.base = p.line * g.n + p.i0;
  return p;
}

// Sum over the CTA, then over CTAs, of each of `cnt` per-thread values dot(i)
// (per-CTA sums at partials[cta*kGmMax + i]); the last CTA returns true in
// thread 0 with the totals in out[i].  Each dot is reduced within its warp by
// shuffles only, so the loads of the next basis vector are not held behind a
// barrier; one barrier then combines the warps.  Fixed order: deterministic.
template <typename F>
__device__ __forceinline__ bool multi_dot_reduce(int cnt, F dot, double* partials, unsigned* ticket, double* out) {
  constexpr int kWarps = kThreads / 32;
  __shared__ double swarp[kWarps][kGmMax + 1];
  __shared__ int am_last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = 0; i < cnt; ++i) {
    double v = dot(i);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if (lane == 0) swarp[warp][i] = v;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
    double a = 0.0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) a += swarp[w][i];
    partials[(size_t)blockIdx.x * kGmMax + i] = a;
    __threadfence();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned t = atomicAdd(ticket, 1u);
    am_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!am_last) return false;
  __threadfence();
  // last CTA: warp w sums dots i = w, w + kWarps, ... over the CTAs
  for (int i = warp; i < cnt; i += kWarps) {
    double a = 0.0;
    for (int b = lane; b < (int)gridDim.x; b += 32) a += __ldcg(partials + (size_t)b * kGmMax + i);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) a += __shfl_down_sync(0xffffffffu, a, off);
    if (lane == 0) out[i] = a;
  }
  __syncthreads();
  if (threadIdx.x == 0) *ticket = 0u;
  return threadIdx.x == 0;
}

// Start of a solve from x = 0: V_0 <- sigma g (rounded to B, unnormalised),
// x <- 0, beta = ||V_0||.
template <typename S, typename B, typename T, int SEG>
__global__ void __launch_bounds__(kThreads) gm_start(HeatGeo g, const double* __restrict__ gv, const RhsScalars* rs,
                                                     B* __restrict__ V0, typename XOf<S>::type* __restrict__ x,
                                                     GmScalars* sc, double* partials) {
  using X = typename XOf<S>::type;
  const double sigma = rs->sigma;
  double acc[1] = {0.0};
  RK_SEG_LOOP(g, SEG)
    (void)j;
    (void)k;
    (void)line;
    double gd[SEG];
    load_seg<double, double, SEG>(gv + base, m, gd);
    T v[SEG], zero[SEG];
#pragma unroll
    for (int e = 0; e < SEG; ++e) {
      v[e] = (e < m) ? rnd<B, T>((T)(gd[e] * sigma)) : T(0);
      zero[e] = T(0);
      acc[0] += (double)(v[e] * v[e]);
    }
    store_seg<B, T, SEG>(V0 + base, m, v);
    store_seg<X, T, SEG>(x + base, m, zero);
  RK_SEG_LOOP_END
  double tot[1];
  if (grid_reduce<1, 0u>(acc, partials, &sc->ticket, tot)) {
    const double beta = sqrt(tot[0]);
    sc->beta = beta;
    sc->bnorm = beta;
    const double ta = sc->tol_abs * sigma;
    sc->thresh = fmax(sc->tol_rel * beta, ta);
    sc->j = 0;
    sc->iter = 0;
    sc->cycle_end = 0;
    sc->jused = 0;
    sc->res = beta;
    sc->gv[0] = beta;
    sc->status = 0;
    if (!isfinite(beta)) {
      sc->done = 1;
      sc->status = 5;
    } else {
      sc->done = (beta <= sc->thresh || beta == 0.0) ? 1 : 0;
    }
  }
}

// Restart: V_0 <- sigma g - (I - shift L) x, beta = ||V_0||.
template <typename S, typename B, typename T, int SEG>
__global__ void __launch_bounds__(kThreads) gm_restart(HeatGeo g, CsrView A, const S* __restrict__ lv, T cs,
                                                       const double* __restrict__ gv, const RhsScalars* rs,
                                                       const typename XOf<S>::type* __restrict__ x,
                                                       B* __restrict__ V0, GmScalars* sc, double* partials) {
  if (sc->done) return;
  const double sigma = rs->sigma;
  double acc[1] = {0.0};
  RK_SEG_LOOP(g, SEG)
    (void)j;
    (void)k;
    (void)line;
    T v[SEG], ax[SEG];
    shifted_seg<T, S, typename XOf<S>::type, SEG>(A, lv, base, m, x, cs, ax);
#pragma unroll
    for (int e = 0; e < SEG; ++e) {
      v[e] = T(0);
      if (e < m) {
        v[e] = rnd<B, T>((T)(gv[base + e] * sigma) - ax[e]);
        acc[0] += (double)(v[e] * v[e]);
      }
    }
    store_seg<B, T, SEG>(V0 + base, m, v);
  RK_SEG_LOOP_END
  double tot[1];
  if (grid_reduce<1, 0u>(acc, partials, &sc->ticket, tot)) {
    const double beta = sqrt(tot[0]);
    const double prev = sc->beta;  // true residual at the start of the cycle that ended
    sc->beta = beta;
    sc->j = 0;
    sc->cycle_end = 0;
    sc->jused = 0;
    sc->res = beta;
    sc->gv[0] = beta;
    if (!isfinite(beta)) {
      sc->done = 1;
      sc->status = 5;
    } else if (beta <= sc->thresh) {
      sc->done = 1;
    } else if (sc->conv_est && beta > 0.5 * prev) {
      // a cycle that converged by its estimate no longer halves the true
      // residual: the attainable accuracy of the working precision is reached
      sc->done = 1;
    }
    sc->conv_est = 0;
  }
}

// Arnoldi step part 1: normalise V_j (lazily: it was stored unnormalised) and
// z = D^{-1} V_j.
template <typename S, typename B, typename T, int BS, int SEG>
__global__ void __launch_bounds__(kThreads) gm_prec(HeatGeo g, B* __restrict__ V, long long ldv,
                                                    const S* __restrict__ minv, S* __restrict__ z, GmScalars* sc) {
  if (sc->done || sc->cycle_end) return;
  const int jj = sc->j;
  const T f = (T)(1.0 / (jj == 0 ? sc->beta : sc->hnext));
  B* Vj = V + (long long)jj * ldv;
  const int nbl = (g.n + BS - 1) / BS;
  RK_SEG_LOOP(g, SEG)
    (void)j;
    (void)k;
    T v[SEG], zv[SEG];
    load_seg<T, B, SEG>(Vj + base, m, v);
#pragma unroll
    for (int e = 0; e < SEG; ++e) v[e] = (e < m) ? rnd<B, T>(v[e] * f) : T(0);
    bj_apply_blocks<T, S, BS, SEG>(minv, line, nbl, i0, v, zv);
    store_seg<B, T, SEG>(Vj + base, m, v);
    store_seg<S, T, SEG>(z + base, m, zv);
  RK_SEG_LOOP_END
}

// Arnoldi step part 2: w = (I - shift L) z written to V_{j+1}; h1_i = V_i . w
// for i <= j (first Gram-Schmidt projection coefficients).
template <typename S, typename B, typename T, int SEG, int R>
__global__ void __launch_bounds__(kThreads) gm_spmv_dots(HeatGeo g, CsrView A, const S* __restrict__ lv, T cs,
                                                         const S* __restrict__ z, B* __restrict__ V, long long ldv,
                                                         GmScalars* sc, double* partials) {
  if (sc->done || sc->cycle_end) return;
  const int jj = sc->j;
  RK_GM_SEGS(g, SEG, R)
  T w[R][SEG];
  SegPos pos[R];
  B* W = V + (long long)(jj + 1) * ldv;
#pragma unroll
  for (int q = 0; q < R; ++q) {
    pos[q] = seg_pos(g, tid_ + q * tthreads_, SEG);
    if (pos[q].valid) {
      shifted_seg<T, S, S, SEG>(A, lv, pos[q].base, pos[q].m, z, cs, w[q]);
#pragma unroll
      for (int e = 0; e < SEG; ++e) w[q][e] = rnd<B, T>(w[q][e]);
      store_seg<B, T, SEG>(W + pos[q].base, pos[q].m, w[q]);
    } else {
#pragma unroll
      for (int e = 0; e < SEG; ++e) w[q][e] = T(0);
    }
  }
  auto dot = [&](int i) {
    const B* Vi = V + (long long)i * ldv;
    T a = T(0);
#pragma unroll
    for (int q = 0; q < R; ++q) {
      if (!pos[q].valid) continue;
      T vi[SEG];
      load_seg<T, B, SEG>(Vi + pos[q].base, pos[q].m, vi);
#pragma unroll
      for (int e = 0; e < SEG; ++e) a = fma(vi[e], w[q][e], a);
    }
    return (double)a;
  };
  multi_dot_reduce(jj + 1, dot, partials, &sc->ticket, sc->h1);
}

// Arnoldi step part 3 (second CGS pass): w <- w - sum_i h1_i V_i, then
// h2_i = V_i . w.
template <typename S, typename B, typename T, int SEG, int R>
__global__ void __launch_bounds__(kThreads) gm_orth(HeatGeo g, B* __restrict__ V, long long ldv, GmScalars* sc,
                                                    double* partials) {
  if (sc->done || sc->cycle_end) return;
  const int jj = sc->j;
  RK_GM_SEGS(g, SEG, R)
  T w[R][SEG];
  SegPos pos[R];
  B* W = V + (long long)(jj + 1) * ldv;
#pragma unroll
  for (int q = 0; q < R; ++q) {
    pos[q] = seg_pos(g, tid_ + q * tthreads_, SEG);
    if (pos[q].valid) {
      load_seg<T, B, SEG>(W + pos[q].base, pos[q].m, w[q]);
    } else {
#pragma unroll
      for (int e = 0; e < SEG; ++e) w[q][e] = T(0);
    }
  }
  for (int i = 0; i <= jj; ++i) {
    const T hi = (T)sc->h1[i];
    const B* Vi = V + (long long)i * ldv;
#pragma unroll
    for (int q = 0; q < R; ++q) {
      if (!pos[q].valid) continue;
      T vi[SEG];
      load_seg<T, B, SEG>(Vi + pos[q].base, pos[q].m, vi);
#pragma unroll
      for (int e = 0; e < SEG; ++e) w[q][e] = fma(-hi, vi[e], w[q][e]);
    }
  }
#pragma unroll
  for (int q = 0; q < R; ++q) {
#pragma unroll
    for (int e = 0; e < SEG; ++e) w[q][e] = (pos[q].valid && e < pos[q].m) ? rnd<B, T>(w[q][e]) : T(0);
    if (pos[q].valid) store_seg<B, T, SEG>(W + pos[q].base, pos[q].m, w[q]);
  }
  auto dot = [&](int i) {
    const B* Vi = V + (long long)i * ldv;
    T a = T(0);
#pragma unroll
    for (int q = 0; q < R; ++q) {
      if (!pos[q].valid) continue;
      T vi[SEG];
      load_seg<T, B, SEG>(Vi + pos[q].base, pos[q].m, vi);
#pragma unroll
      for (int e = 0; e < SEG; ++e) a = fma(vi[e], w[q][e], a);
    }
    return (double)a;
  };
  multi_dot_reduce(jj + 1, dot, partials, &sc->ticket, sc->h2);
}

// Arnoldi step part 4: w <- w - sum_i h2_i V_i, ||w||; the last CTA forms the
// Hessenberg column (h1 + h2, ||w||), applies the Givens rotations, tests
// convergence and, at the end of a cycle, solves the triangular system.
template <typename S, typename B, typename T, int SEG, int R>
__global__ void __launch_bounds__(kThreads) gm_norm(HeatGeo g, B* __restrict__ V, long long ldv, GmScalars* sc,
                                                    double* partials) {
  if (sc->done || sc->cycle_end) return;
  const int jj = sc->j;
  RK_GM_SEGS(g, SEG, R)
  T w[R][SEG];
  SegPos pos[R];
  B* W = V + (long long)(jj + 1) * ldv;
#pragma unroll
  for (int q = 0; q < R; ++q) {
    pos[q] = seg_pos(g, tid_ + q * tthreads_, SEG);
    if (pos[q].valid) {
      load_seg<T, B, SEG>(W + pos[q].base, pos[q].m, w[q]);
    } else {
#pragma unroll
      for (int e = 0; e < SEG; ++e) w[q][e] = T(0);
    }
  }
  for (int i = 0; i <= jj; ++i) {
    const T hi = (T)sc->h2[i];
    const B* Vi = V + (long long)i * ldv;
#pragma unroll
    for (int q = 0; q < R; ++q) {
      if (!pos[q].valid) continue;
      T vi[SEG];
      load_seg<T, B, SEG>(Vi + pos[q].base, pos[q].m, vi);
#pragma unroll
      for (int e = 0; e < SEG; ++e) w[q][e] = fma(-hi, vi[e], w[q][e]);
    }
  }
  double acc[1] = {0.0};
#pragma unroll
  for (int q = 0; q < R; ++q) {
#pragma unroll
    for (int e = 0; e < SEG; ++e) {
      w[q][e] = (pos[q].valid && e < pos[q].m) ? rnd<B, T>(w[q][e]) : T(0);
      acc[0] += (double)(w[q][e] * w[q][e]);
    }
    if (pos[q].valid) store_seg<B, T, SEG>(W + pos[q].base, pos[q].m, w[q]);
  }
  double tot[1];
  if (!grid_reduce<1, 0u>(acc, partials, &sc->ticket, tot)) return;
  // ---- last CTA, thread 0: Hessenberg column, Givens, convergence
  const int m = sc->m;
  double* Hc = sc->H + (size_t)jj * (kGmMax + 1);
  const double hn = sqrt(tot[0]);
  for (int i = 0; i <= jj; ++i) Hc[i] = sc->h1[i] + sc->h2[i];
  Hc[jj + 1] = hn;
  sc->hnext = hn;
  for (int i = 0; i < jj; ++i) {
    const double t = sc->cs[i] * Hc[i] + sc->sn[i] * Hc[i + 1];
    Hc[i + 1] = -sc->sn[i] * Hc[i] + sc->cs[i] * Hc[i + 1];
    Hc[i] = t;
  }
  const double den = hypot(Hc[jj], Hc[jj + 1]);
  const double c = (den > 0.0) ? Hc[jj] / den : 1.0;
  const double s = (den > 0.0) ? Hc[jj + 1] / den : 0.0;
  sc->cs[jj] = c;
  sc->sn[jj] = s;
  Hc[jj] = den;
  Hc[jj + 1] = 0.0;
  sc->gv[jj + 1] = -s * sc->gv[jj];
  sc->gv[jj] = c * sc->gv[jj];
  const double res = fabs(sc->gv[jj + 1]);
  sc->res = res;
  sc->iter += 1;
  const int jn = jj + 1;
  sc->j = jn;
  const bool conv = res <= sc->thresh;
  const bool bad = !isfinite(res) || !isfinite(den);
  const bool breakdown = (hn == 0.0);
  if (conv || bad || breakdown || jn >= m || sc->iter >= sc->max_iter) {
    // back substitution H(0:jn,0:jn) y = g(0:jn)
    for (int i = jn - 1; i >= 0; --i) {
      double v = sc->gv[i];
      for (int kk = i + 1; kk < jn; ++kk) v -= sc->H[(size_t)kk * (kGmMax + 1) + i] * sc->y[kk];
      const double d = sc->H[(size_t)i * (kGmMax + 1) + i];
      sc->y[i] = (d != 0.0) ? v / d : 0.0;
    }
    sc->jused = jn;
    sc->cycle_end = 1;
    if (bad) {
      sc->done = 1;
      sc->status = 5;
    } else if ((conv || breakdown) && !sc->verify) {
      sc->done = 1;
      sc->status = 0;
    } else if (conv || breakdown) {
      sc->conv_est = 1;  // the restart checks the true residual
    } else if (sc->iter >= sc->max_iter) {
      sc->done = 1;
      sc->status = 4;
    }
  }
}

// End of cycle: x += D^{-1} (V y) (right preconditioning).
template <typename S, typename B, typename T, int BS, int SEG>
__global__ void __launch_bounds__(kThreads) gm_update(HeatGeo g, const B* __restrict__ V, long long ldv,
                                                      const S* __restrict__ minv,
                                                      typename XOf<S>::type* __restrict__ x, GmScalars* sc) {
  using X = typename XOf<S>::type;
  if (!sc->cycle_end) return;
  const int ju = sc->jused;
  const int nbl = (g.n + BS - 1) / BS;
  RK_SEG_LOOP(g, SEG)
    (void)j;
    (void)k;
    T u[SEG], zv[SEG], xv[SEG];
#pragma unroll
    for (int e = 0; e < SEG; ++e) u[e] = T(0);
    for (int i = 0; i < ju; ++i) {
      const T yi = (T)sc->y[i];
      T vi[SEG];
      load_seg<T, B, SEG>(V + (long long)i * ldv + base, m, vi);
#pragma unroll
      for (int e = 0; e < SEG; ++e) u[e] = fma(yi, vi[e], u[e]);
    }
    bj_apply_blocks<T, S, BS, SEG>(minv, line, nbl, i0, u, zv);
    load_seg<T, X, SEG>(x + base, m, xv);
#pragma unroll
    for (int e = 0; e < SEG; ++e) xv[e] += zv[e];
    store_seg<X, T, SEG>(x + base, m, xv);
  RK_SEG_LOOP_END
}

}  // namespace rk

// Kernels of the advection-diffusion path: CSR operator (FP64 and storage
// precision), block-Jacobi with per-block inverses, and the start, restart and
// cycle-end update of the right-preconditioned restarted GMRES(m) (the
// Arnoldi step itself is in rk_gmres.cuh).  The Arnoldi/Hessenberg/Givens
// state lives on the device; the last CTA of each reduction updates it, so the
// host only polls a status word.
//
// Thread mapping of the vector kernels is the x-line segment mapping of the
// heat path (RK_SEG_LOOP): block-Jacobi blocks (x-line segments of BS nodes)
// lie inside one thread's segment.
#pragma once
#include "rk_device.cuh"
#include "rk_heat.cuh"
#include "rk_tiled.cuh"

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
  int steps;      // Arnoldi steps that did work (launch bookkeeping of the host)
  double beta;    // residual norm at the start of the cycle
  double bnorm;   // ||sigma g||
  double thresh;  // stopping threshold on the residual norm
  double tol_rel, tol_abs;
  double hnext;   // ||w|| of the last Arnoldi step before rotation
  double res;     // current residual estimate |g_{j+1}|
  double h1[kGmMax + 1], h2[kGmMax + 1];
  double H[(kGmMax + 1) * kGmMax];  // column-major (m+1) x m
  double cs[kGmMax], sn[kGmMax], gv[kGmMax + 1], y[kGmMax];
  // delayed reorthogonalization (see gm_dc_arnoldi)
  double Hraw[(kGmMax + 1) * kGmMax];  // unrotated Hessenberg, column-major (m+1) x m
  double sv[kGmMax];      // reorthogonalization coefficients s of the current step
  double cv[kGmMax + 1];  // coefficients c of u_{j+1} = w / nrm - V c
  double inv_nrm;         // 1 / ||v_j|| before normalisation
  unsigned ticket2;       // completion ticket of gm_dc_update
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
// The x-line-segment blocks of I - shift L.  One thread per block: the block
// of a 7-point operator restricted to an x-line segment is tridiagonal, and
// its Thomas factorisation is formed in FP64 (the blocks are diagonally
// dominant, so no pivoting is needed).
//   * flags == null (no adaptive precision): the slot of 3 BS storage
//     elements holds the factors -- multipliers l_i, inverse pivots 1/d_i and
//     ratios c_i -- and D^-1 r is applied by forward and back substitution
//     (3 values per row instead of the BS of a dense inverse row).
//   * flags != null (adaptive precision, tau > 0; the adaptive-precision
//     block-Jacobi of Ginkgo, Sec. 1): the inverse is formed column by column
//     and stored row-major, zero padded to BS x BS, in a slot of BS*BS storage
//     elements.  A block whose 1-norm condition number
//     kappa_1 = ||D||_1 ||D^-1||_1 satisfies kappa_1 * 2^-11 <= tau is stored
//     in FP16 in the first half of its slot and flagged (flags[b] = 1).
template <typename S, int BS>
__global__ void __launch_bounds__(kThreads) csr_bj_setup(CsrView A, const double* __restrict__ vals, int n,
                                                         double shift, S* __restrict__ minv, double tau,
                                                         unsigned char* __restrict__ flags) {
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
    if (!flags) {  // the factors; rows past m stay zero (their z is 0)
      S* f = minv + b * 3 * BS;
      for (int i = 0; i < BS; ++i) {
        f[i] = nar<S>(i < m && i > 0 ? lo[i] : 0.0);
        f[BS + i] = nar<S>(i < m ? 1.0 / den[i] : 0.0);
        f[2 * BS + i] = nar<S>(i < m ? cp[i] : 0.0);
      }
      continue;
    }
    double inv[BS][BS];
    double ninv = 0.0, nblk = 0.0;  // 1-norms of the inverse and of the block
    for (int jcol = 0; jcol < BS; ++jcol) {
      double xcol[BS];
      if (jcol < m) {
        double dp[BS];
        for (int i = 0; i < m; ++i) {
          const double rhs = (i == jcol) ? 1.0 : 0.0;
          dp[i] = (rhs - (i > 0 ? lo[i] * dp[i - 1] : 0.0)) / den[i];
        }
        double cs = 0.0;
        for (int i = m - 1; i >= 0; --i) {
          xcol[i] = dp[i] - (i + 1 < m ? cp[i] * xcol[i + 1] : 0.0);
          cs += fabs(xcol[i]);
        }
        ninv = fmax(ninv, cs);
        // column jcol of the block: up[jcol-1], di[jcol], lo[jcol+1]
        const double bc = fabs(di[jcol]) + (jcol > 0 ? fabs(up[jcol - 1]) : 0.0) +
                          (jcol + 1 < m ? fabs(lo[jcol + 1]) : 0.0);
        nblk = fmax(nblk, bc);
      }
      for (int i = 0; i < BS; ++i) inv[i][jcol] = (i < m && jcol < m) ? xcol[i] : 0.0;
    }
    const bool low = tau > 0.0 && nblk * ninv * 0x1p-11 <= tau;
    S* out = minv + b * BS * BS;
    if (low) {
      __half* oh = reinterpret_cast<__half*>(out);
      for (int i = 0; i < BS; ++i)
        for (int jcol = 0; jcol < BS; ++jcol) oh[i * BS + jcol] = __double2half(inv[i][jcol]);
    } else {
      for (int i = 0; i < BS; ++i)
        for (int jcol = 0; jcol < BS; ++jcol) out[i * BS + jcol] = nar<S>(inv[i][jcol]);
    }
    if (flags) flags[b] = low ? 1 : 0;
  }
}

// z = D^{-1} r for the blocks of one segment: by the Thomas factors when
// flags is null, else by the per-block inverses (in S, or in FP16 where flags
// marks the block); see csr_bj_setup.
template <typename T, typename S, int BS, int SEG>
__device__ __forceinline__ void bj_apply_blocks(const S* __restrict__ minv, const unsigned char* __restrict__ flags,
                                                long long line, int nbl, int i0, const T (&r)[SEG], T (&z)[SEG]) {
#pragma unroll
  for (int cb = 0; cb < SEG / BS; ++cb) {
    const int bi = i0 / BS + cb;
    if (bi >= nbl) {
#pragma unroll
      for (int i = 0; i < BS; ++i) z[cb * BS + i] = T(0);
      continue;
    }
    const long long blk = line * nbl + bi;
    if (flags == nullptr) {
      const S* F = minv + blk * (long long)(3 * BS);
      T lf[BS], iv[BS], cf[BS], dp[BS];
      load_seg<T, S, BS>(F, BS, lf);
      load_seg<T, S, BS>(F + BS, BS, iv);
      load_seg<T, S, BS>(F + 2 * BS, BS, cf);
      dp[0] = r[cb * BS] * iv[0];
#pragma unroll
      for (int i = 1; i < BS; ++i) dp[i] = fma(-lf[i], dp[i - 1], r[cb * BS + i]) * iv[i];
      z[cb * BS + BS - 1] = dp[BS - 1];
#pragma unroll
      for (int i = BS - 2; i >= 0; --i) z[cb * BS + i] = fma(-cf[i], z[cb * BS + i + 1], dp[i]);
      continue;
    }
    const S* M = minv + blk * (long long)(BS * BS);
    const bool half_block = flags != nullptr && flags[blk] != 0;
#pragma unroll
    for (int i = 0; i < BS; ++i) {
      T row[BS];
      if (half_block)
        load_seg<T, __half, BS>(reinterpret_cast<const __half*>(M) + i * BS, BS, row);
      else
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
                                                               const unsigned char* __restrict__ flags,
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
    bj_apply_blocks<T, S, BS, SEG>(minv, flags, line, nbl, i0, rv, zv);
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

// End of cycle: x += D^{-1} (V y) (right preconditioning).
template <typename S, typename B, typename T, int BS, int SEG>
__global__ void __launch_bounds__(kThreads) gm_update(HeatGeo g, const B* __restrict__ V, long long ldv,
                                                      const S* __restrict__ minv,
                                                      const unsigned char* __restrict__ flags,
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
    bj_apply_blocks<T, S, BS, SEG>(minv, flags, line, nbl, i0, u, zv);
    load_seg<T, X, SEG>(x + base, m, xv);
#pragma unroll
    for (int e = 0; e < SEG; ++e) xv[e] += zv[e];
    store_seg<X, T, SEG>(x + base, m, xv);
  RK_SEG_LOOP_END
}

}  // namespace rk

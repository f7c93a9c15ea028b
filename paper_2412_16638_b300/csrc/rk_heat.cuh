// Kernels of the constant-coefficient heat path (7-point stencil applied
// matrix-free) and the FP64 stage operations on it.
//
// Thread mapping: one thread owns a segment of SEG consecutive x-nodes of one
// x-line (the last segment of a line may be shorter); block-Jacobi blocks are
// x-line segments of BS <= SEG nodes, so every block lies inside one thread's
// segment and z = D^{-1} r is computed in registers.  Neighbours in y and z
// are read from global memory (they are L1/L2 hits: adjacent lines are
// processed by adjacent threads, adjacent planes by CTAs in flight together).
#pragma once
#include "rk_device.cuh"

namespace rk {

struct HeatGeo {
  int n;          // nodes per direction
  int nseg;       // segments per x-line = ceil(n / SEG)
  long long n2;   // n*n
  long long N;    // n^3
};

// Device-resident state of one CG solve.  Written by the last CTA of each
// sweep, read by the next sweep, so no host round trip per iteration.
struct CgScalars {
  double rz;       // r . z of the current residual
  double pAp;      // p . A p
  double rr;       // ||r||^2 (scaled right-hand side units)
  double gg;       // ||g||^2
  double alpha, beta;
  double thresh2;  // squared stopping threshold
  double tol_rel, tol_abs;
  int iter, max_iter;
  int done;        // 1: stop launching sweeps
  int status;      // 0 converged / running, 4 not converged, 5 non-finite/breakdown
  unsigned ticket;
  int warm;        // 1: the solve started from a nonzero x (x is read at iteration 0)
  unsigned wait_spins;  // non-blocking polls of each TMA wait in the sweeps' main
                        // loops (0 = the default bound of kWaitSpins try_wait polls)
};

// Per-solve right-hand-side statistics written by heat_apply_f64 / vec_norms.
struct RhsScalars {
  double gg;     // ||g||_2^2 of the FP64 right-hand side
  double gmax;   // ||g||_inf (the FP64 operators reduce it only when want_scale)
  double sigma;  // storage scale (1/||g||_inf for FP16, else 1)
  double res2;   // ||true residual||^2 from the FP64 correction
  unsigned ticket;
  int want_scale;   // FP16 storage: sigma = 1 / ||g||_inf
  int want_range;   // FP32/BF16 storage: a power-of-two sigma when ||g|| leaves [2^-40, 2^40]
};

// Storage scale sigma of a stage right-hand side g (the solve runs on sigma g).
// FP16 storage: 1 / ||g||_inf, for its narrow range (Sec. 2.3).  FP32 and BF16
// storage: 1 while the RMS of g lies in [2^-40, 2^40], else the power of two
// that brings it near 1.  Scaling by a power of two is exact, so results in
// the normal range are unchanged; it keeps the low-precision products of a
// decayed solution (|g| ~ 1e-20 after many steps of a stiff problem) clear of
// underflow, where r.z and p.Ap would otherwise round to zero and break CG.
// FP64 storage: 1.
__host__ __device__ inline double rhs_scale(const RhsScalars* rs, double gg, double gmax, long long N) {
  if (rs->want_scale) return (gmax > 0.0 && isfinite(gmax)) ? 1.0 / gmax : 1.0;
  if (!rs->want_range || !(gg > 0.0) || !isfinite(gg) || N < 1) return 1.0;
  const double rms = sqrt(gg / (double)N);
  if (rms >= 0x1p-40 && rms <= 0x1p40) return 1.0;
  return ldexp(1.0, -ilogb(rms));
}

// Sum of the six neighbours of every element of a segment (zero outside the
// grid).  own[] holds the field on the segment (zeros past m); seg(off, m, v)
// loads the field on the segment that starts at element index off; pt(idx)
// loads one value.
template <typename T, int SEG, typename SegF, typename PtF>
__device__ __forceinline__ void nb_sum(const HeatGeo& g, int i0, int m, int j, int k, long long base,
                                       const T (&own)[SEG], SegF seg, PtF pt, T (&nb)[SEG]) {
  const T left = (i0 > 0) ? pt(base - 1) : T(0);
  const T right = (i0 + SEG < g.n) ? pt(base + SEG) : T(0);
#pragma unroll
  for (int e = 0; e < SEG; ++e) {
    T l = (e > 0) ? own[e - 1] : left;
    T r = (e + 1 < SEG) ? own[e + 1] : right;
    nb[e] = l + r;
  }
  T tmp[SEG];
  if (j > 0) {
    seg(base - g.n, m, tmp);
#pragma unroll
    for (int e = 0; e < SEG; ++e) nb[e] += tmp[e];
  }
  if (j < g.n - 1) {
    seg(base + g.n, m, tmp);
#pragma unroll
    for (int e = 0; e < SEG; ++e) nb[e] += tmp[e];
  }
  if (k > 0) {
    seg(base - g.n2, m, tmp);
#pragma unroll
    for (int e = 0; e < SEG; ++e) nb[e] += tmp[e];
  }
  if (k < g.n - 1) {
    seg(base + g.n2, m, tmp);
#pragma unroll
    for (int e = 0; e < SEG; ++e) nb[e] += tmp[e];
  }
}

#define RK_SEG_LOOP(g, SEG)                                                            \
  const long long nsegs_ = (long long)(g).n2 * (g).nseg;                               \
  for (long long t_ = (long long)blockIdx.x * blockDim.x + threadIdx.x; t_ < nsegs_;   \
       t_ += (long long)gridDim.x * blockDim.x) {                                      \
    const long long line = t_ / (g).nseg;                                              \
    const int sidx = (int)(t_ - line * (g).nseg);                                      \
    const int i0 = sidx * (SEG);                                                       \
    const int m = min((SEG), (g).n - i0);                                              \
    const int j = (int)(line % (g).n);                                                 \
    const int k = (int)(line / (g).n);                                                 \
    const long long base = line * (g).n + i0;

#define RK_SEG_LOOP_END }

// ------------------------------------------------------------- FP64 operator
// y = d*x + o*(sum of neighbours of x) + f in FP64 (L: d = -6c, o = c with
// c = kappa/h^2; f the optional forcing, nullptr = none, at no extra FP64
// operation).  If rs != null, also ||y||^2, ||y||_inf and the storage scale
// are reduced into *rs (the stage right-hand side g = L r_i + f).
template <int SEG>
__global__ void __launch_bounds__(kThreads) heat_apply_f64(HeatGeo g, const double* __restrict__ x,
                                                           const double* __restrict__ f, double* __restrict__ y,
                                                           double d, double o, RhsScalars* rs, double* partials) {
  double acc[2] = {0.0, 0.0};
  // the max norm only sets the FP16 storage scale: skip its FP64 op otherwise
  const bool wmax = rs != nullptr && rs->want_scale;
  RK_SEG_LOOP(g, SEG)
    double xv[SEG], nb[SEG];
    load_seg<double, double, SEG>(x + base, m, xv);
    nb_sum<double, SEG>(
        g, i0, m, j, k, base, xv,
        [&](long long off, int mm, double (&v)[SEG]) { load_seg<double, double, SEG>(x + off, mm, v); },
        [&](long long idx) { return x[idx]; }, nb);
    double yv[SEG], fv[SEG];
    if (f) {
      load_seg<double, double, SEG>(f + base, m, fv);
    } else {
#pragma unroll
      for (int e = 0; e < SEG; ++e) fv[e] = 0.0;
    }
#pragma unroll
    for (int e = 0; e < SEG; ++e) {
      yv[e] = fma(d, xv[e], fma(o, nb[e], fv[e]));
      if (e < m) {
        acc[0] = fma(yv[e], yv[e], acc[0]);
        if (wmax) acc[1] = fmax(acc[1], fabs(yv[e]));
      }
    }
    store_seg<double, double, SEG>(y + base, m, yv);
  RK_SEG_LOOP_END
  if (rs == nullptr) return;
  double tot[2];
  if (grid_reduce<2, 2u>(acc, partials, &rs->ticket, tot)) {
    rs->gg = tot[0];
    rs->gmax = tot[1];
    rs->sigma = rhs_scale(rs, tot[0], tot[1], g.N);
  }
}

// ------------------------------------------------------ FP64 explicit correction
// k = g + c_s * (sum of neighbours of v - 6 v),  v = ke / sigma widened to FP64,
// c_s = shift * kappa/h^2.  This is k_i = L y_i with y_i = r_i + shift k^eps_i
// (g = L r_i precomputed), and k - v is the true residual of the stage solve;
// its squared norm is reduced into rs->res2.
// Error-free transformations on the FP32 pipe: a + b = s + e exactly (Knuth's
// TwoSum), and c*a = p + e exactly (product error through one FMA).
// (The _rn intrinsics keep the compiler from contracting these into FMAs,
// which would break the exactness.)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Laplacian numerator (sum of the six neighbours - 6 * centre) of FP32 values
// as an unevaluated float pair hi + lo: every rounding error of the sum is
// captured exactly and accumulated in lo, so hi + lo carries the sum to about
// 2^-48 of the terms' magnitude (the FP64 stencil carries about 2^-53); one
// conversion to FP64 then replaces seven.
__device__ __forceinline__ double lap_pair(float c, float xl, float xr, float ym, float yp, float zm, float zp) {
  float s, e, t;
  const float p6 = __fmul_rn(-6.0f, c);
  float lo = fmaf(-6.0f, c, -p6);  // exact error of the product
  two_sum(p6, xl, s, e);
  lo = __fadd_rn(lo, e);
  two_sum(s, xr, t, e);
  lo = __fadd_rn(lo, e);
  two_sum(t, ym, s, e);
  lo = __fadd_rn(lo, e);
  two_sum(s, yp, t, e);
  lo = __fadd_rn(lo, e);
  two_sum(t, zm, s, e);
  lo = __fadd_rn(lo, e);
  two_sum(s, zp, t, e);
  lo = __fadd_rn(lo, e);
  return (double)t + (double)lo;
}

template <typename S, int SEG>
__global__ void __launch_bounds__(kThreads) heat_correct_f64(HeatGeo g, const double* __restrict__ gv,
                                                             const S* __restrict__ ke, double cs,
                                                             double* __restrict__ kout, RhsScalars* rs,
                                                             double* partials) {
  const double inv_sigma = 1.0 / rs->sigma;
  double acc[1] = {0.0};
  if constexpr (sizeof(S) == 4) {
    // FP32 k^eps: exact-pair Laplacian on the FP32 pipe (see lap_pair)
    const double c2 = cs * inv_sigma;
    RK_SEG_LOOP(g, SEG)
      float v[SEG], nb_unused[SEG];
      (void)nb_unused;
      load_seg<float, S, SEG>(ke + base, m, v);
      const float left = (i0 > 0) ? wid<float>(ke[base - 1]) : 0.f;
      const float right = (i0 + SEG < g.n) ? wid<float>(ke[base + SEG]) : 0.f;
      float ym[SEG], yp[SEG], zm[SEG], zp[SEG];
      auto seg_or_zero = [&](bool in, long long off, float (&w)[SEG]) {
        if (in) {
          load_seg<float, S, SEG>(ke + off, m, w);
        } else {
#pragma unroll
          for (int e = 0; e < SEG; ++e) w[e] = 0.f;
        }
      };
      seg_or_zero(j > 0, base - g.n, ym);
      seg_or_zero(j < g.n - 1, base + g.n, yp);
      seg_or_zero(k > 0, base - g.n2, zm);
      seg_or_zero(k < g.n - 1, base + g.n2, zp);
      double gs[SEG], kv[SEG];
      load_seg<double, double, SEG>(gv + base, m, gs);
#pragma unroll
      for (int e = 0; e < SEG; ++e) {
        const float xl = (e > 0) ? v[e - 1] : left;
        const float xr = (e + 1 < SEG) ? v[e + 1] : right;
        const double lap = lap_pair(v[e], xl, xr, ym[e], yp[e], zm[e], zp[e]);
        kv[e] = fma(c2, lap, gs[e]);
        const double res = fma(-(double)v[e], inv_sigma, kv[e]);
        if (e < m) acc[0] = fma(res, res, acc[0]);
      }
      store_seg<double, double, SEG>(kout + base, m, kv);
    RK_SEG_LOOP_END
    double tot[1];
    if (grid_reduce<1, 0u>(acc, partials, &rs->ticket, tot)) rs->res2 = tot[0];
    return;
  }
  RK_SEG_LOOP(g, SEG)
    double v[SEG], nb[SEG], gs[SEG];
    load_seg<double, S, SEG>(ke + base, m, v);
    nb_sum<double, SEG>(
        g, i0, m, j, k, base, v,
        [&](long long off, int mm, double (&w)[SEG]) { load_seg<double, S, SEG>(ke + off, mm, w); },
        [&](long long idx) { return wid<double>(ke[idx]); }, nb);
    load_seg<double, double, SEG>(gv + base, m, gs);
    double kv[SEG];
#pragma unroll
    for (int e = 0; e < SEG; ++e) {
      const double lap = fma(-6.0, v[e], nb[e]);
      kv[e] = fma(cs * inv_sigma, lap, gs[e]);
      const double res = kv[e] - v[e] * inv_sigma;
      if (e < m) acc[0] = fma(res, res, acc[0]);
    }
    store_seg<double, double, SEG>(kout + base, m, kv);
  RK_SEG_LOOP_END
  double tot[1];
  if (grid_reduce<1, 0u>(acc, partials, &rs->ticket, tot)) rs->res2 = tot[0];
}

// ------------------------------------------------------------- CG sweeps
// Block-Jacobi inverse passed by value as a __grid_constant__ kernel
// parameter: [0] the full BS-block, [1] the tail block of a line (n mod BS
// nodes, zero padded).  Indexed with compile-time offsets inside the unrolled
// GEMV, its entries are read from the constant bank as FMA operands, so the
// preconditioner costs no load instructions.
template <typename T, int BS>
struct BjInv {
  T m[2 * BS * BS];
};

// The same block inverse in factored form: the x-line block of I - shift L is
// the constant tridiagonal matrix tridiag(o, d, o) (d = 1 + 6 shift c,
// o = -shift c), whose LU factors have pivots p_1 = d, p_i = d - o^2/p_{i-1}.
// With ip_i = 1/p_i, mo = -o and nu_i = -o ip_i, the solve is
//   y_1 = ip_1 r_1,  y_i = ip_i (r_i + mo y_{i-1}),  z_BS = y_BS,
//   z_i = y_i + nu_i z_{i+1}
// (3 FP32 operations per element instead of BS for the dense inverse); the
// factors are formed in FP64 and rounded.  Full blocks only (the callers'
// segments hold whole blocks).  The blocks are diagonally dominant, so the
// recurrences are stable.
template <typename T, int BS>
struct BjTri {
  T ip[BS];
  T nu[BS];
  T mo;
};

template <typename T, int BS, int SEG>
__device__ __forceinline__ void bj_apply_tri(const BjTri<T, BS>& t, const T (&r)[SEG], T (&z)[SEG]) {
  static_assert(SEG % BS == 0, "segments hold whole blocks");
#pragma unroll
  for (int cb = 0; cb < SEG / BS; ++cb) {
    T y[BS];
    y[0] = t.ip[0] * r[cb * BS];
#pragma unroll
    for (int i = 1; i < BS; ++i) y[i] = t.ip[i] * fma(t.mo, y[i - 1], r[cb * BS + i]);
    z[cb * BS + BS - 1] = y[BS - 1];
#pragma unroll
    for (int i = BS - 2; i >= 0; --i) z[cb * BS + i] = fma(t.nu[i], z[cb * BS + i + 1], y[i]);
  }
}

// z = D^{-1} r on every block of the segment.
template <typename T, int BS, int SEG>
__device__ __forceinline__ void bj_apply(const T* sM, int n, int i0, const T (&r)[SEG], T (&z)[SEG]) {
#pragma unroll
  for (int cb = 0; cb < SEG / BS; ++cb) {
    const bool tail = (i0 + (cb + 1) * BS > n);
    const T* M = sM + (tail ? BS * BS : 0);
#pragma unroll
    for (int i = 0; i < BS; ++i) {
      T a = T(0);
#pragma unroll
      for (int jj = 0; jj < BS; ++jj) a = fma(M[i * BS + jj], r[cb * BS + jj], a);
      z[cb * BS + i] = a;
    }
  }
}

// Initialise from a nonzero guess x (the previous solve of the same stage,
// storage with sigma = 1): r = g - (I - shift L) x (rounded to S),
// z = D^{-1} r, and the first reductions r.z, r.r; the stopping threshold
// stays relative to ||g|| (FP64, from the right-hand side's reduction).
template <typename S, typename T, int BS, int SEG>
__global__ void __launch_bounds__(kThreads) cg_init_warm(HeatGeo g, const double* __restrict__ gv,
                                                         const RhsScalars* rs, T d, T o,
                                                         const __grid_constant__ BjInv<T, BS> inv,
                                                         S* __restrict__ r, S* __restrict__ z,
                                                         const typename XOf<S>::type* __restrict__ x, CgScalars* sc,
                                                         double* partials) {
  using X = typename XOf<S>::type;
  const T* sM = inv.m;
  T rz = T(0), rr = T(0);
  RK_SEG_LOOP(g, SEG)
    T xv[SEG], nb[SEG];
    load_seg<T, X, SEG>(x + base, m, xv);
    nb_sum<T, SEG>(
        g, i0, m, j, k, base, xv, [&](long long off, int mm, T (&v)[SEG]) { load_seg<T, X, SEG>(x + off, mm, v); },
        [&](long long idx) { return wid<T>(x[idx]); }, nb);
    double gd[SEG];
    load_seg<double, double, SEG>(gv + base, m, gd);
    T rv[SEG], zv[SEG];
#pragma unroll
    for (int e = 0; e < SEG; ++e) rv[e] = (e < m) ? rnd<S, T>((T)gd[e] - fma(d, xv[e], o * nb[e])) : T(0);
    bj_apply<T, BS, SEG>(sM, g.n, i0, rv, zv);
#pragma unroll
    for (int e = 0; e < SEG; ++e) {
      zv[e] = rnd<S, T>(zv[e]);
      if (e < m) {
        rz = fma(rv[e], zv[e], rz);
        rr = fma(rv[e], rv[e], rr);
      }
    }
    store_seg<S, T, SEG>(r + base, m, rv);
    store_seg<S, T, SEG>(z + base, m, zv);
  RK_SEG_LOOP_END
  double acc[2] = {(double)rz, (double)rr};
  double tot[2];
  if (grid_reduce<2, 0u>(acc, partials, &sc->ticket, tot)) {
    sc->rz = tot[0];
    sc->rr = tot[1];
    sc->gg = rs->gg;
    const double ta = sc->tol_abs;
    sc->thresh2 = fmax(sc->tol_rel * sc->tol_rel * rs->gg, ta * ta);
    sc->iter = 0;
    sc->beta = 0.0;
    sc->warm = 1;
    sc->done = 0;
    sc->status = 0;
    if (!isfinite(tot[0]) || !isfinite(tot[1])) {
      sc->done = 1;
      sc->status = 5;
    } else if (tot[1] <= sc->thresh2) {
      sc->done = 1;  // the guess already meets the tolerance
    }
  }
}

// Initialise: r = sigma*g (rounded to S), z = D^{-1} r, x = 0, and the first
// reductions r.z, r.r.  g is the FP64 right-hand side.  store_zx = 0 leaves z
// and x unwritten, for callers whose first sweeps do not read them (the tiled
// sweeps recompute z from r, the fast-diagonalization passes write z, and the
// first sweep B starts x from zero without reading it).
template <typename S, typename T, int BS, int SEG>
__global__ void __launch_bounds__(kThreads) cg_init(HeatGeo g, const double* __restrict__ gv,
                                                    const RhsScalars* rs, const __grid_constant__ BjInv<T, BS> inv,
                                                    S* __restrict__ r, S* __restrict__ z,
                                                    typename XOf<S>::type* __restrict__ x, CgScalars* sc,
                                                    double* partials, int store_zx = 1) {
  using X = typename XOf<S>::type;
  const T* sM = inv.m;
  const double sigma = rs->sigma;
  T rz = T(0), rr = T(0);  // per-thread partials in the arithmetic type
  RK_SEG_LOOP(g, SEG)
    double gd[SEG];
    load_seg<double, double, SEG>(gv + base, m, gd);
    T rv[SEG], zv[SEG], zero[SEG];
    if (sigma == 1.0) {  // unscaled storage: no FP64 multiply (same values)
#pragma unroll
      for (int e = 0; e < SEG; ++e) rv[e] = (e < m) ? rnd<S, T>((T)gd[e]) : T(0);
    } else {
#pragma unroll
      for (int e = 0; e < SEG; ++e) rv[e] = (e < m) ? rnd<S, T>((T)(gd[e] * sigma)) : T(0);
    }
#pragma unroll
    for (int e = 0; e < SEG; ++e) zero[e] = T(0);
    bj_apply<T, BS, SEG>(sM, g.n, i0, rv, zv);
#pragma unroll
    for (int e = 0; e < SEG; ++e) {
      zv[e] = rnd<S, T>(zv[e]);
      if (e < m) {
        rz = fma(rv[e], zv[e], rz);
        rr = fma(rv[e], rv[e], rr);
      }
    }
    store_seg<S, T, SEG>(r + base, m, rv);
    if (store_zx) {
      store_seg<S, T, SEG>(z + base, m, zv);
      store_seg<X, T, SEG>(x + base, m, zero);
    }
  RK_SEG_LOOP_END
  double acc[2] = {(double)rz, (double)rr};
  double tot[2];
  if (grid_reduce<2, 0u>(acc, partials, &sc->ticket, tot)) {
    sc->rz = tot[0];
    sc->rr = tot[1];
    sc->gg = tot[1];
    const double ta = sc->tol_abs * sigma;
    sc->thresh2 = fmax(sc->tol_rel * sc->tol_rel * tot[1], ta * ta);
    sc->iter = 0;
    sc->beta = 0.0;
    sc->alpha = 0.0;
    sc->pAp = 0.0;
    if (!isfinite(tot[0]) || !isfinite(tot[1])) {
      sc->done = 1;
      sc->status = 5;
    } else if (tot[1] <= sc->thresh2 || tot[1] == 0.0) {
      sc->done = 1;
      sc->status = 0;
    } else {
      sc->done = 0;
      sc->status = 0;
    }
  }
}

// Sweep A: p = z + beta*p_old (rounded to S), w = A p with A = d I + o*(neighbour
// sum), partial p.w.  Writes p to pnew (ping-pong buffer).  Last CTA: alpha.
template <typename S, typename T, int SEG>
__global__ void __launch_bounds__(kThreads, 4) cg_sweep_a(HeatGeo g, T d, T o, const S* __restrict__ z,
                                                       const S* __restrict__ pold, S* __restrict__ pnew,
                                                       CgScalars* sc, double* partials) {
  if (sc->done) return;
  const T beta = (T)sc->beta;
  const bool first = (sc->iter == 0);
  T pw_t = T(0);  // per-thread partial in the arithmetic type
  RK_SEG_LOOP(g, SEG)
    auto pseg = [&](long long off, int mm, T (&v)[SEG]) {
      load_seg<T, S, SEG>(z + off, mm, v);
      if (!first) {
        T q[SEG];
        load_seg<T, S, SEG>(pold + off, mm, q);
#pragma unroll
        for (int e = 0; e < SEG; ++e) v[e] = rnd<S, T>(fma(beta, q[e], v[e]));
      }
    };
    auto ppt = [&](long long idx) {
      T v = wid<T>(z[idx]);
      if (!first) v = rnd<S, T>(fma(beta, wid<T>(pold[idx]), v));
      return v;
    };
    T p[SEG], nb[SEG];
    pseg(base, m, p);
    nb_sum<T, SEG>(g, i0, m, j, k, base, p, pseg, ppt, nb);
#pragma unroll
    for (int e = 0; e < SEG; ++e) {
      const T w = fma(d, p[e], o * nb[e]);
      if (e < m) pw_t = fma(p[e], w, pw_t);
    }
    store_seg<S, T, SEG>(pnew + base, m, p);
  RK_SEG_LOOP_END
  double acc[1] = {(double)pw_t};
  double tot[1];
  if (grid_reduce<1, 0u>(acc, partials, &sc->ticket, tot)) {
    sc->pAp = tot[0];
    const double alpha = sc->rz / tot[0];
    sc->alpha = alpha;
    if (!isfinite(tot[0]) || !isfinite(sc->rz)) {
      sc->done = 1;
      sc->status = 5;
    } else if (!(tot[0] > 0.0) || !isfinite(alpha)) {
      // p.Ap <= 0 for an SPD operator: rounding has reached the attainable
      // accuracy; stop with the current iterate (valid, not converged)
      sc->done = 1;
      sc->status = 4;
    }
  }
}

// Sweep B: recompute w = A p, x += alpha p, r -= alpha w, z = D^{-1} r,
// partials r.z and r.r.  Last CTA: beta, convergence test, iteration count.
template <typename S, typename T, int BS, int SEG>
__global__ void __launch_bounds__(kThreads, 4) cg_sweep_b(HeatGeo g, T d, T o, const S* __restrict__ p,
                                                       typename XOf<S>::type* __restrict__ x, S* __restrict__ r,
                                                       S* __restrict__ z, const __grid_constant__ BjInv<T, BS> inv,
                                                       CgScalars* sc, double* partials) {
  using X = typename XOf<S>::type;
  if (sc->done) return;
  const T* sM = inv.m;
  const T alpha = (T)sc->alpha;
  const bool xzero = (sc->iter == 0) && !sc->warm;
  T rz = T(0), rr = T(0);  // per-thread partials in the arithmetic type
  RK_SEG_LOOP(g, SEG)
    T pv[SEG], nb[SEG];
    load_seg<T, S, SEG>(p + base, m, pv);
    nb_sum<T, SEG>(
        g, i0, m, j, k, base, pv, [&](long long off, int mm, T (&v)[SEG]) { load_seg<T, S, SEG>(p + off, mm, v); },
        [&](long long idx) { return wid<T>(p[idx]); }, nb);
    T rv[SEG], xv[SEG], zv[SEG];
    load_seg<T, S, SEG>(r + base, m, rv);
    if (!xzero) {
      load_seg<T, X, SEG>(x + base, m, xv);
    } else {
#pragma unroll
      for (int e = 0; e < SEG; ++e) xv[e] = T(0);
    }
#pragma unroll
    for (int e = 0; e < SEG; ++e) {
      const T w = fma(d, pv[e], o * nb[e]);
      rv[e] = (e < m) ? rnd<S, T>(fma(-alpha, w, rv[e])) : T(0);
      xv[e] = fma(alpha, pv[e], xv[e]);
    }
    bj_apply<T, BS, SEG>(sM, g.n, i0, rv, zv);
#pragma unroll
    for (int e = 0; e < SEG; ++e) {
      zv[e] = rnd<S, T>(zv[e]);
      if (e < m) {
        rz = fma(rv[e], zv[e], rz);
        rr = fma(rv[e], rv[e], rr);
      }
    }
    store_seg<X, T, SEG>(x + base, m, xv);
    store_seg<S, T, SEG>(r + base, m, rv);
    store_seg<S, T, SEG>(z + base, m, zv);
  RK_SEG_LOOP_END
  double acc[2] = {(double)rz, (double)rr};
  double tot[2];
  if (grid_reduce<2, 0u>(acc, partials, &sc->ticket, tot)) {
    const double rz_new = tot[0];
    sc->beta = rz_new / sc->rz;
    sc->rz = rz_new;
    sc->rr = tot[1];
    sc->iter += 1;
    if (!isfinite(tot[0]) || !isfinite(tot[1])) {
      sc->done = 1;
      sc->status = 5;
    } else if (tot[1] <= sc->thresh2) {
      sc->done = 1;
      sc->status = 0;
    } else if (sc->iter >= sc->max_iter) {
      sc->done = 1;
      sc->status = 4;
    }
  }
}

// Standalone block-Jacobi apply on an FP64 vector: z = D^{-1} round_S(r),
// returned widened to FP64 (for testing the preconditioner).
template <typename S, typename T, int BS, int SEG>
__global__ void __launch_bounds__(kThreads) bj_apply_f64io(HeatGeo g, const double* __restrict__ r,
                                                           const __grid_constant__ BjInv<T, BS> inv,
                                                           double* __restrict__ z) {
  const T* sM = inv.m;
  RK_SEG_LOOP(g, SEG)
    double rd[SEG];
    load_seg<double, double, SEG>(r + base, m, rd);
    T rv[SEG], zv[SEG];
#pragma unroll
    for (int e = 0; e < SEG; ++e) rv[e] = (e < m) ? rnd<S, T>((T)rd[e]) : T(0);
    bj_apply<T, BS, SEG>(sM, g.n, i0, rv, zv);
    double zd[SEG];
#pragma unroll
    for (int e = 0; e < SEG; ++e) zd[e] = (double)rnd<S, T>(zv[e]);
    store_seg<double, double, SEG>(z + base, m, zd);
  RK_SEG_LOOP_END
}

}  // namespace rk

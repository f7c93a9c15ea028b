// Batched stepping of many independent heat problems: every phase of the
// stage loop -- stage right-hand side, FP64 operator, CG start, the two CG
// sweeps, FP64 correction, update -- is one launch over a work list of
// (problem, tile) items covering every problem of the batch, so a large
// problem spreads over many CTAs and small ones share the GPU.  A tile is
// kThreads consecutive x-line segments of one problem, one segment per
// thread.  Reductions are per problem: each item writes its CTA's partial,
// and the CTA that takes the problem's last ticket sums the partials in item
// order (deterministic, and independent of the other problems in the batch)
// and updates that problem's solver scalars.  Problems whose solve has
// finished skip their items; a device counter of the problems still
// iterating tells the host when a stage's CG is done.
#pragma once
#include "../../include/rk.h"
#include "rk_device.cuh"
#include "rk_heat.cuh"
#include "rk_vec.cuh"

namespace rk {

constexpr int kBatchStages = 8;

// Per-problem batch descriptor (device memory).  Storage S, arithmetic T and
// block size BS are those of the batch group; the geometry uses the group's
// segment length.
template <typename T, int BS>
struct BatchProb {
  HeatGeo g;              // segments of the group's length
  double c;               // kappa / h^2
  double* u;
  double* r;
  double* g64;
  double* k[kBatchStages];
  void* ke[kBatchStages];  // solution type X (FP32 for 16-bit storage)
  void* wr;
  void* wz;
  void* wp[2];
  CgScalars* sc;           // the problem's CG scalars
  RhsScalars* rs;          // the problem's per-stage right-hand-side scalars [0..7]
  double* part;            // per-item partials, nitems x 2
  unsigned* ticket;        // per-problem reduction ticket
  int nitems;              // items (kBatchTilesPerItem tiles) of this problem
  int ld;                  // line pitch of the Krylov vectors and k^eps (elements; >= n)
  int full;                // 1: ld is a multiple of the segment, so Krylov segments are
                           // read and written whole (the padding holds zeros)
  int plane;               // n * ld (n <= 1024, so padded indices fit in int)
  int max_iter;            // CG settings of the problem
  double tol_rel, tol_abs;
  T d[kBatchStages], o[kBatchStages];   // stage matrix I - shift L = d I + o (neighbour sum)
  BjTri<T, BS> tri[kBatchStages];       // factored x-line block of each implicit stage
  // statistics accumulated over the steps of one call
  long long iters_total;
  int iters_max, solves, not_converged, status;
  double true_res_max;
};

// A work item: nch consecutive tiles of one problem (one reduction per item).
struct BatchItem {
  int prob;   // problem index
  int chunk;  // first tile
  int nch;    // tiles
  int idx;    // item index within the problem (slot of its partial sums)
};
constexpr int kBatchTilesPerItem = 4;

// Stage coefficients shared by the group (one tableau, one step size).
struct BatchStage {
  int stage;              // stage index i
  int nh, ne;             // history terms in FP64 (k_j) and in low precision (k^eps_j)
  int hj[kBatchStages];   // stages of the k_j terms
  double ch[kBatchStages];
  int ej[kBatchStages];   // stages of the k^eps_j terms
  double ce[kBatchStages];
  double shift_a;         // dt * a_ii (0 for an explicit stage)
  int correct;            // 1: FP64 correction k = L y; 0: k = widened solve output
  int use_r;              // 1: r was formed (history terms present), else r = u
};

// Per-problem reduction of NV sums (NV <= 2): the item's CTA sum (in the
// arithmetic type A, FP32 for FP32 work: FP64 operations are scarce on this
// part) goes to part[chunk * 2 + c] in FP64; the CTA that takes the problem's
// last ticket adds the items' partials in item order and returns true in
// thread 0 with the totals.  MAXMASK bit c: maximum instead of sum.
template <typename A, int NV, unsigned MAXMASK = 0u>
__device__ __forceinline__ bool prob_reduce(A (&v)[NV], double* part, unsigned* ticket, int chunk, int nitems,
                                            double (&tot)[NV]) {
  __shared__ A sred[32 * 2];
  __shared__ int am_last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int c = 0; c < NV; ++c)
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const A o = __shfl_down_sync(0xffffffffu, v[c], off);
      v[c] = ((MAXMASK >> c) & 1u) ? (o > v[c] ? o : v[c]) : v[c] + o;
    }
  if (lane == 0)
#pragma unroll
    for (int c = 0; c < NV; ++c) sred[warp * NV + c] = v[c];
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int c = 0; c < NV; ++c) {
      double a = 0.0;
      for (int w = 0; w < nw; ++w) {
        const double x = (double)sred[w * NV + c];
        a = ((MAXMASK >> c) & 1u) ? fmax(a, x) : a + x;
      }
      part[(size_t)chunk * 2 + c] = a;
    }
    __threadfence();
    am_last = (atomicAdd(ticket, 1u) == (unsigned)nitems - 1u);
  }
  __syncthreads();
  const bool last = am_last;
  __syncthreads();  // sred and am_last are reused below and by the next item of this CTA
  if (!last) return false;
  __threadfence();
  // the last CTA: thread t adds items t, t + blockDim.x, ... in order, then a
  // fixed-order CTA sum (deterministic for the problem's item count)
  double a[NV];
#pragma unroll
  for (int c = 0; c < NV; ++c) a[c] = 0.0;
  for (int it = threadIdx.x; it < nitems; it += blockDim.x)
#pragma unroll
    for (int c = 0; c < NV; ++c) {
      const double x = __ldcg(part + (size_t)it * 2 + c);
      a[c] = ((MAXMASK >> c) & 1u) ? fmax(a[c], x) : a[c] + x;
    }
  __shared__ double sred2[32 * 2];
#pragma unroll
  for (int c = 0; c < NV; ++c)
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const double o = __shfl_down_sync(0xffffffffu, a[c], off);
      a[c] = ((MAXMASK >> c) & 1u) ? fmax(a[c], o) : a[c] + o;
    }
  if (lane == 0)
#pragma unroll
    for (int c = 0; c < NV; ++c) sred2[warp * NV + c] = a[c];
  __syncthreads();
  // thread 0 reads sred2 before it meets the next barrier; sred2 is written
  // again only after several more barriers, so no barrier is needed here
  if (threadIdx.x != 0) return false;
#pragma unroll
  for (int c = 0; c < NV; ++c) {
    tot[c] = 0.0;
    for (int w = 0; w < nw; ++w)
      tot[c] = ((MAXMASK >> c) & 1u) ? fmax(tot[c], sred2[w * NV + c]) : tot[c] + sred2[w * NV + c];
  }
  *ticket = 0u;
  return true;
}

// Loop over the work list: CTA-strided items; inside, tile by tile, thread t
// owns segment tile * blockDim.x + t of problem P (geometry g).
#define RK_BATCH_ITEMS(items, nitems_total)                                         \
  for (int it_ = blockIdx.x; it_ < (nitems_total); it_ += gridDim.x) {             \
    const BatchItem item_ = (items)[it_];

#define RK_BATCH_CHUNKS_END }
#define RK_BATCH_CHUNKS(P, SEG)                                                    \
  for (int c_ = 0; c_ < item_.nch; ++c_) {                                         \
    const HeatGeo& g = (P).g;                                                      \
    const long long sidx_ = (long long)(item_.chunk + c_) * blockDim.x + threadIdx.x; \
    const bool live_ = sidx_ < g.n2 * g.nseg;                                      \
    const long long line = live_ ? sidx_ / g.nseg : 0;                             \
    const int i0 = live_ ? (int)(sidx_ - line * g.nseg) * (SEG) : 0;               \
    const int m = live_ ? min((SEG), g.n - i0) : 0;                                \
    const int j = (int)(line % g.n);                                               \
    const int k = (int)(line / g.n);                                               \
    const long long base = line * g.n + i0;                                       \
    const int pbase = k * (P).plane + j * (P).ld + i0;                            \
    const int mk = (P).full ? (SEG) : m;

// Sum of the six neighbours of a segment in the padded layout of the Krylov
// vectors and k^eps (line pitch ld, plane pitch `plane`): nb_sum with pitched
// offsets.  own[] holds the field on the segment (zeros past m).
template <typename T, int SEG, typename SegF, typename PtF>
__device__ __forceinline__ void bt_nb_sum(int n, int ld, int plane, int i0, int m, int j, int k, int pb,
                                          const T (&own)[SEG], SegF seg, PtF pt, T (&nb)[SEG]) {
  const T left = (i0 > 0) ? pt(pb - 1) : T(0);
  const T right = (i0 + SEG < n) ? pt(pb + SEG) : T(0);
#pragma unroll
  for (int e = 0; e < SEG; ++e) {
    const T l = (e > 0) ? own[e - 1] : left;
    const T r = (e + 1 < SEG) ? own[e + 1] : right;
    nb[e] = l + r;
  }
  T tmp[SEG];
  if (j > 0) {
    seg(pb - ld, m, tmp);
#pragma unroll
    for (int e = 0; e < SEG; ++e) nb[e] += tmp[e];
  }
  if (j < n - 1) {
    seg(pb + ld, m, tmp);
#pragma unroll
    for (int e = 0; e < SEG; ++e) nb[e] += tmp[e];
  }
  if (k > 0) {
    seg(pb - plane, m, tmp);
#pragma unroll
    for (int e = 0; e < SEG; ++e) nb[e] += tmp[e];
  }
  if (k < n - 1) {
    seg(pb + plane, m, tmp);
#pragma unroll
    for (int e = 0; e < SEG; ++e) nb[e] += tmp[e];
  }
}

// ------------------------------------------------------------ FP64 phases
// Stage right-hand side r = u + sum ch k_j + sum ce k^eps_j / sigma_j (Eqs.
// mpAstep1-4), FP64, element-wise.
template <typename T, int BS, int SEG, typename X>
__global__ void __launch_bounds__(kThreads) bt_combine(BatchProb<T, BS>* P, const BatchItem* items, int nitems,
                                                       BatchStage st) {
  RK_BATCH_ITEMS(items, nitems)
    const BatchProb<T, BS>& pb = P[item_.prob];
    RK_BATCH_CHUNKS(pb, SEG)
    if (!live_) continue;
    double v[SEG], t[SEG];
    load_seg<double, double, SEG>(pb.u + base, m, v);
    for (int h = 0; h < st.nh; ++h) {
      load_seg<double, double, SEG>(pb.k[st.hj[h]] + base, m, t);
#pragma unroll
      for (int e = 0; e < SEG; ++e) v[e] = fma(st.ch[h], t[e], v[e]);
    }
    for (int h = 0; h < st.ne; ++h) {
      const double c = st.ce[h] / pb.rs[st.ej[h]].sigma;
      load_seg<double, X, SEG>(static_cast<const X*>(pb.ke[st.ej[h]]) + pbase, mk, t);
#pragma unroll
      for (int e = 0; e < SEG; ++e) v[e] = fma(c, t[e], v[e]);
    }
    store_seg<double, double, SEG>(pb.r + base, m, v);
    RK_BATCH_CHUNKS_END
  }
}

// y = L x in FP64 (x = r, or u when the stage has no history terms); for an
// implicit stage y = g with ||g||^2, ||g||_inf and the storage scale into the
// problem's stage scalars, for an explicit stage y = k_i.
template <typename T, int BS, int SEG>
__global__ void __launch_bounds__(kThreads) bt_apply(BatchProb<T, BS>* P, const BatchItem* items, int nitems,
                                                     BatchStage st) {
  const bool implicit = st.shift_a != 0.0;
  RK_BATCH_ITEMS(items, nitems)
    BatchProb<T, BS>& pb = P[item_.prob];
    const double* x = st.use_r ? pb.r : pb.u;
    double* y = implicit ? pb.g64 : pb.k[st.stage];
    double acc[2] = {0.0, 0.0};
    RK_BATCH_CHUNKS(pb, SEG)
    (void)pbase;
    (void)mk;
    if (live_) {
      double xv[SEG], nb[SEG], yv[SEG];
      load_seg<double, double, SEG>(x + base, m, xv);
      nb_sum<double, SEG>(
          g, i0, m, j, k, base, xv,
          [&](long long off, int mm, double (&v)[SEG]) { load_seg<double, double, SEG>(x + off, mm, v); },
          [&](long long idx) { return x[idx]; }, nb);
      const double c = pb.c;
#pragma unroll
      for (int e = 0; e < SEG; ++e) {
        yv[e] = c * fma(-6.0, xv[e], nb[e]);
        if (e < m) {
          acc[0] = fma(yv[e], yv[e], acc[0]);
          acc[1] = fmax(acc[1], fabs(yv[e]));
        }
      }
      store_seg<double, double, SEG>(y + base, m, yv);
    }
    RK_BATCH_CHUNKS_END
    if (!implicit) continue;
    double tot[2];
    if (prob_reduce<double, 2, 2u>(acc, pb.part, pb.ticket, item_.idx, pb.nitems, tot)) {
      RhsScalars* rs = pb.rs + st.stage;
      rs->gg = tot[0];
      rs->gmax = tot[1];
      rs->sigma = rhs_scale(rs, tot[0], tot[1], pb.g.N);
    }
  }
}

// Problem-level end of a solve: statistics and the count of problems still
// iterating (called by the thread that finished the problem's reduction).
template <typename T, int BS>
__device__ __forceinline__ void bt_solve_done(BatchProb<T, BS>& pb, int* active) {
  CgScalars* sc = pb.sc;
  pb.iters_total += sc->iter;
  pb.iters_max = max(pb.iters_max, sc->iter);
  pb.solves += 1;
  if (sc->status == 4) pb.not_converged += 1;
  if (sc->status == 5) pb.status = 5;
  atomicSub(active, 1);
}

// k = g + shift c L(ke / sigma) in FP64 (the explicit correction k_i = L y_i,
// y_i = r_i + shift k^eps_i) and ||k - ke/sigma||^2, the true residual of the
// stage system; FP32 k^eps uses the exact FP32-pair Laplacian of the
// single-problem path.  With correct = 0: k = ke / sigma widened.
template <typename T, int BS, int SEG, typename X>
__global__ void __launch_bounds__(kThreads) bt_correct(BatchProb<T, BS>* P, const BatchItem* items, int nitems,
                                                       BatchStage st) {
  RK_BATCH_ITEMS(items, nitems)
    BatchProb<T, BS>& pb = P[item_.prob];
    const RhsScalars* rs = pb.rs + st.stage;
    const double inv_sigma = 1.0 / rs->sigma;
    const X* ke = static_cast<const X*>(pb.ke[st.stage]);
    double* kout = pb.k[st.stage];
    double acc[1] = {0.0};
    RK_BATCH_CHUNKS(pb, SEG)
    if (live_ && !st.correct) {
      double v[SEG];
      load_seg<double, X, SEG>(ke + pbase, mk, v);
#pragma unroll
      for (int e = 0; e < SEG; ++e) v[e] *= inv_sigma;
      store_seg<double, double, SEG>(kout + base, m, v);
    } else if (live_) {
      const double c2 = st.shift_a * pb.c * inv_sigma;
      double gs[SEG], kv[SEG];
      load_seg<double, double, SEG>(pb.g64 + base, m, gs);
      if constexpr (sizeof(X) == 4) {
        float v[SEG], ym[SEG], yp[SEG], zm[SEG], zp[SEG];
        load_seg<float, X, SEG>(ke + pbase, mk, v);
        const float left = (i0 > 0) ? wid<float>(ke[pbase - 1]) : 0.f;
        const float right = (i0 + SEG < g.n) ? wid<float>(ke[pbase + SEG]) : 0.f;
        auto seg_or_zero = [&](bool in, long long off, float (&w)[SEG]) {
          if (in) {
            load_seg<float, X, SEG>(ke + off, mk, w);
          } else {
#pragma unroll
            for (int e = 0; e < SEG; ++e) w[e] = 0.f;
          }
        };
        seg_or_zero(j > 0, pbase - pb.ld, ym);
        seg_or_zero(j < g.n - 1, pbase + pb.ld, yp);
        seg_or_zero(k > 0, pbase - pb.plane, zm);
        seg_or_zero(k < g.n - 1, pbase + pb.plane, zp);
#pragma unroll
        for (int e = 0; e < SEG; ++e) {
          const float xl = (e > 0) ? v[e - 1] : left;
          const float xr = (e + 1 < SEG) ? v[e + 1] : right;
          kv[e] = fma(c2, lap_pair(v[e], xl, xr, ym[e], yp[e], zm[e], zp[e]), gs[e]);
          const double res = fma(-(double)v[e], inv_sigma, kv[e]);
          if (e < m) acc[0] = fma(res, res, acc[0]);
        }
      } else {
        double v[SEG], nb[SEG];
        load_seg<double, X, SEG>(ke + pbase, mk, v);
        bt_nb_sum<double, SEG>(
            g.n, pb.ld, pb.plane, i0, mk, j, k, pbase, v,
            [&](long long off, int mm, double (&w)[SEG]) { load_seg<double, X, SEG>(ke + off, mm, w); },
            [&](long long idx) { return wid<double>(ke[idx]); }, nb);
#pragma unroll
        for (int e = 0; e < SEG; ++e) {
          kv[e] = fma(c2, fma(-6.0, v[e], nb[e]), gs[e]);
          const double res = kv[e] - v[e] * inv_sigma;
          if (e < m) acc[0] = fma(res, res, acc[0]);
        }
      }
      store_seg<double, double, SEG>(kout + base, m, kv);
    }
    RK_BATCH_CHUNKS_END
    if (!st.correct) continue;
    double tot[1];
    if (prob_reduce<double, 1>(acc, pb.part, pb.ticket, item_.idx, pb.nitems, tot)) {
      RhsScalars* w = pb.rs + st.stage;
      w->res2 = tot[0];
      if (w->gg > 0.0) pb.true_res_max = fmax(pb.true_res_max, sqrt(tot[0] / w->gg));
    }
  }
}

// u += sum_j cb_j k_j (Eq. RKstep, cb_j = dt b_j), FP64.
struct BatchUpdate {
  int nb;
  int j[kBatchStages];
  double cb[kBatchStages];
};

template <typename T, int BS, int SEG>
__global__ void __launch_bounds__(kThreads) bt_update(BatchProb<T, BS>* P, const BatchItem* items, int nitems,
                                                      BatchUpdate up) {
  RK_BATCH_ITEMS(items, nitems)
    const BatchProb<T, BS>& pb = P[item_.prob];
    RK_BATCH_CHUNKS(pb, SEG)
    (void)pbase;
    (void)mk;
    if (!live_) continue;
    double v[SEG], t[SEG];
    load_seg<double, double, SEG>(pb.u + base, m, v);
    for (int h = 0; h < up.nb; ++h) {
      load_seg<double, double, SEG>(pb.k[up.j[h]] + base, m, t);
#pragma unroll
      for (int e = 0; e < SEG; ++e) v[e] = fma(up.cb[h], t[e], v[e]);
    }
    store_seg<double, double, SEG>(pb.u + base, m, v);
    RK_BATCH_CHUNKS_END
  }
}

// ------------------------------------------------------------ CG phases
// z = D^{-1} r on the blocks of a segment whose first m elements are valid:
// the factored tridiagonal block of BjTri; a partial block at the end of an
// x-line (m mod BS nodes) uses the leading pivots, which are those of its own
// LU factorisation.
template <typename T, int BS, int SEG>
__device__ __forceinline__ void bj_apply_tri_m(const BjTri<T, BS>& t, const T (&r)[SEG], T (&z)[SEG], int m) {
  static_assert(SEG % BS == 0, "segments hold whole blocks");
#pragma unroll
  for (int cb = 0; cb < SEG / BS; ++cb) {
    const int mb = m - cb * BS;  // valid elements of this block (may be <= 0 or >= BS)
    T y[BS];
    y[0] = t.ip[0] * r[cb * BS];
#pragma unroll
    for (int i = 1; i < BS; ++i) y[i] = t.ip[i] * fma(t.mo, y[i - 1], r[cb * BS + i]);
    T zn = T(0);
#pragma unroll
    for (int i = BS - 1; i >= 0; --i) {
      const T zi = (i == mb - 1) ? y[i] : (i < mb - 1 ? fma(t.nu[i], zn, y[i]) : T(0));
      z[cb * BS + i] = zi;
      zn = zi;
    }
  }
}

// Start of the stage solve of every problem: r = sigma g (rounded to S),
// z = D^{-1} r, x = 0, and r.z, r.r; the problem's scalars get the stopping
// threshold; a problem whose right-hand side already meets it is done.
template <typename S, typename T, int BS, int SEG>
__global__ void __launch_bounds__(kThreads) bt_cg_init(BatchProb<T, BS>* P, const BatchItem* items, int nitems,
                                                       BatchStage st, int* active) {
  using X = typename XOf<S>::type;
  __shared__ BjTri<T, BS> stri;
  RK_BATCH_ITEMS(items, nitems)
    BatchProb<T, BS>& pb = P[item_.prob];
    const double sigma = pb.rs[st.stage].sigma;
    T acc[2] = {T(0), T(0)};
    // the stage's factored block in shared memory (the previous item's last
    // barrier has passed, so no thread still reads it)
    {
      const T* src = reinterpret_cast<const T*>(&pb.tri[st.stage]);
      T* dst = reinterpret_cast<T*>(&stri);
      for (int c = threadIdx.x; c < (int)(sizeof(BjTri<T, BS>) / sizeof(T)); c += blockDim.x) dst[c] = src[c];
    }
    __syncthreads();
    RK_BATCH_CHUNKS(pb, SEG)
    if (live_) {
      double gd[SEG];
      load_seg<double, double, SEG>(pb.g64 + base, m, gd);
      T rv[SEG], zv[SEG], zero[SEG];
#pragma unroll
      for (int e = 0; e < SEG; ++e) {
        rv[e] = (e < m) ? rnd<S, T>(sigma == 1.0 ? (T)gd[e] : (T)(gd[e] * sigma)) : T(0);
        zero[e] = T(0);
      }
      bj_apply_tri_m<T, BS, SEG>(stri, rv, zv, m);
#pragma unroll
      for (int e = 0; e < SEG; ++e) {
        zv[e] = rnd<S, T>(zv[e]);
        acc[0] = fma(rv[e], zv[e], acc[0]);
        acc[1] = fma(rv[e], rv[e], acc[1]);
      }
      // whole segments: the line padding is set to zero here and stays zero
      store_seg<S, T, SEG>(static_cast<S*>(pb.wr) + pbase, mk, rv);
      store_seg<S, T, SEG>(static_cast<S*>(pb.wz) + pbase, mk, zv);
      store_seg<X, T, SEG>(static_cast<X*>(pb.ke[st.stage]) + pbase, mk, zero);
    }
    RK_BATCH_CHUNKS_END
    double tot[2];
    if (prob_reduce<T, 2>(acc, pb.part, pb.ticket, item_.idx, pb.nitems, tot)) {
      CgScalars* sc = pb.sc;
      sc->tol_rel = pb.tol_rel;
      sc->tol_abs = pb.tol_abs;
      sc->max_iter = pb.max_iter;
      sc->rz = tot[0];
      sc->rr = tot[1];
      sc->gg = tot[1];
      const double ta = pb.tol_abs * sigma;
      sc->thresh2 = fmax(pb.tol_rel * pb.tol_rel * tot[1], ta * ta);
      sc->iter = 0;
      sc->beta = 0.0;
      sc->alpha = 0.0;
      sc->pAp = 0.0;
      sc->status = 0;
      sc->done = 0;
      if (!isfinite(tot[0]) || !isfinite(tot[1])) {
        sc->done = 1;
        sc->status = 5;
      } else if (tot[1] <= sc->thresh2 || tot[1] == 0.0) {
        sc->done = 1;
      }
      if (sc->done) bt_solve_done(pb, active);
    }
  }
}

// Sweep A of every unfinished problem: p = z + beta p_old (rounded to S),
// p.Ap from the grid edges; its last CTA forms alpha (ping-pong p buffers
// chosen by the problem's iteration parity).
template <typename S, typename T, int BS, int SEG>
__global__ void __launch_bounds__(kThreads, 4) bt_cg_a(BatchProb<T, BS>* P, const BatchItem* items, const int* nitems_dev,
                                                       BatchStage st, int* active) {
  const int nitems = *nitems_dev;
  RK_BATCH_ITEMS(items, nitems)
    BatchProb<T, BS>& pb = P[item_.prob];
    CgScalars* sc = pb.sc;
    if (sc->done) continue;  // uniform over the CTA
    const int iter = sc->iter;
    const bool first = iter == 0;
    const T beta = (T)sc->beta;
    const T d = pb.d[st.stage], o = pb.o[st.stage];
    const S* z = static_cast<const S*>(pb.wz);
    const S* pold = static_cast<const S*>(pb.wp[(iter & 1) ^ 1]);
    S* pnew = static_cast<S*>(pb.wp[iter & 1]);
    T acc[1] = {T(0)};
    RK_BATCH_CHUNKS(pb, SEG)
    (void)base;
    if (live_) {
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
      // p.Ap from the grid edges: A = d I + o (sum of the six neighbours) is
      // symmetric, so p.Ap = sum_e p_e (d p_e + 2 o (p_{e+x} + p_{e+y} + p_{e+z}))
      // with every edge taken once from its lower element (neighbours outside
      // the grid zero): only the upper neighbours are formed
      T pv[SEG], up[SEG], tmp[SEG];
      pseg(pbase, mk, pv);
      const T right = (i0 + SEG < g.n) ? ppt(pbase + SEG) : T(0);
#pragma unroll
      for (int e = 0; e < SEG; ++e) up[e] = (e + 1 < SEG) ? pv[e + 1] : right;
      if (j < g.n - 1) {
        pseg(pbase + pb.ld, mk, tmp);
#pragma unroll
        for (int e = 0; e < SEG; ++e) up[e] += tmp[e];
      }
      if (k < g.n - 1) {
        pseg(pbase + pb.plane, mk, tmp);
#pragma unroll
        for (int e = 0; e < SEG; ++e) up[e] += tmp[e];
      }
      const T o2 = o + o;
#pragma unroll
      for (int e = 0; e < SEG; ++e)
        if (e < m) acc[0] = fma(pv[e], fma(d, pv[e], o2 * up[e]), acc[0]);
      store_seg<S, T, SEG>(pnew + pbase, mk, pv);
    }
    RK_BATCH_CHUNKS_END
    double tot[1];
    if (prob_reduce<T, 1>(acc, pb.part, pb.ticket, item_.idx, pb.nitems, tot)) {
      sc->pAp = tot[0];
      const double alpha = sc->rz / tot[0];
      sc->alpha = alpha;
      if (!isfinite(tot[0]) || !isfinite(sc->rz)) {
        sc->done = 1;
        sc->status = 5;
      } else if (!(tot[0] > 0.0) || !isfinite(alpha)) {
        sc->done = 1;  // attainable accuracy reached: current iterate, not converged
        sc->status = 4;
      }
      if (sc->done) bt_solve_done(pb, active);
    }
  }
}

// Sweep B of every unfinished problem: q = A p, r -= alpha q, x += alpha p,
// z = D^{-1} r, r.z and r.r; its last CTA forms beta and tests convergence.
template <typename S, typename T, int BS, int SEG>
__global__ void __launch_bounds__(kThreads, 4) bt_cg_b(BatchProb<T, BS>* P, const BatchItem* items, const int* nitems_dev,
                                                       BatchStage st, int* active) {
  using X = typename XOf<S>::type;
  __shared__ BjTri<T, BS> stri;
  const int nitems = *nitems_dev;
  RK_BATCH_ITEMS(items, nitems)
    BatchProb<T, BS>& pb = P[item_.prob];
    CgScalars* sc = pb.sc;
    if (sc->done) continue;  // uniform over the CTA
    const int iter = sc->iter;
    const bool xzero = iter == 0;
    const T alpha = (T)sc->alpha;
    const T d = pb.d[st.stage], o = pb.o[st.stage];
    const S* p = static_cast<const S*>(pb.wp[iter & 1]);
    S* r = static_cast<S*>(pb.wr);
    S* z = static_cast<S*>(pb.wz);
    X* x = static_cast<X*>(pb.ke[st.stage]);
    T acc[2] = {T(0), T(0)};
    // the stage's factored block in shared memory (the previous item's last
    // barrier has passed, so no thread still reads it)
    {
      const T* src = reinterpret_cast<const T*>(&pb.tri[st.stage]);
      T* dst = reinterpret_cast<T*>(&stri);
      for (int c = threadIdx.x; c < (int)(sizeof(BjTri<T, BS>) / sizeof(T)); c += blockDim.x) dst[c] = src[c];
    }
    __syncthreads();
    RK_BATCH_CHUNKS(pb, SEG)
    (void)base;
    if (live_) {
      T pv[SEG], nb[SEG], rv[SEG], xv[SEG], zv[SEG];
      load_seg<T, S, SEG>(p + pbase, mk, pv);
      bt_nb_sum<T, SEG>(
          g.n, pb.ld, pb.plane, i0, mk, j, k, pbase, pv,
          [&](long long off, int mm, T (&v)[SEG]) { load_seg<T, S, SEG>(p + off, mm, v); },
          [&](long long idx) { return wid<T>(p[idx]); }, nb);
      load_seg<T, S, SEG>(r + pbase, mk, rv);
      if (!xzero) {
        load_seg<T, X, SEG>(x + pbase, mk, xv);
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
      bj_apply_tri_m<T, BS, SEG>(stri, rv, zv, m);
#pragma unroll
      for (int e = 0; e < SEG; ++e) {
        zv[e] = rnd<S, T>(zv[e]);
        if (e < m) {
          acc[0] = fma(rv[e], zv[e], acc[0]);
          acc[1] = fma(rv[e], rv[e], acc[1]);
        }
      }
      store_seg<X, T, SEG>(x + pbase, mk, xv);
      store_seg<S, T, SEG>(r + pbase, mk, rv);
      store_seg<S, T, SEG>(z + pbase, mk, zv);
    }
    RK_BATCH_CHUNKS_END
    double tot[2];
    if (prob_reduce<T, 2>(acc, pb.part, pb.ticket, item_.idx, pb.nitems, tot)) {
      const double rz_new = tot[0];
      sc->beta = rz_new / sc->rz;
      sc->rz = rz_new;
      sc->rr = tot[1];
      sc->iter = iter + 1;
      if (!isfinite(tot[0]) || !isfinite(tot[1])) {
        sc->done = 1;
        sc->status = 5;
      } else if (tot[1] <= sc->thresh2) {
        sc->done = 1;
      } else if (sc->iter >= sc->max_iter) {
        sc->done = 1;
        sc->status = 4;
      }
      if (sc->done) bt_solve_done(pb, active);
    }
  }
}

// Work list of the problems still iterating: the items of unfinished problems
// of `in` are appended to `out`.  Their order is arbitrary: every problem's
// reduction adds its partials by item index, so results depend neither on it
// nor on the launch shape.
template <typename T, int BS>
__global__ void __launch_bounds__(kThreads) bt_compact(BatchProb<T, BS>* P, const BatchItem* in, const int* in_count,
                                                       BatchItem* out, int* out_count) {
  const int n = *in_count;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const BatchItem it = in[i];
    if (P[it.prob].sc->done) continue;
    out[atomicAdd(out_count, 1)] = it;
  }
}

// ------------------------------------------------------------ host runner
// Steps a group of problems that share storage, block size, tableau and step
// size (rk_integrate_batch groups them): all phases as work-list launches on
// `st`, the CG sweeps in chunks sized by the previous step's largest
// iteration count, the host reading the count of unfinished problems once
// per chunk.  Instantiated per storage type in rk_batch_*.cu.
struct BatchTotals {
  long long iters_total = 0;
  int iters_max = 0, solves = 0, not_converged = 0, nonfinite = 0;
  double true_res = -1.0;
  long long launches = 0;
  double bytes = 0.0;  // algorithmic bytes of the working launches
};

template <typename S>
rk_status batch_group_run(rk_problem** ps, int count, double dt, int nsteps, cudaStream_t st, int grid_cap,
                          BatchTotals* out);

}  // namespace rk

#ifdef RK_BATCH_INSTANTIATE
#include <algorithm>
#include <vector>

#include "rk_internal.h"

namespace rk {

template <typename S>
struct ArithOf { using type = float; };
template <>
struct ArithOf<double> { using type = double; };

template <typename S, int BS>
static rk_status batch_group_bs(rk_problem** ps, int count, double dt, int nsteps, cudaStream_t st, int grid_cap,
                                BatchTotals* out) {
  using T = typename ArithOf<S>::type;
  using X = typename XOf<S>::type;
  constexpr int SEG = seg_of<S, BS>();
  using Prob = BatchProb<T, BS>;
  const rk_problem* p0 = ps[0];
  const int q = p0->q;
  const bool mixed = p0->sol.correct != 0;
  // host descriptors and the work list
  std::vector<Prob> hp(count);
  std::vector<BatchItem> items;
  long long part_total = 0;
  for (int i = 0; i < count; ++i) {
    const rk_problem* p = ps[i];
    Prob& b = hp[i];
    std::memset(&b, 0, sizeof(Prob));
    b.g = HeatGeo{p->n, (p->n + SEG - 1) / SEG, (long long)p->n * p->n, p->N};
    b.c = p->c;
    b.u = p->u;
    b.r = p->r;
    b.g64 = p->g64;
    for (int s = 0; s < kBatchStages; ++s) {
      b.k[s] = p->k[s];
      b.ke[s] = p->ke[s];
    }
    b.wr = p->wr;
    b.wz = p->wz;
    b.wp[0] = p->wp[0];
    b.wp[1] = p->wp[1];
    b.sc = p->sc;
    b.rs = p->rs;
    // FP64 storage without correction keeps k^eps in k (unpadded); otherwise
    // the Krylov vectors and k^eps use lines padded to batch_pitch(n)
    b.ld = (!mixed && std::is_same<S, double>::value) ? p->n : batch_pitch(p->n, p->sol.storage, BS);
    b.full = (b.ld % SEG == 0) ? 1 : 0;
    b.plane = p->n * b.ld;
    const long long nsegs = b.g.n2 * b.g.nseg;
    const int ntiles = (int)((nsegs + kThreads - 1) / kThreads);
    b.nitems = (ntiles + kBatchTilesPerItem - 1) / kBatchTilesPerItem;
    for (int c = 0; c < b.nitems; ++c)
      items.push_back(BatchItem{i, c * kBatchTilesPerItem, std::min(kBatchTilesPerItem, ntiles - c * kBatchTilesPerItem), c});
    b.part = reinterpret_cast<double*>(part_total);  // offset of the problem's partials (fixed up below)
    part_total += 2LL * b.nitems;
    b.max_iter = p->sol.max_iter;
    b.tol_rel = p->sol.tol_rel;
    b.tol_abs = p->sol.tol_abs;
    for (int s = 0; s < q; ++s) {
      const double a = p->Al[s * q + s];
      const double dd = 1.0 + 6.0 * dt * a * p->c, oo = -dt * a * p->c;
      b.d[s] = (T)dd;
      b.o[s] = (T)oo;
      b.tri[s] = bj_tri<T, BS>(dd, oo);
    }
    b.true_res_max = -1.0;
  }
  // device copies: descriptors, work list, partials, tickets, active counter
  Prob* dp = nullptr;
  BatchItem* ditems = nullptr;
  double* dpart = nullptr;
  unsigned* dtick = nullptr;
  int* dactive = nullptr;
  int* hactive = nullptr;
  BatchItem* dlist[2] = {nullptr, nullptr};  // work lists of the unfinished problems (ping-pong)
  int* dcount = nullptr;                     // [0], [1]: their lengths; [2]: the full list's length
  rk_status status = RK_OK;
  auto cleanup = [&] {
    if (dp) cudaFreeAsync(dp, st);
    if (ditems) cudaFreeAsync(ditems, st);
    if (dpart) cudaFreeAsync(dpart, st);
    if (dtick) cudaFreeAsync(dtick, st);
    if (dactive) cudaFreeAsync(dactive, st);
    if (dlist[0]) cudaFreeAsync(dlist[0], st);
    if (dlist[1]) cudaFreeAsync(dlist[1], st);
    if (dcount) cudaFreeAsync(dcount, st);
    if (hactive) cudaFreeHost(hactive);
  };
  if (cudaMallocAsync((void**)&dp, sizeof(Prob) * count, st) != cudaSuccess ||
      cudaMallocAsync((void**)&ditems, sizeof(BatchItem) * items.size(), st) != cudaSuccess ||
      cudaMallocAsync((void**)&dpart, sizeof(double) * part_total, st) != cudaSuccess ||
      cudaMallocAsync((void**)&dtick, sizeof(unsigned) * count, st) != cudaSuccess ||
      cudaMallocAsync((void**)&dactive, sizeof(int), st) != cudaSuccess ||
      cudaMallocAsync((void**)&dlist[0], sizeof(BatchItem) * items.size(), st) != cudaSuccess ||
      cudaMallocAsync((void**)&dlist[1], sizeof(BatchItem) * items.size(), st) != cudaSuccess ||
      cudaMallocAsync((void**)&dcount, sizeof(int) * 3, st) != cudaSuccess ||
      cudaMallocHost((void**)&hactive, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    cleanup();
    set_error("rk_integrate_batch: work-list allocation failed");
    return RK_ERR_OOM;
  }
  for (int i = 0; i < count; ++i) {
    hp[i].part = dpart + reinterpret_cast<long long>(hp[i].part);
    hp[i].ticket = dtick + i;
  }
  cudaMemcpyAsync(dp, hp.data(), sizeof(Prob) * count, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(ditems, items.data(), sizeof(BatchItem) * items.size(), cudaMemcpyHostToDevice, st);
  cudaMemsetAsync(dtick, 0, sizeof(unsigned) * count, st);
  const int nit = (int)items.size();
  {
    const int counts[3] = {0, 0, nit};
    cudaMemcpyAsync(dcount, counts, sizeof(counts), cudaMemcpyHostToDevice, st);
    cudaStreamSynchronize(st);  // counts lives on this stack frame
  }
  auto grid_of = [&](const void* kern, int nlist) {
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kThreads, 0) != cudaSuccess || occ < 1) occ = 1;
    if (grid_cap > 0 && occ > grid_cap) occ = grid_cap;
    return std::max(1, std::min(nlist, device_sms() * occ));
  };
  auto kcomb = bt_combine<T, BS, SEG, X>;
  auto kapp = bt_apply<T, BS, SEG>;
  auto kini = bt_cg_init<S, T, BS, SEG>;
  auto ka = bt_cg_a<S, T, BS, SEG>;
  auto kb = bt_cg_b<S, T, BS, SEG>;
  auto kcor = bt_correct<T, BS, SEG, X>;
  auto kupd = bt_update<T, BS, SEG>;
  auto kcmp = bt_compact<T, BS>;
  const int gcmp = std::max(1, std::min((nit + kThreads - 1) / kThreads, device_sms() * 4));
  const int gcomb = grid_of((const void*)kcomb, nit), gapp = grid_of((const void*)kapp, nit),
            gini = grid_of((const void*)kini, nit), ga = grid_of((const void*)ka, nit),
            gb = grid_of((const void*)kb, nit), gcor = grid_of((const void*)kcor, nit),
            gupd = grid_of((const void*)kupd, nit);
  // stage coefficients of the shared tableau
  bool implicit[kBatchStages];
  for (int i = 0; i < q; ++i) implicit[i] = p0->Al[i * q + i] != 0.0;
  std::vector<BatchStage> stages(q);
  for (int i = 0; i < q; ++i) {
    BatchStage& sg = stages[i];
    std::memset(&sg, 0, sizeof(sg));
    sg.stage = i;
    for (int jj = 0; jj < i; ++jj) {
      double chj = dt * p0->Ah[i * q + jj], cej = dt * p0->Al[i * q + jj];
      if (cej != 0.0 && (!implicit[jj] || !mixed)) {
        chj += cej;
        cej = 0.0;
      }
      if (chj != 0.0) {
        sg.hj[sg.nh] = jj;
        sg.ch[sg.nh++] = chj;
      }
      if (cej != 0.0) {
        sg.ej[sg.ne] = jj;
        sg.ce[sg.ne++] = cej;
      }
    }
    sg.use_r = (sg.nh + sg.ne) > 0;
    sg.shift_a = implicit[i] ? dt * p0->Al[i * q + i] : 0.0;
    sg.correct = mixed ? 1 : 0;
  }
  BatchUpdate up{};
  for (int jj = 0; jj < q; ++jj)
    if (p0->b[jj] != 0.0) {
      up.j[up.nb] = jj;
      up.cb[up.nb++] = dt * p0->b[jj];
    }
  const bool aliased = p0->ke_alias[0] || (!mixed && std::is_same<S, double>::value);
  std::vector<int> predicted(q, 8);
  long long launches = 0;
  for (int step = 0; step < nsteps && status == RK_OK; ++step) {
    for (int i = 0; i < q && status == RK_OK; ++i) {
      const BatchStage& sg = stages[i];
      if (sg.use_r) {
        kcomb<<<gcomb, kThreads, 0, st>>>(dp, ditems, nit, sg);
        ++launches;
      }
      kapp<<<gapp, kThreads, 0, st>>>(dp, ditems, nit, sg);
      ++launches;
      if (!implicit[i]) continue;
      *hactive = count;
      cudaMemcpyAsync(dactive, hactive, sizeof(int), cudaMemcpyHostToDevice, st);
      kini<<<gini, kThreads, 0, st>>>(dp, ditems, nit, sg, dactive);
      // the work list of the problems whose solve did not end at the start
      int cur = 0;
      cudaMemsetAsync(dcount + cur, 0, sizeof(int), st);
      kcmp<<<gcmp, kThreads, 0, st>>>(dp, ditems, dcount + 2, dlist[cur], dcount + cur);
      launches += 2;
      int launched = 0, chunk = std::max(2, predicted[i]);
      while (true) {
        for (int c = 0; c < chunk; ++c) {
          ka<<<ga, kThreads, 0, st>>>(dp, dlist[cur], dcount + cur, sg, dactive);
          kb<<<gb, kThreads, 0, st>>>(dp, dlist[cur], dcount + cur, sg, dactive);
          // drop the items of the problems that finished in this iteration
          cudaMemsetAsync(dcount + (cur ^ 1), 0, sizeof(int), st);
          kcmp<<<gcmp, kThreads, 0, st>>>(dp, dlist[cur], dcount + cur, dlist[cur ^ 1], dcount + (cur ^ 1));
          cur ^= 1;
        }
        launches += 3 * chunk;
        launched += chunk;
        if (cudaGetLastError() != cudaSuccess) {
          set_error("rk_integrate_batch: CG sweep launch failed");
          status = RK_ERR_CUDA;
          break;
        }
        if (cudaMemcpyAsync(hactive, dactive, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
          set_error("rk_integrate_batch: status readback failed: %s", cudaGetErrorString(cudaGetLastError()));
          status = RK_ERR_CUDA;
          break;
        }
        if (*hactive <= 0) break;
        int cap = 0;
        for (int pi = 0; pi < count; ++pi) cap = std::max(cap, ps[pi]->sol.max_iter);
        if (launched > cap + 4) {  // every problem stops at its own max_iter
          set_error("rk_integrate_batch: CG did not stop after %d sweeps", launched);
          status = RK_ERR_TIMEOUT;
          break;
        }
        chunk = std::max(2, std::min(64, launched / 2));
      }
      predicted[i] = launched;
      if (status != RK_OK) break;
      if (!(aliased && !mixed)) {
        kcor<<<gcor, kThreads, 0, st>>>(dp, ditems, nit, sg);
        ++launches;
      }
    }
    if (status != RK_OK) break;
    kupd<<<gupd, kThreads, 0, st>>>(dp, ditems, nit, up);
    ++launches;
  }
  if (status == RK_OK && cudaGetLastError() != cudaSuccess) {
    set_error("rk_integrate_batch: launch failed");
    status = RK_ERR_CUDA;
  }
  if (status == RK_OK) {
    if (cudaMemcpyAsync(hp.data(), dp, sizeof(Prob) * count, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      set_error("rk_integrate_batch: statistics readback failed");
      status = RK_ERR_CUDA;
    } else {
      // algorithmic bytes per DOF (every element a kernel must read or write
      // once; the sweeps as in the single-problem segment path)
      const double sb = sizeof(S), xb = sizeof(X);
      double fixed = 0.0;  // per step, outside the CG iterations
      for (int i = 0; i < q; ++i) {
        const BatchStage& sg = stages[i];
        if (sg.use_r) fixed += 16.0 + 8.0 * sg.nh + xb * sg.ne;
        fixed += 16.0;
        if (!implicit[i]) continue;
        fixed += 8.0 + 2.0 * sb + xb;                       // CG start
        if (!(aliased && !mixed)) fixed += mixed ? 16.0 + xb : 8.0 + xb;  // correction / widening
      }
      fixed += 16.0 + 8.0 * up.nb;  // update
      const double per_iter = 3.0 * sb + 4.0 * sb + 2.0 * xb;  // sweeps A and B
      const double first_less = sb + xb;                     // no p_old, x read at a solve's first iteration
      for (const Prob& b : hp)
        out->bytes += (double)b.g.N * (fixed * nsteps + per_iter * b.iters_total - first_less * b.solves);
      for (int i = 0; i < count; ++i) {
        const Prob& b = hp[i];
        ps[i]->batch_status = b.status == 5 ? RK_ERR_NONFINITE : (b.not_converged ? RK_ERR_NOT_CONVERGED : RK_OK);
      }
      for (const Prob& b : hp) {
        out->iters_total += b.iters_total;
        out->iters_max = std::max(out->iters_max, b.iters_max);
        out->solves += b.solves;
        out->not_converged += b.not_converged;
        if (b.status == 5) out->nonfinite += 1;
        out->true_res = std::max(out->true_res, b.true_res_max);
      }
    }
  }
  out->launches += launches;
  cleanup();
  cudaStreamSynchronize(st);
  return status;
}

template <typename S>
rk_status batch_group_run(rk_problem** ps, int count, double dt, int nsteps, cudaStream_t st, int grid_cap,
                          BatchTotals* out) {
  switch (ps[0]->sol.bj_block) {
    case 1: return batch_group_bs<S, 1>(ps, count, dt, nsteps, st, grid_cap, out);
    case 2: return batch_group_bs<S, 2>(ps, count, dt, nsteps, st, grid_cap, out);
    case 4: return batch_group_bs<S, 4>(ps, count, dt, nsteps, st, grid_cap, out);
    case 8: return batch_group_bs<S, 8>(ps, count, dt, nsteps, st, grid_cap, out);
    case 16: return batch_group_bs<S, 16>(ps, count, dt, nsteps, st, grid_cap, out);
    default: return batch_group_bs<S, 32>(ps, count, dt, nsteps, st, grid_cap, out);
  }
}

}  // namespace rk
#endif

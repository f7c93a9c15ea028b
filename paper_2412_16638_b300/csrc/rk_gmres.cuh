// Arnoldi step of the right-preconditioned GMRES(m) with delayed classical
// Gram-Schmidt reorthogonalisation (DCGS2: the second Gram-Schmidt pass of
// a basis vector is carried out in the next Arnoldi step, where its dot
// products share the one global reduction of that step).
//
// Per step j, with u_j the once-orthogonalised, unnormalised candidate left in
// basis slot j by the previous step (u_0 = the residual):
//   gm_dc_prec     z = M^{-1} u_j                                 (block-Jacobi)
//   gm_dc_arnoldi  w = (I - shift L) z on the sliced-ELL copy of L; one
//                  reduction of s_i = v_i.u_j, t_i = v_i.w (i < j), u_j.u_j,
//                  u_j.w; the last CTA finishes column j-1 of the Hessenberg
//                  matrix (reorthogonalisation coefficients s, ||v_j|| by
//                  Pythagoras), applies the Givens rotations, tests
//                  convergence and forms the coefficients of the next step
//   gm_dc_update   v_j = (u_j - V s) / ||.||,  u_{j+1} = w / ||.|| - V c
// Algebra of the next candidate: with A = (I - shift L) M^{-1} and the Arnoldi
// relation A V_{<j} = V_{<=j} H, A v_j = (w - V_{<=j} H s) / nrm, so with
// g = H s its projections are h_i = (t_i - g_i) / nrm (i < j),
// h_j = ((u_j.w - s.t) / nrm - g_j) / nrm, and u_{j+1} = A v_j - V h =
// w / nrm - V (g / nrm + h).
//
// The two basis passes stream the vectors tile by tile through a ring of
// shared-memory stages filled by 1-D bulk copies (cp.async.bulk) with an
// mbarrier per stage; every wait is bounded.  Vectors are stored with a
// leading dimension that is a multiple of the tile, zero padded, so every copy
// is a whole 16-byte aligned tile.
#pragma once
#include "rk_csr.cuh"

namespace rk {

constexpr int kSellW = 7;        // entries per row of the sliced-ELL copy (7-point operators)
constexpr int kGmTile = 2048;    // rows per tile of the streaming kernels
constexpr int kGmStages = 6;     // ring stages
constexpr int kGmDots = 2 * kGmMax + 2;
constexpr int kGmThreads = 256;
constexpr int kGmRows = kGmTile / kGmThreads;  // rows per thread in a tile
constexpr int kGmSpmvRows = 2;                   // rows whose slots a thread loads together

// Sliced ELL, slices of 32 rows: entry k of row r sits at
// ((r / 32) * kSellW + k) * 32 + r % 32, so the 32 rows of a warp read each
// entry slot with one coalesced access.  Rows with fewer entries are padded
// with (column r, value 0).
__device__ __forceinline__ long long sell_index(long long r, int k) {
  return (((r >> 5) * kSellW + k) << 5) + (r & 31);
}

// The operator's column offsets (col - row) by slot: the kSellW most common
// offsets of the matrix, ascending (a 7-point stencil: -n^2, -n, -1, 0, 1,
// n, n^2).
struct SellPattern {
  int d[kSellW];
};

// Build the sliced-ELL copy (values * lscale rounded to S) from the CSR
// operator; one thread per row.  An entry whose offset is pat.d[k] goes to
// slot k; entries with other offsets (periodic wrap-around) fill the slots
// left free, in order.  A slot still free holds the value 0 with column
// r + pat.d[k] when that is a row of the matrix (else r), so that the slot
// stays on the pattern: multiplying the zero by that entry of z adds nothing
// for finite z.
template <typename S>
__global__ void __launch_bounds__(kThreads) sell_from_csr(CsrView A, const double* __restrict__ vals, double scale,
                                                          long long N, long long Npad, SellPattern pat,
                                                          int* __restrict__ scol, S* __restrict__ sval) {
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < Npad;
       r += (long long)gridDim.x * blockDim.x) {
    const int e0 = r < N ? A.rowptr[r] : 0, e1 = r < N ? A.rowptr[r + 1] : 0;
    int slot_e[kSellW];
    unsigned used = 0u;  // entries placed (bit e - e0)
#pragma unroll
    for (int k = 0; k < kSellW; ++k) {
      slot_e[k] = -1;
      for (int e = e0; e < e1; ++e)
        if (!((used >> (e - e0)) & 1u) && (long long)A.cols[e] - r == pat.d[k]) {
          slot_e[k] = e;
          used |= 1u << (e - e0);
          break;
        }
    }
    for (int e = e0; e < e1; ++e) {
      if ((used >> (e - e0)) & 1u) continue;
      for (int k = 0; k < kSellW; ++k)
        if (slot_e[k] < 0) {
          slot_e[k] = e;
          used |= 1u << (e - e0);
          break;
        }
    }
#pragma unroll
    for (int k = 0; k < kSellW; ++k) {
      const int e = slot_e[k];
      const long long on = r + pat.d[k];
      scol[sell_index(r, k)] = e >= 0 ? A.cols[e] : (int)((on >= 0 && on < N) ? on : (r < N ? r : 0));
      sval[sell_index(r, k)] = nar<S>(e >= 0 ? vals[e] * scale : 0.0);
    }
  }
}

// Bit k of mask[slice] is set when every row r of the 32-row slice has its
// slot-k column at r + pat.d[k]: the product then forms that column instead
// of loading it.  One thread per slice.
__global__ void __launch_bounds__(kThreads) sell_mask(const int* __restrict__ scol, long long nslices, SellPattern pat,
                                                      unsigned* __restrict__ mask) {
  for (long long sl = (long long)blockIdx.x * blockDim.x + threadIdx.x; sl < nslices;
       sl += (long long)gridDim.x * blockDim.x) {
    unsigned m = 0u;
    for (int k = 0; k < kSellW; ++k) {
      bool all = true;
      for (int i = 0; i < 32 && all; ++i) {
        const long long r = sl * 32 + i;
        all = (long long)scol[sell_index(r, k)] == r + pat.d[k];
      }
      if (all) m |= 1u << k;
    }
    mask[sl] = m;
  }
}

__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}

// Ring of kGmStages tiles fed by thread 0.  Items are numbered q = 0, 1, ...
// over the CTA's tiles (NI items per tile); src(q) gives the global tile of
// item q.  wait(q) is bounded; after every thread has consumed item q,
// refill(q) issues item q + kGmStages.  drain() lets copies in flight land.
template <typename B>
struct TileRing {
  B* st;
  uint64_t* bar;
  long long nitems;
  long long issued;
  __device__ B* stage(long long q) const { return st + (q % kGmStages) * (long long)kGmTile; }
  template <typename Src>
  __device__ void issue(long long q, Src src) {
    uint64_t* b = &bar[q % kGmStages];
    mbar_expect_tx(b, (uint32_t)(kGmTile * sizeof(B)));
    bulk_load(stage(q), src(q), (uint32_t)(kGmTile * sizeof(B)), b);
  }
  template <typename Src>
  __device__ void start(Src src) {
    issued = nitems < kGmStages ? nitems : kGmStages;
    if (threadIdx.x == 0)
      for (long long q = 0; q < issued; ++q) issue(q, src);
  }
  __device__ bool wait(long long q) { return mbar_wait(&bar[q % kGmStages], (uint32_t)((q / kGmStages) & 1)); }
  template <typename Src>
  __device__ void refill(Src src) {
    if (threadIdx.x == 0 && issued < nitems) {
      fence_proxy_async();
      issue(issued, src);
    }
    ++issued;
  }
  __device__ void drain() {
    if (threadIdx.x == 0)
      for (long long q = issued - kGmStages; q < issued; ++q)
        if (q >= 0 && q < nitems) (void)mbar_wait(&bar[q % kGmStages], (uint32_t)((q / kGmStages) & 1));
  }
};

// z = M^{-1} u_j (block-Jacobi with per-block inverses, FP16 where flags
// marks a block), u_j unnormalised.
template <typename S, typename B, typename T, int BS, int SEG>
__global__ void __launch_bounds__(kThreads) gm_dc_prec(HeatGeo g, const B* __restrict__ V, long long ldv,
                                                       const S* __restrict__ minv,
                                                       const unsigned char* __restrict__ flags, S* __restrict__ z,
                                                       const GmScalars* sc) {
  if (sc->done || sc->cycle_end || sc->j >= sc->m) return;
  const B* Vj = V + (long long)sc->j * ldv;
  const int nbl = (g.n + BS - 1) / BS;
  RK_SEG_LOOP(g, SEG)
    (void)j;
    (void)k;
    T v[SEG], zv[SEG];
    load_seg<T, B, SEG>(Vj + base, m, v);
    bj_apply_blocks<T, S, BS, SEG>(minv, flags, line, nbl, i0, v, zv);
    store_seg<S, T, SEG>(z + base, m, zv);
  RK_SEG_LOOP_END
}

// Sums of a and b over the warp (fixed shuffle order, the two chains
// interleaved), added by lane 0 to *da and *db.  In the arithmetic type T: on
// this part an FP64 operation costs about 30 FP32 ones, so FP32 paths reduce
// in FP32 and convert to FP64 once per kernel.
template <typename T>
__device__ __forceinline__ void warp_add2(T a, T b, T* da, T* db) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, off);
    b += __shfl_down_sync(0xffffffffu, b, off);
  }
  if ((threadIdx.x & 31) == 0) {
    *da += a;
    *db += b;
  }
}

// Last CTA of gm_dc_arnoldi, all threads: finish column j-1 of the Hessenberg
// matrix with the reorthogonalisation coefficients s (tot[0..j-1]) and
// ||v_j|| (Pythagoras: ||u_j - V s||^2 = u_j.u_j - s.s for orthonormal V),
// rotate it, test convergence, and either end the cycle (back substitution)
// or form the coefficients of gm_dc_update.  tot: s_0..s_{j-1},
// t_0..t_{j-1}, u_j.u_j, u_j.w (shared memory).  work: >= 3 kGmMax + 4
// doubles of shared memory.
__device__ void gm_dc_finish(GmScalars* sc, const double* tot, int j, double* work) {
  __shared__ int s_end;
  __shared__ double s_nrm;
  double* col = work;                  // rotated column j-1 (rows 0..j)
  double* gg = work + kGmMax + 1;      // g = H s (rows 0..j)
  double* yy = work + 2 * kGmMax + 2;  // back substitution
  const int tid = threadIdx.x;
  const int m = sc->m;
  if (tid == 0) {
    double ss = 0.0;
    for (int i = 0; i < j; ++i) ss = fma(tot[i], tot[i], ss);
    const double uu = tot[2 * j], uw = tot[2 * j + 1];
    const double nrm2 = uu - ss;
    s_nrm = nrm2 > 0.0 ? sqrt(nrm2) : 0.0;
    s_end = 0;
    sc->steps += 1;
    if (!isfinite(uu) || !isfinite(uw) || !isfinite(ss)) {
      s_end = 2;  // non-finite: stop, keep x
    } else if (j == 0 && !(s_nrm > 0.0)) {
      s_end = 3;  // zero start vector: x is the solution
    }
  }
  __syncthreads();
  if (s_end >= 2) {
    if (tid == 0) {
      sc->jused = 0;
      sc->cycle_end = 1;
      sc->done = 1;
      sc->status = (s_end == 2) ? 5 : 0;
    }
    return;
  }
  const double nrm = s_nrm;
  if (j > 0) {
    // column j-1: raw entries += s, subdiagonal = nrm; rotated copy in col
    double* Hr = sc->Hraw + (size_t)(j - 1) * (kGmMax + 1);
    for (int i = tid; i <= j; i += blockDim.x) {
      const double v = (i < j) ? Hr[i] + tot[i] : nrm;
      Hr[i] = v;
      col[i] = v;
    }
    __syncthreads();
    if (tid == 0) {
      for (int i = 0; i + 1 < j; ++i) {
        const double t = sc->cs[i] * col[i] + sc->sn[i] * col[i + 1];
        col[i + 1] = -sc->sn[i] * col[i] + sc->cs[i] * col[i + 1];
        col[i] = t;
      }
      const double den = hypot(col[j - 1], col[j]);
      const double c = (den > 0.0) ? col[j - 1] / den : 1.0;
      const double s = (den > 0.0) ? col[j] / den : 0.0;
      sc->cs[j - 1] = c;
      sc->sn[j - 1] = s;
      col[j - 1] = den;
      col[j] = 0.0;
      sc->gv[j] = -s * sc->gv[j - 1];
      sc->gv[j - 1] = c * sc->gv[j - 1];
      const double res = fabs(sc->gv[j]);
      sc->res = res;
      sc->iter += 1;
      const bool conv = res <= sc->thresh;
      const bool bad = !isfinite(res) || !isfinite(den);
      const bool breakdown = !(nrm > 0.0);
      if (conv || bad || breakdown || j >= m || sc->iter >= sc->max_iter) {
        s_end = 1;
        sc->jused = j;
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
    __syncthreads();
    double* Hc = sc->H + (size_t)(j - 1) * (kGmMax + 1);
    for (int i = tid; i <= j; i += blockDim.x) Hc[i] = col[i];
    if (s_end == 1) {
      // back substitution R(0:j, 0:j) y = gv(0:j), column by column
      for (int i = tid; i < j; i += blockDim.x) yy[i] = sc->gv[i];
      __syncthreads();
      for (int i = j - 1; i >= 0; --i) {
        if (tid == 0) {
          const double d = (i == j - 1) ? col[i] : sc->H[(size_t)i * (kGmMax + 1) + i];
          yy[i] = (d != 0.0) ? yy[i] / d : 0.0;
        }
        __syncthreads();
        for (int l = tid; l < i; l += blockDim.x) {
          const double r = (i == j - 1) ? col[l] : sc->H[(size_t)i * (kGmMax + 1) + l];
          yy[l] -= r * yy[i];
        }
        __syncthreads();
      }
      for (int i = tid; i < j; i += blockDim.x) sc->y[i] = yy[i];
      return;
    }
  }
  // coefficients of gm_dc_update: g = H_raw(0:j, 0:j-1) s, projections h of
  // A v_j, c = g / nrm + h; the raw column j is h (finished next step)
  const double inv = 1.0 / nrm;
  for (int l = tid; l <= j; l += blockDim.x) {
    double g = 0.0;
    for (int i = (l > 0 ? l - 1 : 0); i < j; ++i) g = fma(sc->Hraw[(size_t)i * (kGmMax + 1) + l], tot[i], g);
    gg[l] = g;
  }
  __syncthreads();
  __shared__ double s_vjw;
  if (tid == 0) {
    double st = 0.0;
    for (int i = 0; i < j; ++i) st = fma(tot[i], tot[j + i], st);
    s_vjw = (tot[2 * j + 1] - st) * inv;
    sc->inv_nrm = inv;
  }
  __syncthreads();
  double* Hj = sc->Hraw + (size_t)j * (kGmMax + 1);
  for (int l = tid; l <= j; l += blockDim.x) {
    const double h = ((l < j) ? tot[j + l] - gg[l] : s_vjw - gg[l]) * inv;
    Hj[l] = h;
    sc->cv[l] = fma(gg[l], inv, h);
    if (l < j) sc->sv[l] = tot[l];
  }
}

// Shared memory of the streaming kernels: the ring, its barriers, per-warp
// dot accumulators (gm_dc_arnoldi) or coefficients (gm_dc_update).
template <typename B>
__host__ __device__ constexpr size_t gm_ring_bytes() {
  return (size_t)kGmStages * kGmTile * sizeof(B);
}
template <typename B>
__host__ __device__ constexpr size_t gm_dc_smem() {
  // ring, barriers, per-warp accumulators (arithmetic type, at most 8 bytes)
  // that the last CTA reuses for the FP64 totals
  return gm_ring_bytes<B>() + 8 * kGmStages + sizeof(double) * ((kGmThreads / 32) * kGmDots);
}

// Step j, part 2: w = (I - shift L) z on the sliced-ELL copy (values Lhat =
// lscale L in S, cs = shift / lscale; a column is formed from the pattern
// where the slice's mask bit is set, else loaded), stored to wbuf in the basis type; the
// dots s_i, t_i (i < j), u_j.u_j, u_j.w with the basis tiles streamed through
// the ring (u_j first, then v_0 .. v_{j-1}); one grid reduction, then
// gm_dc_finish in the last CTA.  With j = m (the cycle's last column) only
// the dots of u_m are formed (no product).  Persistent grid over tiles.
template <typename S, typename B, typename T>
__global__ void __launch_bounds__(kGmThreads, sizeof(T) == 4 ? 3 : 2) gm_dc_arnoldi(const int* __restrict__ scol,
                                                               const unsigned* __restrict__ smask, SellPattern pat,
                                                               const S* __restrict__ sval, T cs,
                                                               const S* __restrict__ z, B* __restrict__ V,
                                                               long long ldv, B* __restrict__ wbuf, long long N,
                                                               GmScalars* sc, double* partials) {
  if (sc->done || sc->cycle_end) return;
  extern __shared__ __align__(128) unsigned char smem[];
  constexpr int kWarps = kGmThreads / 32;
  __shared__ int am_last;
  B* ring_st = reinterpret_cast<B*>(smem);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + gm_ring_bytes<B>());
  T* acc = reinterpret_cast<T*>(smem + gm_ring_bytes<B>() + 8 * kGmStages);
  const int jj = sc->j;
  const bool spmv = jj < sc->m;
  const int nd = 2 * jj + 2;
  const int NI = jj + 1;
  const long long ntiles = ldv / kGmTile;
  const long long mytiles = (long long)blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int tid = threadIdx.x, warp = tid >> 5;
  for (int i = tid; i < kWarps * nd; i += blockDim.x) acc[i] = T(0);
  if (tid == 0) {
    for (int s = 0; s < kGmStages; ++s) mbar_init(&bar[s], 1);
    mbar_fence_init();
  }
  __syncthreads();
  const B* uj = V + (long long)jj * ldv;
  auto src = [&](long long q) -> const B* {
    const long long t = blockIdx.x + (q / NI) * (long long)gridDim.x;
    const int it = (int)(q % NI);
    const B* vec = (it == 0) ? uj : V + (long long)(it - 1) * ldv;
    return vec + t * kGmTile;
  };
  TileRing<B> ring{ring_st, bar, mytiles * NI, 0};
  ring.start(src);
  long long q = 0;
  bool timed_out = false;
  T* accw = acc + warp * nd;
  for (long long tt = 0; tt < mytiles && !timed_out; ++tt) {
    const long long r0 = (blockIdx.x + tt * (long long)gridDim.x) * kGmTile;
    T w[kGmRows], u[kGmRows];
    if (spmv) {
      // the product for the tile's rows (coalesced slot loads, L2-resident gathers)
#pragma unroll
      for (int h = 0; h < kGmRows; h += kGmSpmvRows) {
        int c[kGmSpmvRows][kSellW];
        T a[kGmSpmvRows][kSellW];
#pragma unroll
        for (int e = 0; e < kGmSpmvRows; ++e) {
          const long long r = r0 + (long long)(h + e) * kGmThreads + tid;
          const unsigned msk = smask[r >> 5];  // one slice per warp: a broadcast load
#pragma unroll
          for (int k = 0; k < kSellW; ++k) {
            c[e][k] = ((msk >> k) & 1u) ? (int)r + pat.d[k] : scol[sell_index(r, k)];
            a[e][k] = wid<T>(sval[sell_index(r, k)]);
          }
        }
#pragma unroll
        for (int e = 0; e < kGmSpmvRows; ++e) {
          const long long r = r0 + (long long)(h + e) * kGmThreads + tid;
          T acc_r = T(0);
#pragma unroll
          for (int k = 0; k < kSellW; ++k) acc_r = fma(a[e][k], wid<T>(z[c[e][k]]), acc_r);
          T v = T(0);
          if (r < N) {
            v = rnd<B, T>(fma(-cs, acc_r, wid<T>(z[r])));
            wbuf[r] = nar<B>(v);
          }
          w[h + e] = v;
        }
      }
    } else {
#pragma unroll
      for (int e = 0; e < kGmRows; ++e) w[e] = T(0);
    }
    for (int it = 0; it < NI; ++it, ++q) {
      const bool ok = ring.wait(q);
      const B* stg = ring.stage(q);
      T pa = T(0), pb = T(0);
      if (it == 0) {
#pragma unroll
        for (int e = 0; e < kGmRows; ++e) {
          u[e] = wid<T>(stg[e * kGmThreads + tid]);
          pa = fma(u[e], u[e], pa);
          pb = fma(u[e], w[e], pb);
        }
        warp_add2(pa, pb, &accw[2 * jj], &accw[2 * jj + 1]);
      } else {
#pragma unroll
        for (int e = 0; e < kGmRows; ++e) {
          const T v = wid<T>(stg[e * kGmThreads + tid]);
          pa = fma(v, u[e], pa);
          pb = fma(v, w[e], pb);
        }
        warp_add2(pa, pb, &accw[it - 1], &accw[jj + it - 1]);
      }
      if (__syncthreads_or(!ok)) {
        timed_out = true;
        break;
      }
      ring.refill(src);
    }
  }
  if (timed_out) {
    ring.drain();
    if (tid == 0) {
      sc->status = 6;
      sc->done = 1;
    }
  }
  __syncthreads();
  for (int i = tid; i < nd; i += blockDim.x) {
    double v = 0.0;
#pragma unroll
    for (int ww = 0; ww < kWarps; ++ww) v += (double)acc[ww * nd + i];
    partials[(size_t)blockIdx.x * kGmDots + i] = v;
  }
  __threadfence();
  __syncthreads();
  if (tid == 0) am_last = (atomicAdd(&sc->ticket, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!am_last) return;
  __threadfence();
  // totals in fixed CTA order: warp w sums dots w, w + kWarps, ...
  double* tot = reinterpret_cast<double*>(acc);
  const int lane = tid & 31;
  for (int i = warp; i < nd; i += kWarps) {
    double a = 0.0;
    for (int b = lane; b < (int)gridDim.x; b += 32) a += __ldcg(partials + (size_t)b * kGmDots + i);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) a += __shfl_down_sync(0xffffffffu, a, off);
    if (lane == 0) tot[i] = a;
  }
  __syncthreads();
  if (tid == 0) sc->ticket = 0u;
  if (sc->status == 6) return;
  gm_dc_finish(sc, tot, jj, reinterpret_cast<double*>(smem));
}

// Step j, part 3: v_j = (u_j - sum_{i<j} s_i v_i) / nrm (normalised, into
// slot j) and u_{j+1} = w / nrm - sum_{i<=j} c_i v_i (into slot j + 1), with
// u_j, w, v_0 .. v_{j-1} streamed through the ring.  The last CTA advances j.
template <typename S, typename B, typename T>
__global__ void __launch_bounds__(kGmThreads, 2) gm_dc_update(B* __restrict__ V, long long ldv,
                                                              const B* __restrict__ wbuf, long long N,
                                                              GmScalars* sc) {
  if (sc->done || sc->cycle_end) return;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ int am_last;
  __shared__ T s_s[kGmMax], s_c[kGmMax + 1];
  B* ring_st = reinterpret_cast<B*>(smem);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + gm_ring_bytes<B>());
  const int jj = sc->j;
  const int NI = jj + 2;
  const long long ntiles = ldv / kGmTile;
  const long long mytiles = (long long)blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int tid = threadIdx.x;
  for (int i = tid; i <= jj; i += blockDim.x) {
    s_c[i] = (T)sc->cv[i];
    if (i < jj) s_s[i] = (T)sc->sv[i];
  }
  const T inv = (T)sc->inv_nrm;
  if (tid == 0) {
    for (int s = 0; s < kGmStages; ++s) mbar_init(&bar[s], 1);
    mbar_fence_init();
  }
  __syncthreads();
  const B* uj = V + (long long)jj * ldv;
  auto src = [&](long long q) -> const B* {
    const long long t = blockIdx.x + (q / NI) * (long long)gridDim.x;
    const int it = (int)(q % NI);
    const B* vec = (it == 0) ? uj : (it == 1) ? wbuf : V + (long long)(it - 2) * ldv;
    return vec + t * kGmTile;
  };
  TileRing<B> ring{ring_st, bar, mytiles * NI, 0};
  ring.start(src);
  long long q = 0;
  bool timed_out = false;
  B* vj = V + (long long)jj * ldv;
  B* un = V + (long long)(jj + 1) * ldv;
  for (long long tt = 0; tt < mytiles && !timed_out; ++tt) {
    const long long r0 = (blockIdx.x + tt * (long long)gridDim.x) * kGmTile;
    T av[kGmRows], au[kGmRows];
    for (int it = 0; it < NI; ++it, ++q) {
      const bool ok = ring.wait(q);
      const B* stg = ring.stage(q);
      if (it == 0) {
#pragma unroll
        for (int e = 0; e < kGmRows; ++e) av[e] = wid<T>(stg[e * kGmThreads + tid]);
      } else if (it == 1) {
#pragma unroll
        for (int e = 0; e < kGmRows; ++e) au[e] = wid<T>(stg[e * kGmThreads + tid]) * inv;
      } else {
        const T si = s_s[it - 2], ci = s_c[it - 2];
#pragma unroll
        for (int e = 0; e < kGmRows; ++e) {
          const T v = wid<T>(stg[e * kGmThreads + tid]);
          av[e] = fma(-si, v, av[e]);
          au[e] = fma(-ci, v, au[e]);
        }
      }
      if (__syncthreads_or(!ok)) {
        timed_out = true;
        break;
      }
      ring.refill(src);
    }
    if (timed_out) break;
    const T cj = s_c[jj];
#pragma unroll
    for (int e = 0; e < kGmRows; ++e) {
      const long long r = r0 + (long long)e * kGmThreads + tid;
      if (r < N) {
        const T v = rnd<B, T>(av[e] * inv);
        vj[r] = nar<B>(v);
        un[r] = nar<B>(fma(-cj, v, au[e]));
      }
    }
  }
  if (timed_out) {
    ring.drain();
    if (tid == 0) {
      sc->status = 6;
      sc->done = 1;
    }
  }
  __syncthreads();
  __threadfence();
  if (tid == 0) am_last = (atomicAdd(&sc->ticket2, 1u) == gridDim.x - 1);
  __syncthreads();
  if (am_last && tid == 0) {
    __threadfence();
    sc->ticket2 = 0u;
    sc->j = jj + 1;
  }
}

}  // namespace rk

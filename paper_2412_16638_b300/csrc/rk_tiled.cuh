// TMA-fed 2.5D CG sweeps for the constant-coefficient heat stencil.
//
// A CTA owns a tile of TY full x-lines (y0 .. y0+TY-1) and marches in z over
// a chunk of planes.  For every plane one elected thread issues 3-D TMA tile
// loads (cp.async.bulk.tensor) of the tile plus its y halo -- one line on
// each side for sweep B (n x (TY+2) x 1), the line above for sweep A
// (n x (TY+1) x 1) -- into a ring of shared-memory stages,
// completion tracked by an mbarrier per stage.  Tiles that reach outside the
// grid are zero-filled by the TMA unit, which is exactly the homogeneous
// Dirichlet boundary, so no boundary test is needed in the stencil.
//
// Sweep A marches down in z and sweep B up, so each starts on the planes that
// the other wrote last, which are still in L2.
//
// Compared with the per-segment kernels, every input element is fetched from
// global memory once per sweep (plus the y halo, shared with the neighbouring
// tile through L2), and loads run two planes ahead of the arithmetic.  The
// preconditioned residual z = D^{-1} r is recomputed from r inside sweep A
// instead of being stored, so one CG iteration moves 8 vectors instead of 9:
//   sweep A reads r, p_old and writes p        (3 vectors)
//   sweep B reads p, r, x and writes r, x      (5 vectors)
#pragma once
#include <cuda.h>

#include "rk_device.cuh"
#include "rk_heat.cuh"

namespace rk {

struct TileGeo {
  int n;    // nodes per direction (n % SEG == 0, n <= 256)
  int tpl;  // threads per x-line = n / SEG
  int ty;   // lines per tile (divides n)
  int nyt;  // tiles in y = n / ty
  int nzc;  // z chunks
};

constexpr int kStagesA = 4;  // input stages of sweep A (r, p_old tiles)
constexpr int kStagesB = 4;  // p-tile stages of sweep B (planes k-1, k, k+1 + one in flight)
constexpr unsigned kWaitSpins = 1u << 24;

__host__ __device__ constexpr size_t align128(size_t v) { return (v + 127) / 128 * 128; }

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Non-blocking probe of the phase (mbarrier.test_wait returns at once, unlike
// try_wait, which may suspend the thread for a hardware-defined time).
__device__ __forceinline__ bool mbar_test_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait: false after kWaitSpins unsuccessful try_wait polls.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  for (unsigned i = 0; i < kWaitSpins; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// The main-loop wait of the sweeps: `limit` = 0 is the default bound above;
// a problem can set a small limit (rk_set_wait_limit) to exercise the
// timeout path, and then each poll is a non-blocking test_wait, so the bound
// counts checks, not hardware suspend windows.  The drain of copies still in
// flight after a timeout always uses mbar_wait with the full bound, so no
// copy lands after the CTA has exited.
__device__ __forceinline__ bool mbar_wait_main(uint64_t* bar, uint32_t parity, unsigned limit) {
  if (limit == 0) return mbar_wait(bar, parity);
  for (unsigned i = 0; i < limit; ++i)
    if (mbar_test_wait(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 3-D tile load (x, y, z are element coordinates; x must be 0 here, which is
// 16-byte aligned; y and z may be out of range and read as zero).
__device__ __forceinline__ void tma_load3(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(
          smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_addr(bar)), "r"(x), "r"(y), "r"(z)
      : "memory");
}

// The same 3-D tile load with an L2 evict-first policy, for data that is dead
// after this read.
__device__ __forceinline__ void tma_load3_evict_first(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y,
                                                      int z) {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1, {%3, "
      "%4, %5}], [%2], %6;" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_addr(bar)), "r"(x), "r"(y), "r"(z), "l"(pol)
      : "memory");
}

// Global segment load/store with the streaming (evict-first) cache policy, for
// x, which the next CG iteration reads only after both sweeps have moved
// 8 vectors through L2.  Falls back to the plain access when the segment is
// not made of aligned 16-byte words.
template <typename T, typename S, int SEG>
__device__ __forceinline__ void ldcs_seg(const S* __restrict__ p, T (&v)[SEG]) {
  constexpr int BYTES = SEG * (int)sizeof(S);
  if constexpr (BYTES % 16 == 0) {
    if ((reinterpret_cast<uintptr_t>(p) & 15) == 0) {
      alignas(16) S tmp[SEG];
#pragma unroll
      for (int w = 0; w < BYTES / 16; ++w) reinterpret_cast<uint4*>(tmp)[w] = __ldcs(reinterpret_cast<const uint4*>(p) + w);
#pragma unroll
      for (int e = 0; e < SEG; ++e) v[e] = wid<T>(tmp[e]);
      return;
    }
  }
  load_seg<T, S, SEG>(p, SEG, v);
}

template <typename S, typename T, int SEG>
__device__ __forceinline__ void stcs_seg(S* __restrict__ p, const T (&v)[SEG]) {
  constexpr int BYTES = SEG * (int)sizeof(S);
  if constexpr (BYTES % 16 == 0) {
    if ((reinterpret_cast<uintptr_t>(p) & 15) == 0) {
      alignas(16) S tmp[SEG];
#pragma unroll
      for (int e = 0; e < SEG; ++e) tmp[e] = nar<S>(v[e]);
#pragma unroll
      for (int w = 0; w < BYTES / 16; ++w) __stcs(reinterpret_cast<uint4*>(p) + w, reinterpret_cast<const uint4*>(tmp)[w]);
      return;
    }
  }
  store_seg<S, T, SEG>(p, SEG, v);
}

// Shared-memory segment load/store.  A 32-byte segment is moved as two
// 16-byte halves; lanes with bit 2 set take the halves in the opposite order,
// so each 8-lane phase touches all 32 banks once (no 2-way conflict between
// lanes 32 bytes apart).  Other segment sizes use the plain vector access.
template <typename T, typename S, int SEG>
__device__ __forceinline__ void lds_seg(const S* p, T (&v)[SEG]) {
  if constexpr (SEG * sizeof(S) == 32) {
    const bool sw = (threadIdx.x & 4) != 0;
    const uint4* q = reinterpret_cast<const uint4*>(p);
    const uint4 a = q[sw ? 1 : 0];
    const uint4 b = q[sw ? 0 : 1];
    alignas(16) S tmp[SEG];
    reinterpret_cast<uint4*>(tmp)[0] = sw ? b : a;
    reinterpret_cast<uint4*>(tmp)[1] = sw ? a : b;
#pragma unroll
    for (int e = 0; e < SEG; ++e) v[e] = wid<T>(tmp[e]);
  } else {
    load_seg<T, S, SEG>(p, SEG, v);
  }
}

template <typename S, typename T, int SEG>
__device__ __forceinline__ void sts_seg(S* p, const T (&v)[SEG]) {
  if constexpr (SEG * sizeof(S) == 32) {
    alignas(16) S tmp[SEG];
#pragma unroll
    for (int e = 0; e < SEG; ++e) tmp[e] = nar<S>(v[e]);
    const bool sw = (threadIdx.x & 4) != 0;
    const uint4 a = reinterpret_cast<const uint4*>(tmp)[0];
    const uint4 b = reinterpret_cast<const uint4*>(tmp)[1];
    uint4* q = reinterpret_cast<uint4*>(p);
    q[sw ? 1 : 0] = sw ? b : a;
    q[sw ? 0 : 1] = sw ? a : b;
  } else {
    store_seg<S, T, SEG>(p, SEG, v);
  }
}

// ----------------------------------------------------------------- sweep A
// Thread rows 0..TY each own one line of the (TY+1)-line tile y0..y0+TY (row
// TY is the halo line above the tile).  The CTA marches down in z from plane
// z1 (the halo plane above its chunk) to z0.  Per plane: p = D^{-1} r +
// beta p_old for the own line, written to a 2-slot ring for the y neighbour;
// after one barrier the owned rows write p and add their share of p.Ap.
// p.Ap needs no full stencil: A = d I + o (sum of neighbours) is symmetric,
// so p.Ap = sum_i p_i (d p_i + 2 o (p_{i+x} + p_{i+y} + p_{i+z})), every grid
// edge counted once, from the element on its lower side (neighbours outside
// the grid are zero).  Only the upper neighbours are needed: the halo is one
// line and one plane.  Last CTA: alpha = r.z / p.Ap.
template <typename S, typename T, int BS, int SEG>
__global__ void __launch_bounds__(320, 2) cg_tiled_a(const __grid_constant__ CUtensorMap tm_r,
                                                  const __grid_constant__ CUtensorMap tm_po, TileGeo tg, T d, T o,
                                                  const __grid_constant__ BjTri<T, BS> tri, S* __restrict__ pnew,
                                                  CgScalars* sc, double* partials) {
  if (sc->done) return;
  extern __shared__ __align__(128) unsigned char smem[];
  const int n = tg.n, TY = tg.ty, R = TY + 1;
  const size_t tile = align128((size_t)R * n * sizeof(S));
  unsigned char* base = smem;
  auto st_r = [&](int s) { return reinterpret_cast<S*>(base + (size_t)s * 2 * tile); };
  auto st_p = [&](int s) { return reinterpret_cast<S*>(base + (size_t)s * 2 * tile + tile); };
  auto ring = [&](int s) { return reinterpret_cast<S*>(base + (size_t)kStagesA * 2 * tile + (size_t)s * tile); };
  uint64_t* bar = reinterpret_cast<uint64_t*>(base + (size_t)(kStagesA * 2 + 2) * tile);
  const int tid = threadIdx.x;
  const int tx = tid % tg.tpl, row = tid / tg.tpl;  // row in 0..TY
  const bool owner = row < TY;
  const int yt = blockIdx.x % tg.nyt, zc = blockIdx.x / tg.nyt;
  const int y0 = yt * TY;
  const int z0 = (int)((long long)zc * n / tg.nzc), z1 = (int)((long long)(zc + 1) * n / tg.nzc);
  const int L = z1 - z0 + 1;  // planes z1, z1-1, .. z0 (downwards: plane z1 - t at step t)
  const T beta = (T)sc->beta;
  const T o2 = o + o;
  const bool first = (sc->iter == 0);
  const unsigned spins = sc->wait_spins;  // 0: default bound
  const uint32_t tx_bytes = (first ? 1u : 2u) * (uint32_t)(R * n * sizeof(S));
  if (tid == 0) {
    for (int s = 0; s < kStagesA; ++s) mbar_init(&bar[s], 1);
    mbar_fence_init();
  }
  __syncthreads();
  auto issue = [&](int t) {
    const int s = t % kStagesA;
    mbar_expect_tx(&bar[s], tx_bytes);
    tma_load3(st_r(s), &tm_r, &bar[s], 0, y0, z1 - t);
    if (!first) tma_load3_evict_first(st_p(s), &tm_po, &bar[s], 0, y0, z1 - t);  // p_old: last use
  };
  if (tid == 0)
    for (int t = 0; t < kStagesA && t < L; ++t) issue(t);
  int issued = (kStagesA < L) ? kStagesA : L;
  const int xs = tx * SEG;
  T pw = T(0);
  T pup[SEG];  // p of the own line one plane up (z + 1)
#pragma unroll
  for (int e = 0; e < SEG; ++e) pup[e] = T(0);
  bool timed_out = false;
  for (int t = 0; t < L; ++t) {
    const int s = t % kStagesA;
    const bool ok = mbar_wait_main(&bar[s], (uint32_t)((t / kStagesA) & 1), spins);
    // p on plane z1-t for the own line
    T pn[SEG];
    {
      T rv[SEG];
      lds_seg<T, S, SEG>(st_r(s) + (size_t)row * n + xs, rv);
      bj_apply_tri<T, BS, SEG>(tri, rv, pn);
      if (!first) {
        T pv[SEG];
        lds_seg<T, S, SEG>(st_p(s) + (size_t)row * n + xs, pv);
#pragma unroll
        for (int e = 0; e < SEG; ++e) pn[e] = fma(beta, pv[e], pn[e]);
      }
#pragma unroll
      for (int e = 0; e < SEG; ++e) pn[e] = rnd<S, T>(pn[e]);
      sts_seg<S, T, SEG>(ring(t & 1) + (size_t)row * n + xs, pn);
    }
    if (__syncthreads_or(!ok)) {
      timed_out = true;
      break;
    }
    // stage s has been read by every thread: refill it
    if (tid == 0 && issued < L) {
      fence_proxy_async();
      issue(issued);
      ++issued;
    }
    if (t >= 1 && owner) {
      // plane z1-t is owned: its edges to the line above (ring), to the next
      // element in x and to the plane above (registers)
      const S* pc = ring(t & 1);
      T up[SEG];
      lds_seg<T, S, SEG>(pc + (size_t)(row + 1) * n + xs, up);
      const T right = (xs + SEG < n) ? wid<T>(pc[(size_t)row * n + xs + SEG]) : T(0);
#pragma unroll
      for (int e = 0; e < SEG; ++e) {
        const T xr = (e + 1 < SEG) ? pn[e + 1] : right;
        const T nb = (xr + up[e]) + pup[e];
        const T w = fma(d, pn[e], o2 * nb);
        pw = fma(pn[e], w, pw);
      }
      const int k = z1 - t;
      store_seg<S, T, SEG>(pnew + ((size_t)k * n + (y0 + row)) * n + xs, SEG, pn);
    }
#pragma unroll
    for (int e = 0; e < SEG; ++e) pup[e] = pn[e];
  }
  if (timed_out) {
    // let copies that are still in flight land before the CTA exits
    if (tid == 0) {
      for (int t = issued - kStagesA; t < issued; ++t)
        if (t >= 0) (void)mbar_wait(&bar[t % kStagesA], (uint32_t)((t / kStagesA) & 1));
      sc->status = 6;
      sc->done = 1;
    }
    __syncthreads();
  }
  double acc[1] = {(double)pw};
  double tot[1];
  if (grid_reduce<1, 0u>(acc, partials, &sc->ticket, tot)) {
    if (sc->status == 6) return;
    sc->pAp = tot[0];
    const double alpha = sc->rz / tot[0];
    sc->alpha = alpha;
    if (!isfinite(tot[0]) || !isfinite(sc->rz)) {
      sc->done = 1;
      sc->status = 5;
    } else if (!(tot[0] > 0.0) || !isfinite(alpha)) {
      sc->done = 1;
      sc->status = 4;
    }
  }
}

// ----------------------------------------------------------------- sweep B
// Thread rows 0..TY-1 own lines y0..y0+TY-1.  p tiles (with y halo) arrive
// through the TMA ring; the own line of each plane is copied to registers
// (z neighbours), the y neighbours of the centre plane are read from its
// stage.  r and x of the next plane are prefetched into registers before
// the wait.  q = A p, r -= alpha q, x += alpha p, z = D^{-1} r (registers),
// partials r.z and r.r.  One barrier per plane.  Last CTA: beta and the
// convergence test.
template <typename S, typename T, int BS, int SEG>
__global__ void __launch_bounds__(256, 2) cg_tiled_b(const __grid_constant__ CUtensorMap tm_p, TileGeo tg, T d, T o,
                                                  const __grid_constant__ BjTri<T, BS> tri,
                                                  typename XOf<S>::type* __restrict__ x, S* __restrict__ r,
                                                  CgScalars* sc, double* partials) {
  using X = typename XOf<S>::type;
  if (sc->done) return;
  extern __shared__ __align__(128) unsigned char smem[];
  const int n = tg.n, TY = tg.ty, R = TY + 2;
  const size_t tile = align128((size_t)R * n * sizeof(S));
  auto st = [&](int s) { return reinterpret_cast<S*>(smem + (size_t)s * tile); };
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + (size_t)kStagesB * tile);
  const int tid = threadIdx.x;
  const int tx = tid % tg.tpl, ly = tid / tg.tpl;
  const int l = ly + 1;  // row of the own line in the tile
  const int yt = blockIdx.x % tg.nyt, zc = blockIdx.x / tg.nyt;
  const int y0 = yt * TY;
  const int z0 = (int)((long long)zc * n / tg.nzc), z1 = (int)((long long)(zc + 1) * n / tg.nzc);
  const int L = z1 - z0 + 2;
  const T alpha = (T)sc->alpha;
  const bool xzero = (sc->iter == 0) && !sc->warm;  // x = 0 at the first sweep of a cold start
  const unsigned spins = sc->wait_spins;  // 0: default bound
  const uint32_t tx_bytes = (uint32_t)(R * n * sizeof(S));
  if (tid == 0) {
    for (int s = 0; s < kStagesB; ++s) mbar_init(&bar[s], 1);
    mbar_fence_init();
  }
  __syncthreads();
  auto issue = [&](int t) {
    const int s = t % kStagesB;
    mbar_expect_tx(&bar[s], tx_bytes);
    tma_load3_evict_first(st(s), &tm_p, &bar[s], 0, y0 - 1, z0 - 1 + t);
  };
  if (tid == 0)
    for (int t = 0; t < kStagesB && t < L; ++t) issue(t);
  int issued = (kStagesB < L) ? kStagesB : L;
  const int xs = tx * SEG;
  const size_t line_off = (size_t)(y0 + ly) * n + xs;
  // r and x of the first owned plane; later planes are fetched one plane ahead
  T rn[SEG], xn[SEG];
  load_seg<T, S, SEG>(r + (size_t)z0 * n * n + line_off, SEG, rn);
  if (!xzero) {
    ldcs_seg<T, X, SEG>(x + (size_t)z0 * n * n + line_off, xn);
  } else {
#pragma unroll
    for (int e = 0; e < SEG; ++e) xn[e] = T(0);
  }
  T pprev[SEG], pcur[SEG];
#pragma unroll
  for (int e = 0; e < SEG; ++e) pprev[e] = pcur[e] = T(0);
  T rz = T(0), rr = T(0);
  bool timed_out = false;
  for (int t = 0; t < L; ++t) {
    // r and x of the plane this iteration outputs (z0+t-2) were fetched one
    // plane earlier; fetch the next plane's before waiting for the tile
    T rv[SEG], xv[SEG];
    const int k = z0 + t - 2;
    if (t >= 2) {
#pragma unroll
      for (int e = 0; e < SEG; ++e) {
        rv[e] = rn[e];
        xv[e] = xn[e];
      }
      if (k + 1 < z1) {
        load_seg<T, S, SEG>(r + (size_t)(k + 1) * n * n + line_off, SEG, rn);
        if (!xzero) ldcs_seg<T, X, SEG>(x + (size_t)(k + 1) * n * n + line_off, xn);
      }
    }
    const int s = t % kStagesB;
    const bool ok = mbar_wait_main(&bar[s], (uint32_t)((t / kStagesB) & 1), spins);
    T pn[SEG];
    lds_seg<T, S, SEG>(st(s) + (size_t)l * n + xs, pn);
    if (t >= 2) {
      const S* pc = st((t - 1) % kStagesB);
      T a[SEG], b[SEG];
      lds_seg<T, S, SEG>(pc + (size_t)(l - 1) * n + xs, a);
      lds_seg<T, S, SEG>(pc + (size_t)(l + 1) * n + xs, b);
      const T left = (xs > 0) ? wid<T>(pc[(size_t)l * n + xs - 1]) : T(0);
      const T right = (xs + SEG < n) ? wid<T>(pc[(size_t)l * n + xs + SEG]) : T(0);
#pragma unroll
      for (int e = 0; e < SEG; ++e) {
        const T xl = (e > 0) ? pcur[e - 1] : left;
        const T xr = (e + 1 < SEG) ? pcur[e + 1] : right;
        const T nb = ((xl + xr) + (a[e] + b[e])) + (pprev[e] + pn[e]);
        const T w = fma(d, pcur[e], o * nb);
        rv[e] = rnd<S, T>(fma(-alpha, w, rv[e]));
        xv[e] = fma(alpha, pcur[e], xv[e]);
      }
      T zv[SEG];
      bj_apply_tri<T, BS, SEG>(tri, rv, zv);
#pragma unroll
      for (int e = 0; e < SEG; ++e) {
        zv[e] = rnd<S, T>(zv[e]);
        rz = fma(rv[e], zv[e], rz);
        rr = fma(rv[e], rv[e], rr);
      }
      store_seg<S, T, SEG>(r + (size_t)k * n * n + line_off, SEG, rv);
      stcs_seg<X, T, SEG>(x + (size_t)k * n * n + line_off, xv);
    }
#pragma unroll
    for (int e = 0; e < SEG; ++e) {
      pprev[e] = pcur[e];
      pcur[e] = pn[e];
    }
    if (__syncthreads_or(!ok)) {
      timed_out = true;
      break;
    }
    // stage (t-1) % kStagesB is no longer read (its centre-plane role ends here)
    if (tid == 0 && t >= 1 && issued < L) {
      fence_proxy_async();
      issue(issued);
      ++issued;
    }
  }
  if (timed_out) {
    if (tid == 0) {
      for (int t = issued - kStagesB; t < issued; ++t)
        if (t >= 0) (void)mbar_wait(&bar[t % kStagesB], (uint32_t)((t / kStagesB) & 1));
      sc->status = 6;
      sc->done = 1;
    }
    __syncthreads();
  }
  double acc[2] = {(double)rz, (double)rr};
  double tot[2];
  if (grid_reduce<2, 0u>(acc, partials, &sc->ticket, tot)) {
    if (sc->status == 6) return;
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

// Shared-memory bytes of the two sweeps.
template <typename S, typename T, int BS>
__host__ constexpr size_t tiled_smem_a(int n, int ty) {
  return (size_t)(kStagesA * 2 + 2) * align128((size_t)(ty + 1) * n * sizeof(S)) + 8 * kStagesA;
}
template <typename S, typename T, int BS>
__host__ constexpr size_t tiled_smem_b(int n, int ty) {
  return (size_t)kStagesB * align128((size_t)(ty + 2) * n * sizeof(S)) + 8 * kStagesB;
}

}  // namespace rk

// Fast-diagonalization preconditioner of the heat stage matrix on the
// 5th-generation tensor cores (Sec. 3, Eqs. preconbasic, Pinvform,
// TensorDecomp; the tensor operations T_R, T_M, T_L of Sec. 4).
//
// For the constant-coefficient system I - s L with L = kappa/h^2 times the
// 7-point Laplacian, the one-dimensional factors share the orthonormal sine
// basis Q_jk = sqrt(2/(n+1)) sin((j+1)(k+1) pi/(n+1)) (Q = Q^T = Q^-1) and
// P_D = 1 + c (mu_i + mu_j + mu_k), c = s kappa/h^2, mu_k = 4 sin^2((k+1) pi /
// (2(n+1))).  P^-1 = (Q (x) Q (x) Q) P_D^-1 (Q (x) Q (x) Q) is exact.
//
// Each tensor operation is one pass of a persistent GEMM over the vector
// viewed as an (n^2 x n) row-major matrix X (rows = the two slow indices,
// columns = the fastest index):  Y = X Q^T, a K-major x K-major product.
// The epilogue stores Y transposed, out[j n^2 + m] = Y[m][j], which moves the
// contracted index to the slowest position.  Three passes therefore contract
// x, then y, then z, and return the vector to its lexicographic layout:
//   [z][y][x] -> [x'][z][y] -> [y'][x'][z] -> [z'][y'][x'].
// Unlike the paper's three strided kernels (one per T), every pass reads and
// writes with unit stride and contracts on the tensor cores.
//
// n <= 128: one CTA per SM, persistent over 128-row tiles (fdm_pass).  Warp 0
// issues TMA loads (Q once, then 128 x 128-byte K blocks of X into a ring of
// stages); warp 1 owns the tensor memory and issues tcgen05.mma with the
// accumulator in TMEM (two accumulators, so the epilogue of one tile overlaps
// the MMAs of the next); warps 2-17 read the accumulator with tcgen05.ld and
// store (four warps per TMEM lane quadrant, every fourth 16-column chunk each,
// so the stores of one hide the latency of the others).  The ring holds as many
// 16 KB X stages as shared memory allows beside Q, up to 6.
// 128 < n <= 256: Q (up to 256 KB) no longer fits one CTA's shared memory,
// and the pass runs on CTA pairs with tcgen05.mma.cta_group::2 (fdm_pass_pair
// below), each CTA holding one N half of Q.
// Every mbarrier wait is bounded; a wait that runs out sets a shared flag that
// stops the other roles, the CTA lets its copies and MMAs land, frees its
// tensor memory and reports status 6.
//
// Storage float runs kind::tf32, __half and __nv_bfloat16 run kind::f16 with
// the same type for both operands; accumulation is FP32 in TMEM.
#pragma once
#include <cuda.h>

#include <type_traits>

#include "rk_device.cuh"
#include "rk_fdm_geo.h"
#include "rk_heat.cuh"
#include "rk_tiled.cuh"

namespace rk {

constexpr int kFdmMaxStages = 6;  // K-block stages of X (ring depth set per problem)
constexpr int kFdmEpiWarps = 16;   // epilogue warps: four per TMEM lane quadrant
constexpr int kFdmThreads = 32 * (2 + kFdmEpiWarps);
constexpr int kFdmRows = 128;      // rows per tile (TMEM lanes)
constexpr int kFdmTmemCols = 256;  // two FP32 accumulators of up to 128 columns
constexpr uint32_t kFdmStageBytes = kFdmRows * 128;

enum FdmMode { kFdmPlain = 0, kFdmScale = 1, kFdmDot = 2 };

// Dynamic shared memory: 1 KB alignment slack, Q tile, X stages, barriers.
__host__ __device__ constexpr size_t fdm_smem_bytes(int nt, int kblocks, int stages) {
  return 1024 + (size_t)kblocks * nt * 128 + (size_t)stages * kFdmStageBytes + 512;
}

// ---------------------------------------------------------------- PTX wrappers
__device__ __forceinline__ void tma_load2(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
          smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_addr(bar)), "r"(x), "r"(y)
      : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// Bounded wait that also gives up once another role has failed.
__device__ __forceinline__ bool fdm_wait(uint64_t* bar, uint32_t parity, volatile int* fail) {
  for (unsigned i = 0; i < kWaitSpins; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 63u) == 63u && *fail) return false;
  }
  *fail = 1;
  return false;
}

// Shared-memory matrix descriptor of a K-major tile with 128-byte swizzle:
// rows of 128 bytes, 8-row groups 1024 bytes apart (stride byte offset),
// descriptor version 1, swizzle mode 2 (128 B).  The tile base is 1024-aligned.
__device__ __forceinline__ uint64_t fdm_desc(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Instruction descriptor: FP32 accumulator, A/B format, both K-major, N, M=128.
template <typename S>
__host__ __device__ constexpr uint32_t fdm_idesc(int nt) {
  constexpr uint32_t fmt = std::is_same<S, float>::value ? 2u : (std::is_same<S, __half>::value ? 0u : 1u);
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(nt >> 3) << 17) | ((uint32_t)(kFdmRows >> 4) << 24);
}

template <typename S>
__device__ __forceinline__ void fdm_mma(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  if constexpr (std::is_same<S, float>::value) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
  }
}

__device__ __forceinline__ void fdm_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 16 consecutive FP32 accumulator columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// ---------------------------------------------------------------- the pass
// out[j*rows + m] = sum_k in[m*n + k] Q[j*n + k]     (j < n, m < rows)
// mode kFdmScale: divided by P_D = 1 + c (mu[m / n] + mu[m % n] + mu[j]).
// mode kFdmDot:   also r.z over the output (z = out, r = rdot, same layout);
//                 the last CTA turns it into the CG scalars: beta is rescaled
//                 from the unpreconditioned r.r the sweep left behind, rz set.
// cg != 0: the pass belongs to a CG solve and returns at once when sc->done.
// A timed-out wait sets sc->status = 6 and sc->done = 1 in either case.
template <typename S>
__global__ void __launch_bounds__(kFdmThreads, 1)
    fdm_pass(const __grid_constant__ CUtensorMap tm_in, const __grid_constant__ CUtensorMap tm_q, FdmGeo fg, int mode,
             float c, const float* __restrict__ mu, S* __restrict__ out, const S* __restrict__ rdot, int cg,
             CgScalars* sc, double* partials) {
  if (cg && sc->done) return;
  extern __shared__ unsigned char fdm_smem_raw[];
  // 1024-byte alignment of the shared-window offset (128-byte swizzle atoms)
  unsigned char* sm = fdm_smem_raw + ((1024u - (smem_addr(fdm_smem_raw) & 1023u)) & 1023u);
  const uint32_t qbytes = (uint32_t)fg.kblocks * fg.nt * 128;
  unsigned char* sQ = sm;
  unsigned char* sX = sm + qbytes;
  const int NS = fg.stages;
  uint64_t* bars = reinterpret_cast<uint64_t*>(sX + (size_t)NS * kFdmStageBytes);
  uint64_t* full = bars;                       // [NS] X stage landed
  uint64_t* empty = bars + kFdmMaxStages;      // [NS] X stage consumed by the MMAs
  uint64_t* qfull = bars + 2 * kFdmMaxStages;  // Q tile landed
  uint64_t* accfull = qfull + 1;            // [2] accumulator ready
  uint64_t* accempty = qfull + 3;           // [2] accumulator drained
  uint64_t* mmadone = qfull + 5;            // every MMA of the CTA finished
  uint32_t* tholder = reinterpret_cast<uint32_t*>(qfull + 6);
  volatile int* fail = reinterpret_cast<volatile int*>(qfull + 7);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int total = fg.mtiles;
  constexpr int KB = 128 / (int)sizeof(S);  // elements per 128-byte K block

  if (threadIdx.x == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(qfull, 1);
    mbar_init(&accfull[0], 1);
    mbar_init(&accfull[1], 1);
    mbar_init(&accempty[0], kFdmEpiWarps * 32);
    mbar_init(&accempty[1], kFdmEpiWarps * 32);
    mbar_init(mmadone, 1);
    *fail = 0;
    mbar_fence_init();
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tholder)),
                 "r"(kFdmTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    tc_fence_before();
  }
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = *tholder;

  float dot = 0.f;
  if (warp == 0) {
    if (lane == 0) {
      // ---- TMA producer
      mbar_expect_tx(qfull, qbytes);
      for (int kb = 0; kb < fg.kblocks; ++kb)
        tma_load2(sQ + (size_t)kb * fg.nt * 128, &tm_q, qfull, kb * KB, 0);
      uint32_t it = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < total && ok; t += gridDim.x) {
        const int mt = t;
        for (int kb = 0; kb < fg.kblocks; ++kb, ++it) {
          const int s = (int)(it % NS);
          if (!fdm_wait(&empty[s], ((it / NS) & 1u) ^ 1u, fail)) {
            ok = false;
            break;
          }
          mbar_expect_tx(&full[s], kFdmStageBytes);
          tma_load2(sX + (size_t)s * kFdmStageBytes, &tm_in, &full[s], kb * KB, mt * kFdmRows);
        }
      }
      // every copy issued must land before the CTA exits
      (void)mbar_wait(qfull, 0);
      const uint32_t first = it > (uint32_t)NS ? it - NS : 0u;
      for (uint32_t j = first; j < it; ++j) (void)mbar_wait(&full[j % NS], (j / NS) & 1u);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---- MMA issuer
      const uint32_t idesc = fdm_idesc<S>(fg.nt);
      bool ok = fdm_wait(qfull, 0, fail);
      tc_fence_after();
      const uint32_t q0 = smem_addr(sQ), x0 = smem_addr(sX);
      uint32_t it = 0, lt = 0;
      for (int t = blockIdx.x; t < total && ok; t += gridDim.x, ++lt) {
        const uint32_t acc = lt & 1u;
        if (!fdm_wait(&accempty[acc], ((lt >> 1) & 1u) ^ 1u, fail)) break;
        tc_fence_after();
        const uint32_t d = tbase + acc * 128u;
        for (int kb = 0; kb < fg.kblocks; ++kb, ++it) {
          const int s = (int)(it % NS);
          if (!fdm_wait(&full[s], (it / NS) & 1u, fail)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint64_t ad = fdm_desc(x0 + (uint32_t)s * kFdmStageBytes);
          const uint64_t bd = fdm_desc(q0 + (uint32_t)kb * fg.nt * 128u);
#pragma unroll
          for (int k = 0; k < 4; ++k)  // 32 bytes of K per instruction
            fdm_mma<S>(d, ad + (uint64_t)(2 * k), bd + (uint64_t)(2 * k), idesc, (kb | k) != 0);
          fdm_commit(&empty[s]);
        }
        if (ok) fdm_commit(&accfull[acc]);
      }
      // all MMAs issued by this thread complete before the commit below arrives
      fdm_commit(mmadone);
      (void)mbar_wait(mmadone, 0);
    }
  } else {
    // ---- epilogue: warp w owns TMEM lane quadrant w % 4 (the hardware
    // restriction) and every fourth 16-column chunk, starting at (w - 2) / 4
    const int quad = warp & 3;
    const int part = (warp - 2) >> 2;  // 0..3
    const int row = quad * 32 + lane;
    float dacc[4] = {0.f, 0.f, 0.f, 0.f};
    uint32_t lt = 0;
    for (int t = blockIdx.x; t < total; t += gridDim.x, ++lt) {
      const uint32_t acc = lt & 1u;
      // warp-uniform: tcgen05.ld below is a warp-collective instruction
      if (!__all_sync(0xffffffffu, fdm_wait(&accfull[acc], (lt >> 1) & 1u, fail))) break;
      tc_fence_after();
      const int m = t * kFdmRows + row;
      const bool mrow = m < fg.rows;
      float cab = 0.f;
      if (mode == kFdmScale && mrow) cab = fmaf(c, mu[m / fg.n] + mu[m % fg.n], 1.0f);
      for (int c0 = 16 * part; c0 < fg.nt; c0 += 64) {
        float rv[16];
        if (mode == kFdmDot) {  // r loads in flight during the TMEM read
#pragma unroll
          for (int jj = 0; jj < 16; ++jj) {
            const int j = c0 + jj;
            rv[jj] = (mrow && j < fg.n) ? wid<float>(rdot[(size_t)j * fg.rows + m]) : 0.f;
          }
        }
        float v[16];
        tmem_ld16(tbase + ((uint32_t)(quad * 32) << 16) + acc * 128u + (uint32_t)c0, v);
#pragma unroll
        for (int jj = 0; jj < 16; ++jj) {
          const int j = c0 + jj;
          if (mrow && j < fg.n) {
            float y = v[jj];
            // P_D >= 1: the fast division's 2-ulp error is far below TF32/FP16 rounding
            if (mode == kFdmScale) y = __fdividef(y, fmaf(c, mu[j], cab));
            const S ys = nar<S>(y);
            out[(size_t)j * fg.rows + m] = ys;
            if (mode == kFdmDot) dacc[jj & 3] = fmaf(rv[jj], wid<float>(ys), dacc[jj & 3]);
          }
        }
      }
      tc_fence_before();
      mbar_arrive(&accempty[acc]);
    }
    dot = (dacc[0] + dacc[1]) + (dacc[2] + dacc[3]);
  }
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(kFdmTmemCols) : "memory");
  }
  const bool failed = *fail != 0;
  if (failed && threadIdx.x == 0) {
    sc->status = 6;
    sc->done = 1;
  }
  if (mode != kFdmDot) return;
  double a[1] = {(double)dot};
  double tot[1];
  if (grid_reduce<1, 0u>(a, partials, &sc->ticket, tot)) {
    if (sc->status == 6) return;
    const double rz = tot[0];
    if (sc->iter > 0) sc->beta = sc->beta * (rz / sc->rz);
    sc->rz = rz;
    if (!isfinite(rz)) {
      sc->done = 1;
      sc->status = 5;
    } else if (!(rz > 0.0)) {
      sc->done = 1;
      sc->status = 4;
    }
  }
}

// ------------------------------------------------------------- the CTA pair
// For 128 < n <= 256 the pass runs on CTA pairs (clusters of two) with
// tcgen05.mma.cta_group::2.  A pair owns 256-row tiles of X: CTA rank r holds
// rows 128 r .. 128 r + 127 of each tile (its half of the A operand) and the
// N half r of Q (its half of the B operand, loaded once), and its tensor
// memory receives its 128 rows x all N columns.  Every X tile then crosses
// from L2 to shared memory once; with one CTA per N half (all that shared
// memory holds of Q) it crossed twice.  Each CTA's epilogue has 256 columns
// per tile, so it runs 16 warps, four per TMEM lane quadrant.
//
// Rank 0 issues the MMAs.  Each CTA loads its own operands with TMA, and
// every copy of the pair completes on rank 0's barriers (rank 0 expects the
// bytes of both; rank 1's copies name rank 0's barrier, the .cta_group::2
// form).  The MMA completions arrive on both CTAs' barriers (multicast
// commit); both CTAs' epilogue warps release an accumulator on rank 0's
// barrier.  These hand-offs order tensor-memory accesses only (tcgen05 fences
// around a CTA-scope arrive and wait), so the epilogue's global stores never
// wait for a cluster-scope release.  A wait that runs out sets the failure
// flag of both CTAs, so the peer stops too.  At the end rank 0 learns how many
// copies rank 1 issued and waits for every copy of the pair to land, and both
// CTAs meet at a cluster barrier before freeing the tensor memory.
constexpr int kFdmPairRows = 2 * kFdmRows;  // rows of X per pair tile
constexpr int kFdmPairEpiWarps = 16;        // epilogue warps: four per TMEM lane quadrant
constexpr int kFdmPairThreads = 32 * (2 + kFdmPairEpiWarps);
constexpr int kFdmPairTmemCols = 512;       // two FP32 accumulators of up to 256 columns

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Shared::cluster address of the same shared variable in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t cluster_addr(const void* p, uint32_t rank) {
  uint32_t a;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(a) : "r"(smem_addr(p)), "r"(rank));
  return a;
}

// Arrive on a barrier of either CTA of the cluster (CTA-scope release).
__device__ __forceinline__ void mbar_arrive_remote(uint32_t cluster_bar) {
  asm volatile("mbarrier.arrive.shared::cluster.b64 _, [%0];" ::"r"(cluster_bar) : "memory");
}

// Completes `bytes` of the current phase's transaction count without a copy
// (accounts for a copy that was expected but never issued).
__device__ __forceinline__ void mbar_complete_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.complete_tx.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void st_cluster_u32(uint32_t cluster_addr_, uint32_t v) {
  asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(cluster_addr_), "r"(v) : "memory");
}

// Bounded wait of the pair kernel: gives up once either CTA has failed, and
// a wait that runs out marks both CTAs failed.
__device__ __forceinline__ bool pair_wait(uint64_t* bar, uint32_t parity, volatile int* fail, uint32_t peer_fail) {
  for (unsigned i = 0; i < kWaitSpins; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 63u) == 63u && *fail) return false;
  }
  *fail = 1;
  st_cluster_u32(peer_fail, 1u);
  return false;
}

// Full bound, for draining copies in flight (no early exit on failure).
__device__ __forceinline__ bool pair_drain(uint64_t* bar, uint32_t parity) {
  for (unsigned i = 0; i < kWaitSpins; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// 2-D tile load by either CTA of a pair onto a barrier of rank 0 (its
// shared::cluster address): the copy's bytes complete there.
__device__ __forceinline__ void tma_load2_pair(void* dst, const CUtensorMap* map, uint32_t cluster_bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], "
      "[%2];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(cluster_bar), "r"(x), "r"(y)
      : "memory");
}

template <typename S>
__device__ __forceinline__ void fdm_mma2(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  if constexpr (std::is_same<S, float>::value) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
  }
}

// Arrives once on the barrier at this offset in both CTAs of the pair when
// the MMAs issued so far have completed.
__device__ __forceinline__ void fdm_commit2_both(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
          smem_addr(bar)),
      "h"((unsigned short)3)
      : "memory");
}

__device__ __forceinline__ void fdm_commit2_own(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
               : "memory");
}

// Instruction descriptor of the pair MMA: M = 256 rows (128 per CTA), N = nt.
template <typename S>
__host__ __device__ constexpr uint32_t fdm_idesc2(int nt) {
  constexpr uint32_t fmt = std::is_same<S, float>::value ? 2u : (std::is_same<S, __half>::value ? 0u : 1u);
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(nt >> 3) << 17) | ((uint32_t)(kFdmPairRows >> 4) << 24);
}

// The pass of fdm_pass on CTA pairs.  fg.nt is the full N (a multiple of 16,
// <= 256; each CTA holds nt/2 rows of Q), fg.mtiles counts 256-row tiles.
template <typename S>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kFdmPairThreads, 1)
    fdm_pass_pair(const __grid_constant__ CUtensorMap tm_in, const __grid_constant__ CUtensorMap tm_q, FdmGeo fg,
                  int mode, float c, const float* __restrict__ mu, S* __restrict__ out, const S* __restrict__ rdot,
                  int cg, CgScalars* sc, double* partials) {
  extern __shared__ unsigned char fdm_smem_raw[];
  unsigned char* sm = fdm_smem_raw + ((1024u - (smem_addr(fdm_smem_raw) & 1023u)) & 1023u);
  const int nh = fg.nt / 2;  // Q rows (N columns) held by each CTA
  const uint32_t qbytes = (uint32_t)fg.kblocks * nh * 128;
  unsigned char* sQ = sm;
  unsigned char* sX = sm + qbytes;
  const int NS = fg.stages;
  uint64_t* bars = reinterpret_cast<uint64_t*>(sX + (size_t)NS * kFdmStageBytes);
  uint64_t* landed = bars;                       // [NS] rank 0: the stage of both CTAs landed
  uint64_t* empty = bars + kFdmMaxStages;        // [NS] stage consumed by the pair's MMAs (both CTAs)
  uint64_t* qlanded = bars + 2 * kFdmMaxStages;  // rank 0: both Q halves landed
  uint64_t* accfull = qlanded + 1;               // [2] accumulator ready (both CTAs)
  uint64_t* accempty = qlanded + 3;              // [2] rank 0: accumulator drained by both CTAs
  uint64_t* mmadone = qlanded + 5;               // rank 0: every MMA finished
  uint32_t* tholder = reinterpret_cast<uint32_t*>(qlanded + 6);
  volatile int* fail = reinterpret_cast<volatile int*>(tholder + 1);
  volatile int* skip = reinterpret_cast<volatile int*>(tholder + 2);
  volatile uint32_t* peer_issued = reinterpret_cast<volatile uint32_t*>(tholder + 3);  // rank 0: rank 1's copies

  const uint32_t rank = cluster_rank();
  const uint32_t peer = rank ^ 1u;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int pair_id = (int)(blockIdx.x >> 1), npairs = (int)(gridDim.x >> 1);
  const int total = fg.mtiles;
  constexpr int KB = 128 / (int)sizeof(S);
  const uint32_t peer_fail = cluster_addr((const void*)fail, peer);

  if (threadIdx.x == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(&landed[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(qlanded, 1);
    mbar_init(&accfull[0], 1);
    mbar_init(&accfull[1], 1);
    mbar_init(&accempty[0], 2 * kFdmPairEpiWarps);
    mbar_init(&accempty[1], 2 * kFdmPairEpiWarps);
    mbar_init(mmadone, 1);
    *fail = 0;
    mbar_fence_init();
  }
  cluster_sync();  // both CTAs running, barriers initialised: remote access is safe from here
  if (threadIdx.x == 0 && rank == 0) {  // one decision for the pair: both CTAs return, or neither
    const uint32_t v = (cg && sc->done) ? 1u : 0u;
    *skip = (int)v;
    st_cluster_u32(cluster_addr((const void*)skip, 1u), v);
  }
  cluster_sync();
  if (*skip) return;
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tholder)),
                 "r"(kFdmPairTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
    tc_fence_before();
  }
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = *tholder;

  float dot = 0.f;
  uint32_t issued = 0;  // X copies issued by this CTA's producer
  if (warp == 0) {
    if (lane == 0) {
      // ---- TMA producer (both CTAs): own Q half once, own 128 rows of each
      // tile; the bytes of both CTAs complete on rank 0's barriers
      const uint32_t qbar = cluster_addr(qlanded, 0u);
      if (rank == 0) mbar_expect_tx(qlanded, 2u * qbytes);
      for (int kb = 0; kb < fg.kblocks; ++kb)
        tma_load2_pair(sQ + (size_t)kb * nh * 128, &tm_q, qbar, kb * KB, (int)rank * nh);
      bool ok = true;
      for (int t = pair_id; t < total && ok; t += npairs) {
        for (int kb = 0; kb < fg.kblocks; ++kb, ++issued) {
          const int s = (int)(issued % NS);
          if (!pair_wait(&empty[s], ((issued / NS) & 1u) ^ 1u, fail, peer_fail) || *fail) {
            ok = false;
            break;
          }
          if (rank == 0) mbar_expect_tx(&landed[s], 2u * kFdmStageBytes);
          tma_load2_pair(sX + (size_t)s * kFdmStageBytes, &tm_in, cluster_addr(&landed[s], 0u), kb * KB,
                         t * kFdmPairRows + (int)rank * kFdmRows);
        }
      }
      if (rank == 1) st_cluster_u32(cluster_addr((const void*)peer_issued, 0u), issued);
    }
  } else if (warp == 1) {
    if (lane == 0 && rank == 0) {
      // ---- MMA issuer (rank 0): both CTAs' stages, pair MMAs, multicast commits
      const uint32_t idesc = fdm_idesc2<S>(fg.nt);
      bool ok = pair_wait(qlanded, 0, fail, peer_fail);
      tc_fence_after();
      const uint32_t q0 = smem_addr(sQ), x0 = smem_addr(sX);
      uint32_t it = 0, lt = 0;
      for (int t = pair_id; t < total && ok; t += npairs, ++lt) {
        const uint32_t acc = lt & 1u;
        if (!pair_wait(&accempty[acc], ((lt >> 1) & 1u) ^ 1u, fail, peer_fail)) break;
        tc_fence_after();
        const uint32_t d = tbase + acc * 256u;
        for (int kb = 0; kb < fg.kblocks; ++kb, ++it) {
          const int s = (int)(it % NS);
          if (!pair_wait(&landed[s], (it / NS) & 1u, fail, peer_fail)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint64_t ad = fdm_desc(x0 + (uint32_t)s * kFdmStageBytes);
          const uint64_t bd = fdm_desc(q0 + (uint32_t)kb * nh * 128u);
#pragma unroll
          for (int k = 0; k < 4; ++k)  // 32 bytes of K per instruction
            fdm_mma2<S>(d, ad + (uint64_t)(2 * k), bd + (uint64_t)(2 * k), idesc, (kb | k) != 0);
          fdm_commit2_both(&empty[s]);
        }
        if (ok) fdm_commit2_both(&accfull[acc]);
      }
      // all MMAs issued by this thread complete before the commit below arrives
      fdm_commit2_own(mmadone);
      (void)pair_drain(mmadone, 0);
    }
  } else {
    // ---- epilogue (both CTAs): warp w owns TMEM lane quadrant w % 4 and every
    // fourth 16-column chunk, starting at (w - 2) / 4
    const int quad = warp & 3;
    const int part = (warp - 2) >> 2;  // 0..3
    const int row = quad * 32 + lane;
    const uint32_t release0 = cluster_addr(&accempty[0], 0u), release1 = cluster_addr(&accempty[1], 0u);
    float dacc[4] = {0.f, 0.f, 0.f, 0.f};
    uint32_t lt = 0;
    for (int t = pair_id; t < total; t += npairs, ++lt) {
      const uint32_t acc = lt & 1u;
      if (!__all_sync(0xffffffffu, pair_wait(&accfull[acc], (lt >> 1) & 1u, fail, peer_fail))) break;
      tc_fence_after();
      const int m = t * kFdmPairRows + (int)rank * kFdmRows + row;
      const bool mrow = m < fg.rows;
      float cab = 0.f;
      if (mode == kFdmScale && mrow) cab = fmaf(c, mu[m / fg.n] + mu[m % fg.n], 1.0f);
      for (int c0 = 16 * part; c0 < fg.nt; c0 += 64) {
        float rv[16];
        if (mode == kFdmDot) {
#pragma unroll
          for (int jj = 0; jj < 16; ++jj) {
            const int j = c0 + jj;
            rv[jj] = (mrow && j < fg.n) ? wid<float>(rdot[(size_t)j * fg.rows + m]) : 0.f;
          }
        }
        float v[16];
        tmem_ld16(tbase + ((uint32_t)(quad * 32) << 16) + acc * 256u + (uint32_t)c0, v);
#pragma unroll
        for (int jj = 0; jj < 16; ++jj) {
          const int j = c0 + jj;
          if (mrow && j < fg.n) {
            float y = v[jj];
            if (mode == kFdmScale) y = __fdividef(y, fmaf(c, mu[j], cab));
            const S ys = nar<S>(y);
            out[(size_t)j * fg.rows + m] = ys;
            if (mode == kFdmDot) dacc[jj & 3] = fmaf(rv[jj], wid<float>(ys), dacc[jj & 3]);
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive_remote(acc ? release1 : release0);
    }
    dot = (dacc[0] + dacc[1]) + (dacc[2] + dacc[3]);
  }
  __syncthreads();
  cluster_sync();  // both producers done; rank 1's copy count visible to rank 0
  if (rank == 0 && warp == 0 && lane == 0) {
    // every copy of the pair lands before either CTA exits.  Stage s's last
    // phases: rank 0 expected both CTAs' bytes for its own copies; a copy one
    // CTA issued and the other did not (after a failure) is balanced here.
    (void)pair_drain(qlanded, 0);
    const uint32_t i0 = issued, i1 = *peer_issued;
    const uint32_t hi = i0 > i1 ? i0 : i1;
    for (uint32_t jj = hi > (uint32_t)NS ? hi - NS : 0u; jj < hi; ++jj) {
      uint64_t* bar = &landed[jj % NS];
      const bool e0 = jj < i0, e1 = jj < i1;
      if (e0 && !e1) mbar_complete_tx(bar, kFdmStageBytes);  // rank 1's share never comes
      if (!e0 && e1) mbar_expect_tx(bar, kFdmStageBytes);    // only rank 1's share comes
      (void)pair_drain(bar, (jj / NS) & 1u);
    }
  }
  __syncthreads();
  // no copy, remote arrive, multicast commit or flag store targets either CTA after this
  cluster_sync();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(kFdmPairTmemCols)
                 : "memory");
  }
  const bool failed = *fail != 0;
  if (failed && threadIdx.x == 0) {
    sc->status = 6;
    sc->done = 1;
  }
  if (mode != kFdmDot) return;
  double a[1] = {(double)dot};
  double tot[1];
  if (grid_reduce<1, 0u>(a, partials, &sc->ticket, tot)) {
    if (sc->status == 6) return;
    const double rz = tot[0];
    if (sc->iter > 0) sc->beta = sc->beta * (rz / sc->rz);
    sc->rz = rz;
    if (!isfinite(rz)) {
      sc->done = 1;
      sc->status = 5;
    } else if (!(rz > 0.0)) {
      sc->done = 1;
      sc->status = 4;
    }
  }
}

}  // namespace rk

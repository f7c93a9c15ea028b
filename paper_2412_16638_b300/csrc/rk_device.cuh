// Device helpers shared by all kernels of the library: storage/arithmetic
// conversions (the "accessor": vectors are stored in S and operated on in T),
// vectorised segment loads, and a deterministic one-pass grid reduction.
#pragma once
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace rk {

constexpr int kThreads = 256;  // threads per CTA of every grid-stride kernel

// ---------------------------------------------------------------- conversions
template <typename T> __device__ __forceinline__ T wid(double v) { return (T)v; }
template <typename T> __device__ __forceinline__ T wid(float v) { return (T)v; }
template <typename T> __device__ __forceinline__ T wid(__half v) { return (T)__half2float(v); }
template <typename T> __device__ __forceinline__ T wid(__nv_bfloat16 v) { return (T)__bfloat162float(v); }

template <typename S> __device__ __forceinline__ S nar(float v);
template <> __device__ __forceinline__ double nar<double>(float v) { return (double)v; }
template <> __device__ __forceinline__ float nar<float>(float v) { return v; }
template <> __device__ __forceinline__ __half nar<__half>(float v) { return __float2half_rn(v); }
template <> __device__ __forceinline__ __nv_bfloat16 nar<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }

template <typename S> __device__ __forceinline__ S nar(double v);
template <> __device__ __forceinline__ double nar<double>(double v) { return v; }
template <> __device__ __forceinline__ float nar<float>(double v) { return (float)v; }
template <> __device__ __forceinline__ __half nar<__half>(double v) { return __double2half(v); }
template <> __device__ __forceinline__ __nv_bfloat16 nar<__nv_bfloat16>(double v) { return __double2bfloat16(v); }

// Type of the Krylov solution vector x = k^eps for work-vector storage S: with
// 16-bit work vectors the solution is accumulated and kept in FP32, because
// k^eps feeds the FP64 explicit correction and later stages, where a 16-bit
// rounding of it would dominate the error.
template <typename S> struct XOf { using type = S; };
template <> struct XOf<__half> { using type = float; };
template <> struct XOf<__nv_bfloat16> { using type = float; };

// value as it will be read back after a store in S
template <typename S, typename T> __device__ __forceinline__ T rnd(T v) { return wid<T>(nar<S>(v)); }

// ---------------------------------------------------------------- segments
// Load SEG consecutive values p[0..SEG) (only the first m <= SEG valid; the
// rest read as zero).  Uses 16/8-byte vector loads when the whole segment
// is valid and the address is aligned.
template <typename T, typename S, int SEG>
__device__ __forceinline__ void load_seg(const S* __restrict__ p, int m, T (&v)[SEG]) {
  constexpr int BYTES = SEG * (int)sizeof(S);
  if (m == SEG) {
    if constexpr (BYTES % 16 == 0) {
      if ((reinterpret_cast<uintptr_t>(p) & 15) == 0) {
        alignas(16) S tmp[SEG];
        const uint4* src = reinterpret_cast<const uint4*>(p);
        uint4* dst = reinterpret_cast<uint4*>(tmp);
#pragma unroll
        for (int w = 0; w < BYTES / 16; ++w) dst[w] = src[w];
#pragma unroll
        for (int e = 0; e < SEG; ++e) v[e] = wid<T>(tmp[e]);
        return;
      }
    } else if constexpr (BYTES % 8 == 0) {
      if ((reinterpret_cast<uintptr_t>(p) & 7) == 0) {
        alignas(8) S tmp[SEG];
        const uint2* src = reinterpret_cast<const uint2*>(p);
        uint2* dst = reinterpret_cast<uint2*>(tmp);
#pragma unroll
        for (int w = 0; w < BYTES / 8; ++w) dst[w] = src[w];
#pragma unroll
        for (int e = 0; e < SEG; ++e) v[e] = wid<T>(tmp[e]);
        return;
      }
    }
  }
#pragma unroll
  for (int e = 0; e < SEG; ++e) v[e] = (e < m) ? wid<T>(p[e]) : T(0);
}

// Store the first m of SEG values (narrowed to S).
template <typename S, typename T, int SEG>
__device__ __forceinline__ void store_seg(S* __restrict__ p, int m, const T (&v)[SEG]) {
  constexpr int BYTES = SEG * (int)sizeof(S);
  if (m == SEG) {
    if constexpr (BYTES % 16 == 0) {
      if ((reinterpret_cast<uintptr_t>(p) & 15) == 0) {
        alignas(16) S tmp[SEG];
#pragma unroll
        for (int e = 0; e < SEG; ++e) tmp[e] = nar<S>(v[e]);
        const uint4* src = reinterpret_cast<const uint4*>(tmp);
        uint4* dst = reinterpret_cast<uint4*>(p);
#pragma unroll
        for (int w = 0; w < BYTES / 16; ++w) dst[w] = src[w];
        return;
      }
    } else if constexpr (BYTES % 8 == 0) {
      if ((reinterpret_cast<uintptr_t>(p) & 7) == 0) {
        alignas(8) S tmp[SEG];
#pragma unroll
        for (int e = 0; e < SEG; ++e) tmp[e] = nar<S>(v[e]);
        const uint2* src = reinterpret_cast<const uint2*>(tmp);
        uint2* dst = reinterpret_cast<uint2*>(p);
#pragma unroll
        for (int w = 0; w < BYTES / 8; ++w) dst[w] = src[w];
        return;
      }
    }
  }
#pragma unroll
  for (int e = 0; e < SEG; ++e)
    if (e < m) p[e] = nar<S>(v[e]);
}

// ---------------------------------------------------------------- reductions
// Reduction of NV doubles across the CTA; bit c of MAXMASK selects max
// (otherwise sum).  Result valid in thread 0.  Fixed order: deterministic.
template <int NV, unsigned MAXMASK>
__device__ __forceinline__ void block_reduce(double (&v)[NV], double* sred /* >= 32*NV */) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int c = 0; c < NV; ++c) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      double o = __shfl_down_sync(0xffffffffu, v[c], off);
      v[c] = ((MAXMASK >> c) & 1u) ? fmax(v[c], o) : v[c] + o;
    }
  }
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int c = 0; c < NV; ++c) sred[warp * NV + c] = v[c];
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int c = 0; c < NV; ++c) {
      v[c] = (lane < nw) ? sred[lane * NV + c] : 0.0;
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        double o = __shfl_down_sync(0xffffffffu, v[c], off);
        v[c] = ((MAXMASK >> c) & 1u) ? fmax(v[c], o) : v[c] + o;
      }
    }
  }
  __syncthreads();
}

// One-pass grid reduction: every CTA writes its partial, the CTA that takes
// the last ticket sums the partials in CTA order (deterministic for a given
// grid size) and resets the ticket.  Returns true in thread 0 of that CTA,
// with the totals in tot.  partials must hold gridDim.x * NV doubles.
// Max reductions assume non-negative inputs (identity 0).
template <int NV, unsigned MAXMASK>
__device__ __forceinline__ bool grid_reduce(double (&v)[NV], double* __restrict__ partials,
                                            unsigned* ticket, double (&tot)[NV]) {
  __shared__ double sred[32 * NV];
  __shared__ int am_last;
  block_reduce<NV, MAXMASK>(v, sred);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int c = 0; c < NV; ++c) partials[(size_t)blockIdx.x * NV + c] = v[c];
    __threadfence();
    unsigned t = atomicAdd(ticket, 1u);
    am_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!am_last) return false;
  __threadfence();
  double acc[NV];
#pragma unroll
  for (int c = 0; c < NV; ++c) acc[c] = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
#pragma unroll
    for (int c = 0; c < NV; ++c) {
      double x = __ldcg(partials + (size_t)b * NV + c);
      acc[c] = ((MAXMASK >> c) & 1u) ? fmax(acc[c], x) : acc[c] + x;
    }
  }
  block_reduce<NV, MAXMASK>(acc, sred);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int c = 0; c < NV; ++c) tot[c] = acc[c];
    *ticket = 0u;
    return true;
  }
  return false;
}

}  // namespace rk

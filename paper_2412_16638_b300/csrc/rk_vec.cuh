// Element-wise FP64 kernels of the stage loop: stage right-hand sides and the
// solution update (linear combinations in high precision, Sec. 4.2), plus
// small helpers (norms, widening, refinement updates).
#pragma once
#include "rk_device.cuh"
#include "rk_heat.cuh"

namespace rk {

constexpr int kMaxStages = 8;

// out = u + sum_j ch[j]*kh[j] + sum_j ce[j]*ke[j]/sigma_j   (FP64 arithmetic)
// Stage right-hand side r_i = u_n + tau sum_{j<i}(a^h_ij k_j + a^eps_ij k^eps_j)
// (Eqs. mpAstep1-4) and the update u_{n+1} = u_n + tau sum_j b_j k_j (Eq. RKstep).
struct CombineArgs {
  const double* u;
  const double* kh[kMaxStages];
  double ch[kMaxStages];
  const void* ke[kMaxStages];
  double ce[kMaxStages];
  const RhsScalars* rs[kMaxStages];
  int nh, ne;
  double* out;
  long long N;
};

// The term loops run to the actual counts (not unrolled to kMaxStages): on
// this part a predicated-off FP64 instruction still costs an FP64 issue slot.
template <typename S>
__global__ void __launch_bounds__(kThreads) combine_f64(CombineArgs a) {
  __shared__ const double* s_kh[kMaxStages];
  __shared__ const S* s_ke[kMaxStages];
  __shared__ double s_ch[kMaxStages], s_ce[kMaxStages];
  if (threadIdx.x < kMaxStages) {
    const int j = threadIdx.x;
    s_kh[j] = a.kh[j];
    s_ch[j] = a.ch[j];
    s_ke[j] = static_cast<const S*>(a.ke[j]);
    s_ce[j] = (j < a.ne) ? a.ce[j] / a.rs[j]->sigma : 0.0;
  }
  __syncthreads();
  const int nh = a.nh, ne = a.ne;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < a.N;
       i += (long long)gridDim.x * blockDim.x) {
    double v = a.u ? a.u[i] : 0.0;
#pragma unroll 1
    for (int j = 0; j < nh; ++j) v = fma(s_ch[j], s_kh[j][i], v);
#pragma unroll 1
    for (int j = 0; j < ne; ++j) v = fma(s_ce[j], wid<double>(s_ke[j][i]), v);
    a.out[i] = v;
  }
}

// ||g||^2, ||g||_inf and the storage scale of an FP64 vector into *rs.
static __global__ void __launch_bounds__(kThreads) vec_norms_f64(const double* __restrict__ g, long long N,
                                                                 RhsScalars* rs, double* partials) {
  double acc[2] = {0.0, 0.0};
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    const double v = g[i];
    acc[0] = fma(v, v, acc[0]);
    acc[1] = fmax(acc[1], fabs(v));
  }
  double tot[2];
  if (grid_reduce<2, 2u>(acc, partials, &rs->ticket, tot)) {
    rs->gg = tot[0];
    rs->gmax = tot[1];
    rs->sigma = rhs_scale(rs, tot[0], tot[1], N);
  }
}

// out = x / sigma widened to FP64.
template <typename S>
__global__ void __launch_bounds__(kThreads) widen_f64(const S* __restrict__ x, const RhsScalars* rs,
                                                      double* __restrict__ out, long long N) {
  const double inv = 1.0 / rs->sigma;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = wid<double>(x[i]) * inv;
}

// x holds sigma_x * k, dx holds sigma_dx * delta: x <- x + (sigma_x/sigma_dx) dx
// (refinement update of k^eps, arithmetic in FP64).  With an FP64 x the
// corrections accumulate without rounding k^eps back to the solver's type.
template <typename SX, typename SD>
__global__ void __launch_bounds__(kThreads) add_scaled_inplace(SX* __restrict__ x, const SD* __restrict__ dx,
                                                               const RhsScalars* rs_x, const RhsScalars* rs_dx,
                                                               long long N) {
  const double f = rs_x->sigma / rs_dx->sigma;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x)
    x[i] = nar<SX>(fma(f, wid<double>(dx[i]), wid<double>(x[i])));
}

// out = x widened to FP64, keeping its storage scale (out holds sigma * k as x
// does): the solver output moved into an FP64 k^eps.
template <typename S>
__global__ void __launch_bounds__(kThreads) widen_keep_f64(const S* __restrict__ x, double* __restrict__ out,
                                                           long long N) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = wid<double>(x[i]);
}

// res = k - ke/sigma (FP64): the true residual of the last stage solve, used
// as the right-hand side of a refinement solve.
template <typename S>
__global__ void __launch_bounds__(kThreads) true_residual_f64(const double* __restrict__ kfull,
                                                              const S* __restrict__ ke, const RhsScalars* rs,
                                                              double* __restrict__ res, long long N) {
  const double inv = 1.0 / rs->sigma;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x)
    res[i] = kfull[i] - wid<double>(ke[i]) * inv;
}

}  // namespace rk

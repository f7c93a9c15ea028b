// Complex fast diagonalization of the periodic advection stage matrix
// (Sec. 3, Eq. Pinvform, applied to the operator of Sec. 5.2.2):
// P = I - s L with L = -sum_d beta_d D_d, D the periodic central difference.
// Every 1-D factor is a polynomial in the circulant D, whose eigenvectors are
// the Fourier modes e^{2 pi i j k / n} with eigenvalues i sin(2 pi k / n) / h, so
//   P^-1 r = F^-1 [ (F r)_k / (1 + i s theta_k) ],
//   theta_k = sum_d beta_d sin(2 pi k_d / n) / h,
// with F the 3-D discrete Fourier transform.  Each of the six passes contracts
// one axis of the n^3 array against the n x n Fourier matrix (the mode-n
// products T_R, T_M, T_L of Eq. TensorDecomp) and stores the result with the
// contracted index moved to the slowest position, so every pass reads lines
// along the fastest index and writes coalesced:
//   [z][y][x] -> [kx][z][y] -> [ky][kx][z] -> [kz][ky][kx]   (forward, P_D^-1 in
//   the third pass's epilogue) -> [x][kz][ky] -> [y][x][kz] -> [z][y][x]  (inverse).
// A CTA takes a tile of kCfTile lines (fixed slow index a, consecutive middle
// indices b) into shared memory and transforms each line: for n = n1 n2 in two
// steps of n1 and n2 terms (in place, see cfdm_pass), for a prime n as direct
// n-term sums; the twiddles e^{-+2 pi i m / n} come from a table indexed by
// the exponent mod n.
// Arithmetic in T (FP32 for FP32 storage, FP64 for the FP64 path).
#pragma once
#include "rk_csr.cuh"

namespace rk {

constexpr int kCfTile = 32;  // lines per CTA (consecutive middle indices)
constexpr int kCfThreads = 256;
constexpr int kCfK = 4;      // outputs per thread per round

template <typename T> struct Cplx { T re, im; };

constexpr int kCfMaxN1 = 20;    // largest first factor (n <= 400)
constexpr int kCfMaxTab = 1024;  // entries of the two small-DFT tables, n1^2 + n2^2

// Factor n = n1 n2 for the two-step transform: n1 the largest divisor of n
// not above sqrt(n), provided the tables of the two small transforms (n1^2 +
// n2^2 entries) stay small; else 1 (the direct n-term sums, e.g. for a prime n).
__host__ __device__ inline int cfdm_factor(int n) {
  int n1 = 1;
  for (int d = 2; d * d <= n && d <= kCfMaxN1; ++d)
    if (n % d == 0) n1 = d;
  const int n2 = n / n1;
  return (n1 > 1 && n1 * n1 + n2 * n2 <= kCfMaxTab) ? n1 : 1;
}

// Dynamic shared memory of a pass: the line tile (the factored transform works
// in place), the n twiddles, and for n = n1 n2 the tables of the two small
// transforms.
template <typename T>
__host__ __device__ inline size_t cfdm_smem(int n) {
  const int n1 = cfdm_factor(n), n2 = n / n1;
  const size_t tab = n1 > 1 ? (size_t)n1 * n1 + (size_t)n2 * n2 : 0;
  return (size_t)kCfTile * (n + 1) * sizeof(Cplx<T>) + ((size_t)n + tab) * sizeof(Cplx<T>);
}

// Parameters of the diagonal scaling P_D^-1 (third pass).
struct CfScale {
  double s;          // shift s of I - s L
  double beta[3];    // velocity
  double inv_h;      // 1 / h = n
  double norm;       // 1 / n^3 (normalisation of the inverse transform)
};

// One pass.  in: real S (IN_REAL) or complex; out: complex, or the real part
// in S (OUT_REAL).  tw: n twiddles e^{-2 pi i m / n}; inverse passes use the
// conjugates.  scale != 0: divide by 1 + i s theta (and normalise), with the
// output index (k, a, b) = (kz, ky, kx).  sc != null: the GMRES step's
// preconditioner application, skipped when the solver state says none is due.
// in_jstride > 0 (first pass of a GMRES step): the input is basis slot sc->j,
// in + sc->j * in_jstride elements.
//
// With n = n1 n2 (n1 > 1) each line is transformed in two steps (Cooley-Tukey,
// decimation in time: j = n2 j1 + j2, k = k1 + n1 k2, w = e^{-+2 pi i / n}):
//   A[k1][j2]      = w^{j2 k1} sum_{j1} x[n2 j1 + j2] w^{n2 j1 k1}   (n1 terms)
//   X[k1 + n1 k2]  = sum_{j2} A[k1][j2] w^{n1 j2 k2}                  (n2 terms)
// since w^{jk} = w^{n2 j1 k1} w^{j2 k1} w^{n1 j2 k2} (the w^{n j1 k2} factor is
// 1): n1 + n2 + 1 products per output instead of n.  The two small transforms
// read their twiddles from n1 x n1 and n2 x n2 tables, so the inner loops do
// no index arithmetic mod n.
template <typename SI, typename SO, typename T, bool IN_REAL, bool OUT_REAL>
__global__ void __launch_bounds__(kCfThreads) cfdm_pass(const void* __restrict__ in, void* __restrict__ out, int n,
                                                        int n1, const Cplx<T>* __restrict__ tw, int inverse,
                                                        int scale, CfScale sp, const GmScalars* sc,
                                                        long long in_jstride) {
  if (sc && (sc->done || sc->cycle_end || sc->j >= sc->m)) return;
  if (sc && in_jstride > 0) in = static_cast<const SI*>(in) + (long long)sc->j * in_jstride;
  extern __shared__ __align__(128) unsigned char smem[];
  using C = Cplx<T>;
  C* tile = reinterpret_cast<C*>(smem);                       // [kCfTile][n + 1]
  C* tws = tile + (size_t)kCfTile * (n + 1);                  // [n]
  const int n2 = n / n1;
  C* W1 = tws + n;             // [n1][n1]: w^{n2 (j1 k1 mod n1)} at k1 n1 + j1
  C* W2 = W1 + n1 * n1;        // [n2][n2]: w^{n1 (j2 k2 mod n2)} at k2 n2 + j2
  const int nbt = (n + kCfTile - 1) / kCfTile;
  const int a = blockIdx.x / nbt;
  const int b0 = (blockIdx.x % nbt) * kCfTile;
  const int tb = min(kCfTile, n - b0);
  auto twid = [&](int m) {
    C w = tw[m];
    if (inverse) w.im = -w.im;
    return w;
  };
  for (int m = threadIdx.x; m < n; m += blockDim.x) tws[m] = twid(m);
  if (n1 > 1) {
    for (int e = threadIdx.x; e < n1 * n1; e += blockDim.x) {
      const int k1 = e / n1, j1 = e - k1 * n1;
      W1[e] = twid(n2 * ((j1 * k1) % n1));
    }
    for (int e = threadIdx.x; e < n2 * n2; e += blockDim.x) {
      const int k2 = e / n2, j2 = e - k2 * n2;
      W2[e] = twid(n1 * ((j2 * k2) % n2));
    }
  }
  // load the lines (a, b0 + bb, 0..n-1), coalesced along the line
  for (int e = threadIdx.x; e < tb * n; e += blockDim.x) {
    const int bb = e / n, j = e - bb * n;
    const long long gi = ((long long)a * n + b0 + bb) * n + j;
    C v;
    if constexpr (IN_REAL) {
      v.re = wid<T>(static_cast<const SI*>(in)[gi]);
      v.im = T(0);
    } else {
      v = static_cast<const C*>(in)[gi];
    }
    tile[(size_t)bb * (n + 1) + j] = v;
  }
  __syncthreads();
  const int bb = threadIdx.x % kCfTile;
  const int warp = threadIdx.x / kCfTile;
  constexpr int kWarps = kCfThreads / kCfTile;
  // output k of line bb: P_D^-1 in the third pass, then the store; lanes of a
  // warp take consecutive bb (coalesced stores)
  auto emit = [&](int k, T r, T i) {
    if (scale) {
      // (kz, ky, kx) = (k, a, b); sin(2 pi m / n) = -Im e^{-2 pi i m / n}
      const int kx = b0 + bb;
      const T th = ((T)sp.beta[0] * (-tw[kx].im) + (T)sp.beta[1] * (-tw[a].im) + (T)sp.beta[2] * (-tw[k].im)) *
                   (T)sp.inv_h;
      const T c = (T)sp.s * th;
      const T den = (T)sp.norm / fma(c, c, T(1));
      const T r2 = fma(i, c, r) * den, i2 = fma(-r, c, i) * den;
      r = r2;
      i = i2;
    }
    const long long go = ((long long)k * n + a) * n + b0 + bb;
    if constexpr (OUT_REAL) {
      static_cast<SO*>(out)[go] = nar<SO>(r);
    } else {
      C v;
      v.re = r;
      v.im = i;
      static_cast<C*>(out)[go] = v;
    }
  };
  const C* row = tile + (size_t)bb * (n + 1);
  if (n1 <= 1) {
    // direct n-term sums; each thread forms kCfK outputs k0, k0 + 8, ... of its
    // line at once, so one read of the line element serves kCfK products
    if (bb >= tb) return;
    for (int k0 = warp; k0 < n; k0 += kWarps * kCfK) {
      T re[kCfK], im[kCfK];
      int idx[kCfK], kk[kCfK];  // j k mod n, and k (0 for outputs past the end)
#pragma unroll
      for (int q = 0; q < kCfK; ++q) {
        const int k = k0 + q * kWarps;
        kk[q] = k < n ? k : 0;
        idx[q] = 0;
        re[q] = im[q] = T(0);
      }
      for (int j = 0; j < n; ++j) {
        const C x = row[j];
#pragma unroll
        for (int q = 0; q < kCfK; ++q) {
          const C w = tws[idx[q]];
          re[q] = fma(x.re, w.re, fma(-x.im, w.im, re[q]));
          im[q] = fma(x.re, w.im, fma(x.im, w.re, im[q]));
          idx[q] += kk[q];
          if (idx[q] >= n) idx[q] -= n;
        }
      }
#pragma unroll
      for (int q = 0; q < kCfK; ++q) {
        const int k = k0 + q * kWarps;
        if (k < n) emit(k, re[q], im[q]);
      }
    }
    return;
  }
  // step 1, in place: task j2 (one per warp at a time) reads the n1 elements
  // n2 j1 + j2 of its line into registers and writes
  // A[k1][j2] = w^{j2 k1} sum_{j1} x[n2 j1 + j2] w^{n2 j1 k1} to the same slots
  // n2 k1 + j2 (the tasks' slot sets are disjoint); j2 k1 < n, so the twiddle
  // needs no reduction mod n
  {
    C* rowA = tile + (size_t)bb * (n + 1);
    for (int j2 = warp; j2 < n2; j2 += kWarps) {
      if (bb >= tb) continue;
      C xr[kCfMaxN1];
#pragma unroll
      for (int j1 = 0; j1 < kCfMaxN1; ++j1)
        if (j1 < n1) xr[j1] = rowA[n2 * j1 + j2];
      for (int k1 = 0; k1 < n1; ++k1) {
        const C* w1 = W1 + k1 * n1;
        T re = T(0), im = T(0);
#pragma unroll
        for (int j1 = 0; j1 < kCfMaxN1; ++j1)
          if (j1 < n1) {
            const C w = w1[j1];
            re = fma(xr[j1].re, w.re, fma(-xr[j1].im, w.im, re));
            im = fma(xr[j1].re, w.im, fma(xr[j1].im, w.re, im));
          }
        const C t = tws[j2 * k1];
        C v;
        v.re = fma(re, t.re, -im * t.im);
        v.im = fma(re, t.im, im * t.re);
        rowA[n2 * k1 + j2] = v;
      }
    }
  }
  __syncthreads();
  if (bb >= tb) return;
  // step 2: X[k1 + n1 k2] = sum_{j2} A[k1][j2] w^{n1 (j2 k2 mod n2)}; tasks
  // (k1, group of kCfK consecutive k2) share the reads of A[k1][.]
  {
    const int kg = (n2 + kCfK - 1) / kCfK;
    const C* rowA = tile + (size_t)bb * (n + 1);
    for (int task = warp; task < n1 * kg; task += kWarps) {
      const int k1 = task / kg;
      const int k2b = (task - k1 * kg) * kCfK;
      T re[kCfK], im[kCfK];
      const C* w2[kCfK];
#pragma unroll
      for (int q = 0; q < kCfK; ++q) {
        w2[q] = W2 + (size_t)(k2b + q < n2 ? k2b + q : 0) * n2;
        re[q] = im[q] = T(0);
      }
      const C* a1 = rowA + (size_t)k1 * n2;
      for (int j2 = 0; j2 < n2; ++j2) {
        const C x = a1[j2];
#pragma unroll
        for (int q = 0; q < kCfK; ++q) {
          const C w = w2[q][j2];
          re[q] = fma(x.re, w.re, fma(-x.im, w.im, re[q]));
          im[q] = fma(x.re, w.im, fma(x.im, w.re, im[q]));
        }
      }
#pragma unroll
      for (int q = 0; q < kCfK; ++q)
        if (k2b + q < n2) emit(k1 + n1 * (k2b + q), re[q], im[q]);
    }
  }
}

// u = sum_{i < jused} y_i V_i (the cycle-end combination of the basis,
// before the preconditioner is applied to it), stored in S.
template <typename S, typename B, typename T>
__global__ void __launch_bounds__(kThreads) gm_basis_combine(const B* __restrict__ V, long long ldv, long long N,
                                                             const double* __restrict__ y, const int* jused,
                                                             S* __restrict__ u) {
  __shared__ T ys[kGmMax];
  const int ju = *jused;
  for (int i = threadIdx.x; i < ju; i += blockDim.x) ys[i] = (T)y[i];
  __syncthreads();
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < N; r += (long long)gridDim.x * blockDim.x) {
    T a = T(0);
    for (int i = 0; i < ju; ++i) a = fma(ys[i], wid<T>(V[(long long)i * ldv + r]), a);
    u[r] = nar<S>(a);
  }
}

// out = in converted (FP64 <-> storage type; for the single-application entry point).
template <typename A, typename B2>
__global__ void __launch_bounds__(kThreads) convert_vec(const A* __restrict__ in, B2* __restrict__ out, long long N) {
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < N; r += (long long)gridDim.x * blockDim.x)
    out[r] = nar<B2>(wid<double>(in[r]));
}

// x += z (x in the solution type, z the preconditioned combination).
template <typename S, typename X>
__global__ void __launch_bounds__(kThreads) add_into(X* __restrict__ x, const S* __restrict__ z, long long N) {
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < N; r += (long long)gridDim.x * blockDim.x)
    x[r] = x[r] + wid<X>(z[r]);
}

}  // namespace rk

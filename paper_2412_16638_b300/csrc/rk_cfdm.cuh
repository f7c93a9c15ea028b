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
#include <type_traits>

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
  // P_D^-1 constants in T, converted once (an FP64 -> FP32 conversion per
  // element would run on the slow conversion path); (kz, ky, kx) = (k, a, b),
  // sin(2 pi m / n) = -Im e^{-2 pi i m / n}, theta summed in the order
  // kx, ky, kz
  const T sb2 = (T)sp.beta[2], sinvh = (T)sp.inv_h, ss = (T)sp.s, snorm = (T)sp.norm;
  const T th_ab = scale ? (T)sp.beta[0] * (-tw[min(b0 + bb, n - 1)].im) + (T)sp.beta[1] * (-tw[a].im) : T(0);
  // output k of line bb: P_D^-1 in the third pass, then the store; lanes of a
  // warp take consecutive bb (coalesced stores)
  auto emit = [&](int k, T r, T i) {
    if (scale) {
      const T th = (th_ab + sb2 * (-tw[k].im)) * sinvh;
      const T c = ss * th;
      const T den = snorm / fma(c, c, T(1));
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

// ------------------------------------------------ compile-time small DFTs
// For the grid sizes below, n = N1 N2 is a template parameter and every small
// transform is written out at compile time: mixed-radix Cooley-Tukey down to
// sizes 2 and odd primes, the twiddles as constants (cos and sin of 2 pi m / N
// by Taylor series at compile time), multiplications by +-1 and +-i turned
// into adds, and the odd-prime sizes through the symmetric pairs x_j +- x_{N-j}
// (outputs k and N - k share their products).  No twiddle table is read and
// no index is formed at run time inside a small transform.

// cos / sin of 2 pi m / N (0 <= m < N), for compile-time twiddles.
constexpr double cf_series_sin(double x) {
  double t = x, s = x;
  for (int i = 1; i < 30; ++i) {
    t *= -x * x / ((2.0 * i) * (2.0 * i + 1.0));
    s += t;
  }
  return s;
}
constexpr double cf_series_cos(double x) {
  double t = 1.0, s = 1.0;
  for (int i = 1; i < 30; ++i) {
    t *= -x * x / ((2.0 * i - 1.0) * (2.0 * i));
    s += t;
  }
  return s;
}
constexpr double cf_angle(int m, int N) {  // 2 pi m / N reduced to [-pi, pi]
  const double pi = 3.14159265358979323846;
  return (2 * m > N ? 2.0 * pi * (m - N) : 2.0 * pi * m) / N;
}
constexpr double cf_cos(int m, int N) { return cf_series_cos(cf_angle(m, N)); }
constexpr double cf_sin(int m, int N) { return cf_series_sin(cf_angle(m, N)); }

constexpr int cf_small_factor(int N) {
  for (int p = 2; p * p <= N; ++p)
    if (N % p == 0) return p;
  return N;
}

template <int I, int E, typename F>
__device__ __forceinline__ void cf_for(F&& f) {
  if constexpr (I < E) {
    f(std::integral_constant<int, I>{});
    cf_for<I + 1, E>(f);
  }
}

// x * e^{-2 pi i M / N}
template <typename T, int N, int M>
__device__ __forceinline__ Cplx<T> cf_twiddle(Cplx<T> x) {
  constexpr int m = M % N;
  if constexpr (m == 0) {
    return x;
  } else if constexpr (2 * m == N) {
    return Cplx<T>{-x.re, -x.im};
  } else if constexpr (4 * m == N) {
    return Cplx<T>{x.im, -x.re};
  } else if constexpr (4 * m == 3 * N) {
    return Cplx<T>{-x.im, x.re};
  } else {
    constexpr double c = cf_cos(m, N), sn = -cf_sin(m, N);  // w = c + i sn
    return Cplx<T>{fma(x.re, (T)c, -x.im * (T)sn), fma(x.re, (T)sn, x.im * (T)c)};
  }
}

// In place: x[k] <- sum_j x[j] e^{-2 pi i j k / N}.
template <typename T, int N>
__device__ __forceinline__ void cf_dft(Cplx<T> (&x)[N]) {
  if constexpr (N == 1) {
    return;
  } else if constexpr (N == 2) {
    const Cplx<T> a = x[0], b = x[1];
    x[0] = Cplx<T>{a.re + b.re, a.im + b.im};
    x[1] = Cplx<T>{a.re - b.re, a.im - b.im};
  } else if constexpr (cf_small_factor(N) == N) {
    // odd prime: s_j = x_j + x_{N-j}, d_j = x_j - x_{N-j} (j = 1 .. H);
    // y_k = x_0 + sum_j s_j cos(2 pi j k / N) - i d_j sin(2 pi j k / N), and
    // y_{N-k} the same with the sine terms negated
    constexpr int H = (N - 1) / 2;
    Cplx<T> sv[H], dv[H];
    Cplx<T> y0 = x[0];
    cf_for<1, H + 1>([&](auto jc) {
      constexpr int J = decltype(jc)::value;
      sv[J - 1] = Cplx<T>{x[J].re + x[N - J].re, x[J].im + x[N - J].im};
      dv[J - 1] = Cplx<T>{x[J].re - x[N - J].re, x[J].im - x[N - J].im};
      y0.re += sv[J - 1].re;
      y0.im += sv[J - 1].im;
    });
    Cplx<T> out[N];
    out[0] = y0;
    cf_for<1, H + 1>([&](auto kc) {
      constexpr int K = decltype(kc)::value;
      T are = x[0].re, aim = x[0].im, bre = T(0), bim = T(0);
      cf_for<1, H + 1>([&](auto jc) {
        constexpr int J = decltype(jc)::value;
        constexpr double c = cf_cos((J * K) % N, N), sn = cf_sin((J * K) % N, N);
        are = fma(sv[J - 1].re, (T)c, are);
        aim = fma(sv[J - 1].im, (T)c, aim);
        bre = fma(dv[J - 1].im, (T)sn, bre);
        bim = fma(dv[J - 1].re, (T)sn, bim);
      });
      out[K] = Cplx<T>{are + bre, aim - bim};
      out[N - K] = Cplx<T>{are - bre, aim + bim};
    });
    cf_for<0, N>([&](auto kc) { x[decltype(kc)::value] = out[decltype(kc)::value]; });
  } else {
    // N = P Q: j = Q j1 + j2, k = k1 + P k2
    constexpr int P = cf_small_factor(N), Q = N / P;
    Cplx<T> a[Q][P];
    cf_for<0, Q>([&](auto j2c) {
      constexpr int J2 = decltype(j2c)::value;
      Cplx<T> v[P];
      cf_for<0, P>([&](auto j1c) { v[decltype(j1c)::value] = x[Q * decltype(j1c)::value + J2]; });
      cf_dft<T, P>(v);
      cf_for<0, P>([&](auto k1c) {
        constexpr int K1 = decltype(k1c)::value;
        a[J2][K1] = cf_twiddle<T, N, J2 * K1>(v[K1]);
      });
    });
    cf_for<0, P>([&](auto k1c) {
      constexpr int K1 = decltype(k1c)::value;
      Cplx<T> v[Q];
      cf_for<0, Q>([&](auto j2c) { v[decltype(j2c)::value] = a[decltype(j2c)::value][K1]; });
      cf_dft<T, Q>(v);
      cf_for<0, Q>([&](auto k2c) { x[K1 + P * decltype(k2c)::value] = v[decltype(k2c)::value]; });
    });
  }
}

// The pass of cfdm_pass for n = N1 N2 known at compile time, 32 N1 threads
// (warp w, lane = line bb of the tile).  Step 1: task j2 (warps in turn)
// transforms x[N2 j1 + j2] over j1 with cf_dft<N1>, multiplies by w^{j2 k1}
// (table, j2 varies at run time) and writes back in place; step 2: warp k1
// transforms A[k1][.] with cf_dft<N2> and emits X[k1 + N1 k2].  The inverse
// transform is conj(F conj(x)).
template <typename SI, typename SO, typename T, bool IN_REAL, bool OUT_REAL, int N1, int N2>
__global__ void __launch_bounds__(32 * N1) cfdm_pass_ct(const void* __restrict__ in, void* __restrict__ out,
                                                        const Cplx<T>* __restrict__ tw, int inverse, int scale,
                                                        CfScale sp, const GmScalars* sc, long long in_jstride) {
  constexpr int n = N1 * N2;
  if (sc && (sc->done || sc->cycle_end || sc->j >= sc->m)) return;
  if (sc && in_jstride > 0) in = static_cast<const SI*>(in) + (long long)sc->j * in_jstride;
  extern __shared__ __align__(128) unsigned char smem[];
  using C = Cplx<T>;
  C* tile = reinterpret_cast<C*>(smem);       // [kCfTile][n + 1]
  C* tws = tile + (size_t)kCfTile * (n + 1);  // [n], forward twiddles
  constexpr int nbt = (n + kCfTile - 1) / kCfTile;
  const int a = blockIdx.x / nbt;
  const int b0 = (blockIdx.x % nbt) * kCfTile;
  const int tb = min(kCfTile, n - b0);
  const T cj = inverse ? T(-1) : T(1);  // conjugation of the inverse transform
  for (int m = threadIdx.x; m < n; m += blockDim.x) tws[m] = tw[m];
  for (int e = threadIdx.x; e < tb * n; e += blockDim.x) {
    const int bb = e / n, j = e - bb * n;
    const long long gi = ((long long)a * n + b0 + bb) * n + j;
    C v;
    if constexpr (IN_REAL) {
      v.re = wid<T>(static_cast<const SI*>(in)[gi]);
      v.im = T(0);
    } else {
      v = static_cast<const C*>(in)[gi];
      v.im *= cj;
    }
    tile[(size_t)bb * (n + 1) + j] = v;
  }
  __syncthreads();
  const int bb = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  C* row = tile + (size_t)bb * (n + 1);
  if (bb < tb) {
    for (int j2 = warp; j2 < N2; j2 += N1) {
      C x[N1];
      cf_for<0, N1>([&](auto j1c) { x[decltype(j1c)::value] = row[N2 * decltype(j1c)::value + j2]; });
      cf_dft<T, N1>(x);
      cf_for<0, N1>([&](auto k1c) {
        constexpr int K1 = decltype(k1c)::value;
        C v = x[K1];
        if constexpr (K1 > 0) {
          const C t = tws[j2 * K1];
          v = C{fma(x[K1].re, t.re, -x[K1].im * t.im), fma(x[K1].re, t.im, x[K1].im * t.re)};
        }
        row[N2 * K1 + j2] = v;
      });
    }
  }
  __syncthreads();
  if (bb >= tb) return;
  const int k1 = warp;  // N1 warps: one task each
  // P_D^-1 constants in T, converted once (see cfdm_pass)
  const T sb2 = (T)sp.beta[2], sinvh = (T)sp.inv_h, ss = (T)sp.s, snorm = (T)sp.norm;
  const T th_ab = scale ? (T)sp.beta[0] * (-tws[b0 + bb].im) + (T)sp.beta[1] * (-tws[a].im) : T(0);
  C y[N2];
  cf_for<0, N2>([&](auto j2c) { y[decltype(j2c)::value] = row[N2 * k1 + decltype(j2c)::value]; });
  cf_dft<T, N2>(y);
  cf_for<0, N2>([&](auto k2c) {
    constexpr int K2 = decltype(k2c)::value;
    const int k = k1 + N1 * K2;
    T r = y[K2].re, i = y[K2].im * cj;
    if (scale) {
      const T th = (th_ab + sb2 * (-tws[k].im)) * sinvh;
      const T c = ss * th;
      const T den = snorm / fma(c, c, T(1));
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
  });
}

// Grid sizes with a compile-time pass (FP32 and FP64 paths): n -> (N1, N2) =
// 200 -> (10, 20), 64 -> (8, 8), 32 -> (4, 8), 20 -> (4, 5), the factors of
// cfdm_factor.
__host__ __device__ constexpr bool cfdm_has_ct(int n) { return n == 200 || n == 64 || n == 32 || n == 20; }

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

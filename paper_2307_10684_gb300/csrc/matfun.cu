// FP64 matrix functions on the GPU: e^X, phi_1(X), phi_2(X) for X = tau A_mu
// (phi_ell as in Sec. 2, Eq. 9), computed once per plan.
//
// Method: the exponential of the augmented matrix
//     Ahat = [[X, I, 0], [0, 0, I], [0, 0, 0]],
//     exp(Ahat) = [[e^X, phi_1(X), phi_2(X)], [0, I, I], [0, 0, I]],
// by Pade [13/13] scaling and squaring (Higham, SIMAX 26, 2005).  Every
// polynomial in Ahat / 2^s is block upper triangular with blocks that are
// polynomials in Xs = X / 2^s, so the 3n x 3n computation is carried out on
// n x n blocks only (c = 2^-s):
//     r(Ahat/2^s) first block row = [q^-1 p,  c q^-1 (p1 - q1),
//                                    c^2 q^-1 (p2 - q1 - q2)]
// with p = sum_j b_j Xs^j, q = sum_j (-1)^j b_j Xs^j, p1 = sum_{j>=1} b_j
// Xs^(j-1), q1 likewise with signs, p2 = sum_{j>=2} b_j Xs^(j-2), q2 likewise.
// Squaring the block form gives the recurrences
//     R13 <- R11 R13 + c R12 + R13,  R12 <- R11 R12 + R12,  R11 <- R11^2,
//     c <- 2c,
// which after s steps leave (e^X, phi_1(X), phi_2(X)) in (R11, R12, R13).
// Pade coefficients come from the closed form b_j = (2m-j)! m! /
// ((2m)! j! (m-j)!), normalised to b_13 = 1, in exact 128-bit integers.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "adr_internal.h"

namespace adr {

static constexpr double kTheta13 = 5.371920351148152;  // Higham 2005, Table 2.3

// b_j / b_13 = (26 - j)! / (j! (13 - j)!), an integer, j = 0..13.
static void pade13(double b[14]) {
  for (int j = 0; j <= 13; ++j) {
    unsigned __int128 num = 1;
    for (int i = 14 - j; i <= 26 - j; ++i) num *= (unsigned __int128)i;  // (26-j)!/(13-j)!
    unsigned __int128 den = 1;
    for (int i = 2; i <= j; ++i) den *= (unsigned __int128)i;
    b[j] = (double)(num / den);
  }
}

__global__ void build_dense_kernel(int n, Tridiag A, double scale, double* __restrict__ X) {
  const int64_t total = (int64_t)n * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / n), j = (int)(e - (int64_t)i * n);
    double a = 0.0;
    if (i == 0) {
      a = (j == 0) ? A.di : (j == 1 ? A.b0 : 0.0);
    } else if (i == n - 1) {
      a = (j == n - 1) ? A.di : (j == n - 2 ? A.bn : 0.0);
    } else {
      a = (j == i - 1) ? A.lo : (j == i ? A.di : (j == i + 1 ? A.up : 0.0));
    }
    X[e] = scale * a;
  }
}

// Y = Ts X for the tridiagonal Ts (row i: lo, di, up; Neumann rows b0, bn)
// scaled by `scale`; X == nullptr stands for the identity.
__global__ void tridiag_apply_kernel(int n, Tridiag A, double scale, const double* __restrict__ X,
                                     double* __restrict__ Y) {
  const int64_t total = (int64_t)n * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / n), j = (int)(e - (int64_t)i * n);
    auto x = [&](int r) -> double {
      return X ? X[(int64_t)r * n + j] : (r == j ? 1.0 : 0.0);
    };
    double y;
    if (i == 0)
      y = A.di * x(0) + A.b0 * x(1);
    else if (i == n - 1)
      y = A.bn * x(n - 2) + A.di * x(n - 1);
    else
      y = A.lo * x(i - 1) + A.di * x(i) + A.up * x(i + 1);
    Y[e] = scale * y;
  }
}

// ||Ts||_1 for the tridiagonal operator (column abs sums).
__global__ void norm1_tridiag_kernel(int n, Tridiag A, double scale, unsigned long long* out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  auto a = [&](int i, int jj) -> double {
    if (i < 0 || i >= n) return 0.0;
    if (i == 0) return jj == 0 ? A.di : (jj == 1 ? A.b0 : 0.0);
    if (i == n - 1) return jj == n - 1 ? A.di : (jj == n - 2 ? A.bn : 0.0);
    return jj == i - 1 ? A.lo : (jj == i ? A.di : (jj == i + 1 ? A.up : 0.0));
  };
  const double s = fabs(scale) * (fabs(a(j - 1, j)) + fabs(a(j, j)) + fabs(a(j + 1, j)));
  atomicMax(out, (unsigned long long)__double_as_longlong(s));
}

// out_b += coef[b] * P for the four polynomial accumulators (P == nullptr:
// identity).
struct Coef4 {
  double c[4];
};
__global__ void accumulate4_kernel(int n, const double* __restrict__ P, Coef4 coef,
                                   double* __restrict__ Q0, double* __restrict__ Q1,
                                   double* __restrict__ Q2, double* __restrict__ Q3) {
  const int64_t total = (int64_t)n * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / n), j = (int)(e - (int64_t)i * n);
    const double x = P ? P[e] : (i == j ? 1.0 : 0.0);
    if (x == 0.0) continue;
    Q0[e] += coef.c[0] * x;
    Q1[e] += coef.c[1] * x;
    Q2[e] += coef.c[2] * x;
    Q3[e] += coef.c[3] * x;
  }
}

// In-place LU with partial pivoting of a banded matrix (lower bandwidth bl,
// upper bandwidth bu before pivoting) held in dense row-major storage, one
// thread block, steps in sequence.  Row interchanges are applied to columns
// >= k only, so the multipliers of column k stay in place (the forward solve
// applies the interchanges in the same order).  piv[k] = row swapped with k.
__global__ void __launch_bounds__(1024) band_lu_kernel(int n, int bl, int bu, double* __restrict__ Q,
                                                       int* __restrict__ piv,
                                                       int* __restrict__ info) {
  __shared__ int sp;
  const int tid = threadIdx.x;
  const int wu = bl + bu;  // upper bandwidth of U
  for (int k = 0; k < n; ++k) {
    const int rlast = min(n - 1, k + bl);
    const int clast = min(n - 1, k + wu);
    if (tid < 32) {
      double best = -1.0;
      int bi = k;
      for (int i = k + tid; i <= rlast; i += 32) {
        const double a = fabs(Q[(int64_t)i * n + k]);
        if (a > best) {
          best = a;
          bi = i;
        }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) {
          best = ob;
          bi = oi;
        }
      }
      if (tid == 0) {
        sp = bi;
        piv[k] = bi;
      }
    }
    __syncthreads();
    const int p = sp;
    if (p != k) {
      for (int j = k + tid; j <= clast; j += blockDim.x) {
        const double t = Q[(int64_t)k * n + j];
        Q[(int64_t)k * n + j] = Q[(int64_t)p * n + j];
        Q[(int64_t)p * n + j] = t;
      }
    }
    __syncthreads();
    const double pv = Q[(int64_t)k * n + k];
    if (pv == 0.0) {
      if (tid == 0 && *info == 0) *info = k + 1;
      __syncthreads();
      continue;
    }
    for (int i = k + 1 + tid; i <= rlast; i += blockDim.x) Q[(int64_t)i * n + k] /= pv;
    __syncthreads();
    const int nr = rlast - k, nc = clast - k;
    for (int t = tid; t < nr * nc; t += blockDim.x) {
      const int i = k + 1 + t / nc, j = k + 1 + t % nc;
      Q[(int64_t)i * n + j] -= Q[(int64_t)i * n + k] * Q[(int64_t)k * n + j];
    }
    __syncthreads();
  }
}

// Solve q y = rhs for every column of three n x n right-hand sides using the
// banded LU above; one thread per column, y overwrites rhs and is scaled by
// scale_b at the end.
__global__ void band_solve_kernel(int n, int bl, int bu, const double* __restrict__ Q,
                                  const int* __restrict__ piv, double* R0, double* R1, double* R2,
                                  double s0, double s1, double s2) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= 3 * n) return;
  const int b = g / n, j = g - b * n;
  double* Y = b == 0 ? R0 : (b == 1 ? R1 : R2);
  const double sc = b == 0 ? s0 : (b == 1 ? s1 : s2);
  const int wu = bl + bu;
  for (int k = 0; k < n; ++k) {
    const int p = piv[k];
    double yk = Y[(int64_t)k * n + j];
    if (p != k) {
      const double yp = Y[(int64_t)p * n + j];
      Y[(int64_t)p * n + j] = yk;
      yk = yp;
      Y[(int64_t)k * n + j] = yk;
    }
    const int rlast = min(n - 1, k + bl);
    for (int i = k + 1; i <= rlast; ++i) Y[(int64_t)i * n + j] -= Q[(int64_t)i * n + k] * yk;
  }
  for (int k = n - 1; k >= 0; --k) {
    double s = Y[(int64_t)k * n + j];
    const int clast = min(n - 1, k + wu);
    for (int jj = k + 1; jj <= clast; ++jj) s -= Q[(int64_t)k * n + jj] * Y[(int64_t)jj * n + j];
    Y[(int64_t)k * n + j] = s / Q[(int64_t)k * n + k];
  }
  for (int k = 0; k < n; ++k) Y[(int64_t)k * n + j] *= sc;
}

__global__ void convert_kernel(const double* __restrict__ src, void* __restrict__ dst, int64_t count,
                               int to_double, int transpose_n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t se = e;
    if (transpose_n > 0) {  // dst[i][j] = src[j][i]
      const int64_t i = e / transpose_n, j = e - i * transpose_n;
      se = j * transpose_n + i;
    }
    if (to_double)
      ((double*)dst)[e] = src[se];
    else
      ((float*)dst)[e] = (float)src[se];
  }
}

__global__ void max_abs_diff_kernel(const void* __restrict__ x, int x_is_double,
                                    const double* __restrict__ ref, int64_t count,
                                    unsigned long long* out2) {
  double md = 0.0, mr = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count;
       e += (int64_t)gridDim.x * blockDim.x) {
    const double xv = x_is_double ? ((const double*)x)[e] : (double)((const float*)x)[e];
    const double r = ref[e];
    const double dd = fabs(xv - r);
    md = (dd > md || dd != dd) ? dd : md;  // NaN propagates
    mr = fmax(mr, fabs(r));
  }
  for (int o = 16; o > 0; o >>= 1) {
    const double a = __shfl_xor_sync(0xffffffffu, md, o);
    md = (a > md || a != a) ? a : md;
    mr = fmax(mr, __shfl_xor_sync(0xffffffffu, mr, o));
  }
  if ((threadIdx.x & 31) == 0) {
    // NaN maps to the largest pattern so that it wins the maximum
    const unsigned long long bd =
        (md != md) ? 0x7ff8000000000000ull : (unsigned long long)__double_as_longlong(md);
    atomicMax(&out2[0], bd);
    atomicMax(&out2[1], (unsigned long long)__double_as_longlong(mr));
  }
}

// Weighted sums for the dynamics indicators: acc[0] += w u, acc[1] += w v,
// acc[2] += (u - up)^2, acc[3] += (v - vp)^2 with trapezoid weights w.
__global__ void __launch_bounds__(256) indicators_kernel(PointwiseArgs a, const void* __restrict__ up,
                                                         const void* __restrict__ vp,
                                                         const void* __restrict__ u,
                                                         const void* __restrict__ v, int is_double,
                                                         double* __restrict__ acc) {
  double s[4] = {0.0, 0.0, 0.0, 0.0};
  const int64_t n1 = a.n[0], n2 = a.n[1], n3 = a.d == 3 ? a.n[2] : 1;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < a.N;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i1 = e % n1, r = e / n1, i2 = r % n2, i3 = r / n2;
    double w = (i1 == 0 || i1 == n1 - 1) ? 0.5 : 1.0;
    w *= (i2 == 0 || i2 == n2 - 1) ? 0.5 : 1.0;
    if (a.d == 3) w *= (i3 == 0 || i3 == n3 - 1) ? 0.5 : 1.0;
    double x, y, xp, yp;
    if (is_double) {
      x = ((const double*)u)[e];
      y = ((const double*)v)[e];
      xp = ((const double*)up)[e];
      yp = ((const double*)vp)[e];
    } else {
      x = ((const float*)u)[e];
      y = ((const float*)v)[e];
      xp = ((const float*)up)[e];
      yp = ((const float*)vp)[e];
    }
    s[0] += w * x;
    s[1] += w * y;
    s[2] += (x - xp) * (x - xp);
    s[3] += (y - yp) * (y - yp);
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    double t = s[k];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(&acc[k], t);
  }
}

static int grid_for(int64_t total) {
  int64_t b = (total + 255) / 256;
  if (b < 1) b = 1;
  if (b > 152 * 16) b = 152 * 16;
  return (int)b;
}

cudaError_t launch_indicators(const PointwiseArgs& a, const void* up, const void* vp,
                              const void* u, const void* v, int is_double, double* acc,
                              cudaStream_t s) {
  indicators_kernel<<<grid_for(a.N), 256, 0, s>>>(a, up, vp, u, v, is_double, acc);
  return cudaGetLastError();
}

cudaError_t launch_build_dense(int n, const Tridiag& A, double scale, double* X, cudaStream_t s) {
  build_dense_kernel<<<grid_for((int64_t)n * n), 256, 0, s>>>(n, A, scale, X);
  return cudaGetLastError();
}

cudaError_t launch_convert(const double* src, void* dst, int64_t count, int to_double,
                           int transpose_n, cudaStream_t s) {
  convert_kernel<<<grid_for(count), 256, 0, s>>>(src, dst, count, to_double, transpose_n);
  return cudaGetLastError();
}

cudaError_t launch_max_abs_diff(const void* x, int x_is_double, const double* ref, int64_t count,
                                unsigned long long* out2, cudaStream_t s) {
  max_abs_diff_kernel<<<grid_for(count), 256, 0, s>>>(x, x_is_double, ref, count, out2);
  return cudaGetLastError();
}

// RAII list of device allocations for one matfun call.
struct DevBufs {
  std::vector<void*> p;
  ~DevBufs() {
    for (void* q : p) cudaFree(q);
  }
  cudaError_t alloc(double** out, size_t count) {
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, count * sizeof(double));
    if (e != cudaSuccess) return e;
    p.push_back(q);
    *out = (double*)q;
    return cudaSuccess;
  }
};

#define MF_TRY(x)                          \
  do {                                     \
    cudaError_t e_ = (x);                  \
    if (e_ != cudaSuccess) return e_;      \
  } while (0)

static cudaError_t gemm64(int n, const double* A, const double* B, double* C, const double* base,
                          double beta, const double* base2, double beta2, cudaStream_t s) {
  GemmArgs g{};
  g.A[0] = A;
  g.B[0] = B;
  g.C[0] = C;
  g.base[0] = base;
  g.base2[0] = base2;
  g.lda = g.ldb = g.ldc = n;
  g.M = g.N = g.K = n;
  g.batch = 1;
  g.ncomp = 1;
  g.alpha = 1.0;
  g.beta = beta;
  g.beta2 = beta2;
  return launch_gemm_simt<double>(g, s);
}

// Evaluate (e^X, phi_1(X), phi_2(X)) for X = tau * A into E, P1, P2 (device,
// row-major n x n).  A is tridiagonal, so the powers Xs^k (k <= 13) are
// banded with bandwidth k and q(Xs) has bandwidth 13: powers are formed by
// three-term recurrences and q is factorised as a band matrix; only the
// squaring phase uses dense products.  Synchronises the stream.
// Xs = scale * A for a dense row-major A (the first power of the dense path).
__global__ void scale_kernel(const double* __restrict__ A, double scale, double* __restrict__ X,
                             int64_t total) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x)
    X[e] = scale * A[e];
}

static cudaError_t matfun_core(int n, const Tridiag* Atri, const double* Adense, double norm1,
                               double tau, double* E, double* P1, double* P2, cudaStream_t s);

cudaError_t matfun_phi_dense(int n, const double* A, double norm1_A, double tau, double* E,
                             double* P1, double* P2, cudaStream_t s) {
  return matfun_core(n, nullptr, A, norm1_A * tau, tau, E, P1, P2, s);
}

cudaError_t matfun_phi(int n, const Tridiag& A, double tau, double* E, double* P1, double* P2,
                       cudaStream_t s) {
  return matfun_core(n, &A, nullptr, -1.0, tau, E, P1, P2, s);
}

// The same algorithm for a tridiagonal A (banded powers and band LU) or a
// dense A (norm1 = ||tau A||_1 given; dense products and a full-bandwidth
// LU).
static cudaError_t matfun_core(int n, const Tridiag* Atri, const double* Adense, double norm1,
                               double tau, double* E, double* P1, double* P2, cudaStream_t s) {
  DevBufs mem;
  const size_t nn = (size_t)n * n;
  double *Pa, *Pb, *Qm, *Pm, *R1m, *R2m, *T1, *T2, *T3;
  unsigned long long* nrm;
  int *info, *piv;
  MF_TRY(mem.alloc(&Pa, nn));
  MF_TRY(mem.alloc(&Pb, nn));
  MF_TRY(mem.alloc(&Qm, nn));
  MF_TRY(mem.alloc(&Pm, nn));
  MF_TRY(mem.alloc(&R1m, nn));
  MF_TRY(mem.alloc(&R2m, nn));
  MF_TRY(mem.alloc(&T1, nn));
  MF_TRY(mem.alloc(&T2, nn));
  MF_TRY(mem.alloc(&T3, nn));
  MF_TRY(mem.alloc((double**)&nrm, 1));
  MF_TRY(mem.alloc((double**)&info, 1));
  MF_TRY(mem.alloc((double**)&piv, (size_t)n));  // n ints fit in n doubles

  // ||tau A||_1 -> scaling power s (the augmented matrix's identity blocks
  // have column norm 1 < theta_13, so only X matters)
  MF_TRY(cudaMemsetAsync(nrm, 0, sizeof(unsigned long long), s));
  MF_TRY(cudaMemsetAsync(info, 0, sizeof(int), s));
  double norm = norm1;
  if (Atri) {
    norm1_tridiag_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, *Atri, tau, nrm);
    MF_TRY(cudaGetLastError());
    unsigned long long nbits = 0;
    MF_TRY(cudaMemcpyAsync(&nbits, nrm, sizeof(nbits), cudaMemcpyDeviceToHost, s));
    MF_TRY(cudaStreamSynchronize(s));
    memcpy(&norm, &nbits, sizeof(norm));
  }
  int sp = 0;
  if (norm > kTheta13) sp = std::max(0, (int)ceil(log2(norm / kTheta13)));
  const double c = ldexp(1.0, -sp);
  const double xs = tau * c;  // Xs = xs * A  (exact power-of-two scaling of tau A)

  double b[14];
  pade13(b);
  // coefficient of Xs^k in q, p, p1 - q1, p2 - q1 - q2
  auto coef = [&](int k) {
    Coef4 cf;
    const double sg = (k % 2 == 0) ? 1.0 : -1.0;
    const double bk = b[k];
    const double bk1 = (k + 1 <= 13) ? b[k + 1] : 0.0;
    const double bk2 = (k + 2 <= 13) ? b[k + 2] : 0.0;
    cf.c[0] = sg * bk;                                      // q
    cf.c[1] = bk;                                           // p
    cf.c[2] = (k % 2 == 0) ? 2.0 * bk1 : 0.0;               // p1 - q1
    cf.c[3] = ((k % 2 == 1) ? 2.0 * bk2 : 0.0) + sg * bk1;  // p2 - q1 - q2
    return cf;
  };
  for (double* q : {Qm, Pm, R1m, R2m}) MF_TRY(cudaMemsetAsync(q, 0, nn * sizeof(double), s));
  const int g = grid_for((int64_t)nn);
  accumulate4_kernel<<<g, 256, 0, s>>>(n, nullptr, coef(0), Qm, Pm, R1m, R2m);
  MF_TRY(cudaGetLastError());
  const double* prev = nullptr;  // identity
  double* bufs[2] = {Pa, Pb};
  double* X1 = nullptr;  // dense path: Xs, the factor of every power
  if (Adense) {
    MF_TRY(mem.alloc(&X1, nn));
    scale_kernel<<<g, 256, 0, s>>>(Adense, xs, X1, (int64_t)nn);
    MF_TRY(cudaGetLastError());
  }
  for (int k = 1; k <= 13; ++k) {
    double* cur = bufs[k & 1];
    if (Atri) {
      tridiag_apply_kernel<<<g, 256, 0, s>>>(n, *Atri, xs, prev, cur);
      MF_TRY(cudaGetLastError());
    } else if (k == 1) {
      MF_TRY(cudaMemcpyAsync(cur, X1, nn * sizeof(double), cudaMemcpyDeviceToDevice, s));
    } else {
      MF_TRY(gemm64(n, prev, X1, cur, nullptr, 0.0, nullptr, 0.0, s));
    }
    accumulate4_kernel<<<g, 256, 0, s>>>(n, cur, coef(k), Qm, Pm, R1m, R2m);
    MF_TRY(cudaGetLastError());
    prev = cur;
  }

  // q R = [p | p1 - q1 | p2 - q1 - q2] (LU with partial pivoting: banded for
  // a tridiagonal A, full bandwidth for a dense one)
  const int bl = Atri ? 13 : n - 1, bu = Atri ? 13 : n - 1;
  band_lu_kernel<<<1, 1024, 0, s>>>(n, bl, bu, Qm, piv, info);
  MF_TRY(cudaGetLastError());
  band_solve_kernel<<<(3 * n + 127) / 128, 128, 0, s>>>(n, bl, bu, Qm, piv, Pm, R1m, R2m, 1.0, c,
                                                        c * c);
  MF_TRY(cudaGetLastError());
  double* R11 = Pm;
  double* R12 = R1m;
  double* R13 = R2m;

  // squaring
  double* S11 = T1;
  double* S12 = T2;
  double* S13 = T3;
  double cc = c;
  for (int it = 0; it < sp; ++it) {
    MF_TRY(gemm64(n, R11, R13, S13, R13, 1.0, R12, cc, s));
    MF_TRY(gemm64(n, R11, R12, S12, R12, 1.0, nullptr, 0.0, s));
    MF_TRY(gemm64(n, R11, R11, S11, nullptr, 0.0, nullptr, 0.0, s));
    std::swap(R11, S11);
    std::swap(R12, S12);
    std::swap(R13, S13);
    cc *= 2.0;
  }
  MF_TRY(cudaMemcpyAsync(E, R11, nn * sizeof(double), cudaMemcpyDeviceToDevice, s));
  MF_TRY(cudaMemcpyAsync(P1, R12, nn * sizeof(double), cudaMemcpyDeviceToDevice, s));
  MF_TRY(cudaMemcpyAsync(P2, R13, nn * sizeof(double), cudaMemcpyDeviceToDevice, s));
  int hinfo = 0;
  MF_TRY(cudaMemcpyAsync(&hinfo, info, sizeof(int), cudaMemcpyDeviceToHost, s));
  MF_TRY(cudaStreamSynchronize(s));  // also keeps `mem` alive until the work is done
  if (hinfo != 0) return cudaErrorInvalidValue;  // singular Pade denominator
  return cudaSuccess;
}

}  // namespace adr

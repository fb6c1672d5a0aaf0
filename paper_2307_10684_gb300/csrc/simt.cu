// SIMT kernels of the FP64 and FP32 paths: register-blocked batched GEMM
// for the mu-mode products (Sec. 2, Eq. 5), the stage-1 right-hand side
// W = sum_mu U x_mu A_mu + G(U, V) (Eq. 6, Eq. 11) and the stage-2 reaction
// difference D = G(U2, V2) - G(U, V) (Eq. 11).
#include <cuda_runtime.h>
#include <stdint.h>

#include "adr_internal.h"
#include "pointwise.cuh"

namespace adr {

template <typename T>
__global__ void __launch_bounds__(128) rhs_kernel(PointwiseArgsT<T> a, const T* __restrict__ u,
                                                  const T* __restrict__ v, T* __restrict__ wu,
                                                  T* __restrict__ wv) {
  const int i1 = blockIdx.x * blockDim.x + threadIdx.x;
  if (i1 >= (int)a.n[0]) return;
  const int i2 = blockIdx.y, i3 = blockIdx.z;
  const int64_t idx = ((int64_t)i3 * a.n[1] + i2) * a.n[0] + i1;
  T x, y;
  rhs_point<T>(a, u, v, idx, i1, i2, i3, x, y);
  wu[idx] = x;
  wv[idx] = y;
}

template <typename T>
__global__ void __launch_bounds__(256) rdiff_kernel(PointwiseArgsT<T> a, const T* __restrict__ u,
                                                    const T* __restrict__ v,
                                                    const T* __restrict__ u2,
                                                    const T* __restrict__ v2, T* __restrict__ du,
                                                    T* __restrict__ dv) {
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < a.N;
       idx += (int64_t)gridDim.x * blockDim.x) {
    react_diff<T>(a.rx, u[idx], v[idx], u2[idx], v2[idx], du[idx], dv[idx]);
  }
}

// Lawson2b (Eq. 7) pointwise stages: x = u + scale G^u(u, v) (both
// components), and u += scale G^u(u2, v2).
template <typename T>
__global__ void __launch_bounds__(256) lawson_pre_kernel(PointwiseArgsT<T> a, const T* __restrict__ u,
                                                         const T* __restrict__ v, T scale,
                                                         T* __restrict__ xu, T* __restrict__ xv) {
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < a.N;
       idx += (int64_t)gridDim.x * blockDim.x) {
    T gu, gv;
    const T uu = u[idx], vv = v[idx];
    react<T>(a.rx, uu, vv, gu, gv);
    xu[idx] = uu + scale * gu;
    xv[idx] = vv + scale * gv;
  }
}

template <typename T>
__global__ void __launch_bounds__(256) lawson_post_kernel(PointwiseArgsT<T> a,
                                                          const T* __restrict__ u2,
                                                          const T* __restrict__ v2, T scale,
                                                          T* __restrict__ u, T* __restrict__ v) {
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < a.N;
       idx += (int64_t)gridDim.x * blockDim.x) {
    T gu, gv;
    react<T>(a.rx, u2[idx], v2[idx], gu, gv);
    u[idx] += scale * gu;
    v[idx] += scale * gv;
  }
}

static int pointwise_grid(int64_t N) {
  int64_t b = (N + 255) / 256;
  const int64_t cap = 152 * 16;
  return (int)(b < cap ? (b < 1 ? 1 : b) : cap);
}

template <typename T>
cudaError_t launch_rhs(const PointwiseArgsT<T>& a, const T* u, const T* v, T* wu, T* wv,
                       cudaStream_t s) {
  dim3 grid((unsigned)((a.n[0] + 127) / 128), (unsigned)a.n[1], (unsigned)(a.d == 3 ? a.n[2] : 1));
  rhs_kernel<T><<<grid, 128, 0, s>>>(a, u, v, wu, wv);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_rdiff(const PointwiseArgsT<T>& a, const T* u, const T* v, const T* u2, const T* v2,
                         T* du, T* dv, cudaStream_t s) {
  rdiff_kernel<T><<<pointwise_grid(a.N), 256, 0, s>>>(a, u, v, u2, v2, du, dv);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_lawson_pre(const PointwiseArgsT<T>& a, const T* u, const T* v, T scale, T* xu,
                              T* xv, cudaStream_t s) {
  lawson_pre_kernel<T><<<pointwise_grid(a.N), 256, 0, s>>>(a, u, v, scale, xu, xv);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_lawson_post(const PointwiseArgsT<T>& a, const T* u2, const T* v2, T scale, T* u,
                               T* v, cudaStream_t s) {
  lawson_post_kernel<T><<<pointwise_grid(a.N), 256, 0, s>>>(a, u2, v2, scale, u, v);
  return cudaGetLastError();
}

template cudaError_t launch_lawson_pre<float>(const PointwiseArgsT<float>&, const float*,
                                              const float*, float, float*, float*, cudaStream_t);
template cudaError_t launch_lawson_pre<double>(const PointwiseArgsT<double>&, const double*,
                                               const double*, double, double*, double*,
                                               cudaStream_t);
template cudaError_t launch_lawson_post<float>(const PointwiseArgsT<float>&, const float*,
                                               const float*, float, float*, float*, cudaStream_t);
template cudaError_t launch_lawson_post<double>(const PointwiseArgsT<double>&, const double*,
                                                const double*, double, double*, double*,
                                                cudaStream_t);
template cudaError_t launch_rhs<float>(const PointwiseArgsT<float>&, const float*, const float*, float*,
                                       float*, cudaStream_t);
template cudaError_t launch_rhs<double>(const PointwiseArgsT<double>&, const double*, const double*,
                                        double*, double*, cudaStream_t);
template cudaError_t launch_rdiff<float>(const PointwiseArgsT<float>&, const float*, const float*,
                                         const float*, const float*, float*, float*,
                                         cudaStream_t);
template cudaError_t launch_rdiff<double>(const PointwiseArgsT<double>&, const double*, const double*,
                                          const double*, const double*, double*, double*,
                                          cudaStream_t);

// ---------------------------------------------------------------- GEMM
// Tile configuration: 256 threads as a 16 x 16 grid; each thread owns a
// TM x TN block of C split into 4-wide groups spread over the tile so that
// shared-memory reads are conflict free.
template <typename T>
struct SimtTile;
template <>
struct SimtTile<float> {
  static constexpr int BM = 128, BN = 128, BK = 8, TM = 8, TN = 8;
};
template <>
struct SimtTile<double> {
  static constexpr int BM = 64, BN = 64, BK = 8, TM = 4, TN = 4;
};

template <typename T>
__global__ void __launch_bounds__(256) gemm_simt_kernel(GemmArgs g) {
  using Cfg = SimtTile<T>;
  constexpr int BM = Cfg::BM, BN = Cfg::BN, BK = Cfg::BK, TM = Cfg::TM, TN = Cfg::TN;
  constexpr int LA = BM * BK / 256;  // A elements loaded per thread (along k)
  constexpr int LB = BK * BN / 256;  // B elements loaded per thread (along n)
  constexpr int RS = TM / 4, CS = TN / 4;

  __shared__ __align__(16) T As[2][BK][BM];
  __shared__ __align__(16) T Bs[2][BK][BN];

  const int z = blockIdx.z;
  const int comp = z / g.batch;
  const int p = z - comp * g.batch;
  const T* __restrict__ A = (const T*)g.A[comp] + (int64_t)p * g.a_bs;
  const T* __restrict__ B = (const T*)g.B[comp] + (int64_t)p * g.b_bs;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int t = threadIdx.x;
  const int tx = t & 15, ty = t >> 4;

  // load coordinates
  const int a_row = t / (BK / LA), a_k = (t % (BK / LA)) * LA;
  const int b_k = t / (BN / LB), b_n = (t % (BN / LB)) * LB;

  T ra[LA], rb[LB];
  auto load_tiles = [&](int k0) {
    const int gr = m0 + a_row;
#pragma unroll
    for (int i = 0; i < LA; ++i) {
      const int gk = k0 + a_k + i;
      ra[i] = (gr < g.M && gk < g.K) ? A[(int64_t)gr * g.lda + gk] : (T)0;
    }
    const int gk = k0 + b_k;
#pragma unroll
    for (int i = 0; i < LB; ++i) {
      const int gn = n0 + b_n + i;
      rb[i] = (gk < g.K && gn < g.N) ? B[(int64_t)gk * g.ldb + gn] : (T)0;
    }
  };
  auto store_tiles = [&](int buf) {
#pragma unroll
    for (int i = 0; i < LA; ++i) As[buf][a_k + i][a_row] = ra[i];
#pragma unroll
    for (int i = 0; i < LB; ++i) Bs[buf][b_k][b_n + i] = rb[i];
  };

  T acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = (T)0;

  load_tiles(0);
  store_tiles(0);
  __syncthreads();

  const int ktiles = (g.K + BK - 1) / BK;
  for (int kt = 0; kt < ktiles; ++kt) {
    const int cur = kt & 1;
    if (kt + 1 < ktiles) load_tiles((kt + 1) * BK);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[TM], b[TN];
#pragma unroll
      for (int r = 0; r < RS; ++r)
#pragma unroll
        for (int i = 0; i < 4; ++i) a[r * 4 + i] = As[cur][kk][r * (BM / RS) + ty * 4 + i];
#pragma unroll
      for (int c = 0; c < CS; ++c)
#pragma unroll
        for (int j = 0; j < 4; ++j) b[c * 4 + j] = Bs[cur][kk][c * (BN / CS) + tx * 4 + j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    if (kt + 1 < ktiles) {
      store_tiles(cur ^ 1);
    }
    __syncthreads();
  }

  // epilogue
  T* __restrict__ C = (T*)g.C[comp] + (int64_t)p * g.c_bs;
  const T* __restrict__ base = g.base[comp] ? (const T*)g.base[comp] + (int64_t)p * g.c_bs : nullptr;
  const T* __restrict__ base2 =
      g.base2[comp] ? (const T*)g.base2[comp] + (int64_t)p * g.c_bs : nullptr;
  const T alpha = (T)g.alpha, beta = (T)g.beta, beta2 = (T)g.beta2;
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int r = m0 + (i / 4) * (BM / RS) + ty * 4 + (i % 4);
    if (r >= g.M) continue;
    // gather the row's epilogue inputs before any store (C may share no
    // memory with base/base2, but the compiler cannot assume it)
    T extra[TN];
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int c = n0 + (j / 4) * (BN / CS) + tx * 4 + (j % 4);
      const int64_t o = (int64_t)r * g.ldc + c;
      T x = (T)0;
      if (c < g.N) {
        if (base) x += beta * base[o];
        if (base2) x += beta2 * base2[o];
      }
      extra[j] = x;
    }
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int c = n0 + (j / 4) * (BN / CS) + tx * 4 + (j % 4);
      if (c < g.N) C[(int64_t)r * g.ldc + c] = alpha * acc[i][j] + extra[j];
    }
  }
}

// Small-problem variant: an 8 x 8 output tile per 64-thread CTA, one output
// per thread.  Used when the register-blocked kernel would leave most SMs
// idle (GB300 runs FP64 at about two FMAs per clock per SM, so a 64^3
// product on a single SM takes tens of microseconds).
template <typename T>
__global__ void __launch_bounds__(64) gemm_small_kernel(GemmArgs g) {
  constexpr int TS = 8;
  __shared__ T As[TS][TS + 1];
  __shared__ T Bs[TS][TS + 1];
  const int z = blockIdx.z;
  const int comp = z / g.batch;
  const int p = z - comp * g.batch;
  const T* __restrict__ A = (const T*)g.A[comp] + (int64_t)p * g.a_bs;
  const T* __restrict__ B = (const T*)g.B[comp] + (int64_t)p * g.b_bs;
  const int tx = threadIdx.x & 7, ty = threadIdx.x >> 3;
  const int r = blockIdx.y * TS + ty, c = blockIdx.x * TS + tx;
  T acc = (T)0;
  for (int k0 = 0; k0 < g.K; k0 += TS) {
    As[ty][tx] = (r < g.M && k0 + tx < g.K) ? A[(int64_t)r * g.lda + k0 + tx] : (T)0;
    Bs[ty][tx] = (k0 + ty < g.K && c < g.N) ? B[(int64_t)(k0 + ty) * g.ldb + c] : (T)0;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < TS; ++k) acc = fma(As[ty][k], Bs[k][tx], acc);
    __syncthreads();
  }
  if (r < g.M && c < g.N) {
    const int64_t o = (int64_t)r * g.ldc + c;
    T* __restrict__ C = (T*)g.C[comp] + (int64_t)p * g.c_bs;
    T x = (T)g.alpha * acc;
    if (g.base[comp]) x += (T)g.beta * ((const T*)g.base[comp] + (int64_t)p * g.c_bs)[o];
    if (g.base2[comp]) x += (T)g.beta2 * ((const T*)g.base2[comp] + (int64_t)p * g.c_bs)[o];
    C[o] = x;
  }
}

template <typename T>
cudaError_t launch_gemm_simt(const GemmArgs& g, cudaStream_t s) {
  using Cfg = SimtTile<T>;
  if (g.M <= 0 || g.N <= 0) return cudaSuccess;
  dim3 grid((g.N + Cfg::BN - 1) / Cfg::BN, (g.M + Cfg::BM - 1) / Cfg::BM, g.batch * g.ncomp);
  // FP64 runs ~40x slower per SM than FP32, so FP64 products spread over
  // small tiles whenever the large tiles leave SMs idle; FP32 only for tiny
  // problems
  const int64_t min_ctas = sizeof(T) == 8 ? 152 : 32;
  if ((int64_t)grid.x * grid.y * grid.z < min_ctas) {
    dim3 sg((g.N + 7) / 8, (g.M + 7) / 8, g.batch * g.ncomp);
    if (sg.y > 65535 || sg.z > 65535) return cudaErrorInvalidConfiguration;
    gemm_small_kernel<T><<<sg, 64, 0, s>>>(g);
    return cudaGetLastError();
  }
  if (grid.y > 65535 || grid.z > 65535) return cudaErrorInvalidConfiguration;
  gemm_simt_kernel<T><<<grid, 256, 0, s>>>(g);
  return cudaGetLastError();
}

template cudaError_t launch_gemm_simt<float>(const GemmArgs&, cudaStream_t);
template cudaError_t launch_gemm_simt<double>(const GemmArgs&, cudaStream_t);

}  // namespace adr

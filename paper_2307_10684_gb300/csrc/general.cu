// General ETD2RKds plans: m = 1..4 components, directional matrices A_mu^c
// given densely by the caller, polynomial reactions.
//
// The method needs nothing of the A_mu but their size (Sec. 1, Eq. 3-4: any
// matrices in the Kronecker sum) and extends to more than two components
// (Sec. 3, closing remark).  One step is Eq. 11 for every component c:
//     W_c  = sum_mu U_c x_mu A_mu^c + G_c(U)               (mode products)
//     U2_c = U_c + tau W_c x_1 phi_1(tau A_1^c) ... x_d phi_1(tau A_d^c)
//     D_c  = G_c(U2) - G_c(U)                              (all U2 first)
//     U_c <- U2_c + 2^(d-1) tau D_c x_mu phi_2(tau A_mu^c)
// K U is a sum of d dense mode products (the finite-difference plans use a
// stencil instead).  The products run on the FP64 / FP32 SIMT GEMM, in the
// natural layout; the matrix functions come from the dense path of the FP64
// Pade scaling and squaring on the GPU.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <string>
#include <vector>

#include "adr_internal.h"

namespace adr {

constexpr int kMaxTerms = 64;

struct PolyTerms {
  int n, m;
  int comp[kMaxTerms];
  int pw[kMaxTerms][4];
  double coef[kMaxTerms];
};

// g^c(U) for every component at one point.
template <typename T>
__device__ __forceinline__ void poly_eval(const PolyTerms& P, const T (&u)[4], T (&g)[4]) {
  for (int c = 0; c < 4; ++c) g[c] = (T)0;
  for (int t = 0; t < P.n; ++t) {
    T x = (T)P.coef[t];
    for (int j = 0; j < P.m; ++j)
      for (int e = 0; e < P.pw[t][j]; ++e) x *= u[j];
    g[P.comp[t]] += x;
  }
}

struct GenPtrs {
  const void* u[4];
  const void* u2[4];
  void* w[4];
};

// W_c += G_c(U) (stage 1) or W_c = G_c(U2) - G_c(U) (stage 2, u2 set).
template <typename T>
__global__ void __launch_bounds__(256) poly_kernel(const __grid_constant__ PolyTerms P, GenPtrs q,
                                                   int64_t N, int stage2) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    T u[4] = {(T)0, (T)0, (T)0, (T)0}, g[4];
    for (int j = 0; j < P.m; ++j) u[j] = ((const T*)q.u[j])[i];
    poly_eval<T>(P, u, g);
    if (stage2) {
      T u2[4] = {(T)0, (T)0, (T)0, (T)0}, g2[4];
      for (int j = 0; j < P.m; ++j) u2[j] = ((const T*)q.u2[j])[i];
      poly_eval<T>(P, u2, g2);
      for (int c = 0; c < P.m; ++c) ((T*)q.w[c])[i] = g2[c] - g[c];
    } else {
      for (int c = 0; c < P.m; ++c) ((T*)q.w[c])[i] += g[c];
    }
  }
}

struct GeneralState {
  int m;
  PolyTerms terms;
  // FP64 masters [c][mu][which]: 0 = A, 1 = e^(tau A), 2 = phi_1, 3 = phi_2
  double* master[4][3][4];
  // state-type operands [c][mu][k], k: 0 = A, 1 = phi_1, 2 = phi_2; row-major and transposed
  void* op[4][3][3];
  void* opT[4][3][3];
  void* w[4];
  void* u2[4];
  void* t0[4];
  void* t1[4];
};

static int grid_of(int64_t N) {
  int64_t b = (N + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  return (int)(b < 1 ? 1 : b);
}

// out = alpha * (in x_mu M) + beta * base for one component, natural layout
// (x_1 fastest): mode 1 is X M^T over the rows of length n_1, mode mu > 1 is
// M X over the n_mu x (n_1 .. n_{mu-1}) slabs.
template <typename T>
static cudaError_t mode_one(adr_plan P, int mu, const void* M, const void* MT, const void* in,
                            void* out, const void* base, double alpha, double beta) {
  const int64_t n = P->n[mu];
  int64_t Q = 1;
  for (int k = 0; k < mu; ++k) Q *= P->n[k];
  const int64_t Pb = P->N / (n * Q);
  GemmArgs g{};
  g.ncomp = 1;
  g.alpha = alpha;
  g.beta = beta;
  g.C[0] = out;
  g.base[0] = base;
  g.base2[0] = nullptr;
  if (mu == 0) {
    g.A[0] = in;
    g.B[0] = MT;
    g.M = (int)Pb;
    g.N = (int)n;
    g.K = (int)n;
    g.lda = g.ldb = g.ldc = n;
    g.batch = 1;
  } else {
    g.A[0] = M;
    g.B[0] = in;
    g.M = (int)n;
    g.N = (int)Q;
    g.K = (int)n;
    g.lda = n;
    g.ldb = Q;
    g.ldc = Q;
    g.a_bs = 0;
    g.b_bs = n * Q;
    g.c_bs = n * Q;
    g.batch = (int)Pb;
  }
  const double flops = 2.0 * (double)n * (double)P->N;
  const double bytes = (double)sizeof(T) * (2.0 * P->N + (base ? P->N : 0) + n * n);
  return timed_kernel(P, KC_MODE_SIMT, flops, bytes, [&] { return launch_gemm_simt<T>(g, P->stream); });
}

template <typename T>
static cudaError_t step_general(adr_plan P, void* const* U) {
  GeneralState& G = *P->gen;
  const int d = P->d, m = G.m;
  const double tau = P->prob.tau;
  const int64_t N = P->N;
  cudaError_t e = cudaSuccess;
  // W_c = sum_mu U_c x_mu A_mu^c
  for (int c = 0; c < m && e == cudaSuccess; ++c)
    for (int mu = 0; mu < d && e == cudaSuccess; ++mu)
      e = mode_one<T>(P, mu, G.op[c][mu][0], G.opT[c][mu][0], U[c], G.w[c], mu ? G.w[c] : nullptr,
                      1.0, mu ? 1.0 : 0.0);
  if (e != cudaSuccess) return e;
  GenPtrs q{};
  for (int c = 0; c < m; ++c) {
    q.u[c] = U[c];
    q.u2[c] = G.u2[c];
    q.w[c] = G.w[c];
  }
  const int gr = grid_of(N);
  e = timed_kernel(P, KC_RHS, (double)N * 8.0 * G.terms.n, (double)sizeof(T) * N * 3 * m, [&] {
    poly_kernel<T><<<gr, 256, 0, P->stream>>>(G.terms, q, N, 0);
    return cudaGetLastError();
  });
  if (e != cudaSuccess) return e;
  // U2_c = U_c + tau W_c x_mu phi_1, then the stage-2 pair
  auto tucker = [&](int c, int k, const void* in, void* out, const void* base, double alpha) {
    const void* cur = in;
    cudaError_t r = cudaSuccess;
    for (int mu = 0; mu < d && r == cudaSuccess; ++mu) {
      const bool last = mu == d - 1;
      void* dst = last ? out : ((mu & 1) ? G.t1[c] : G.t0[c]);
      r = mode_one<T>(P, mu, G.op[c][mu][k], G.opT[c][mu][k], cur, dst, last ? base : nullptr,
                      last ? alpha : 1.0, last ? 1.0 : 0.0);
      cur = dst;
    }
    return r;
  };
  for (int c = 0; c < m && e == cudaSuccess; ++c) e = tucker(c, 1, G.w[c], G.u2[c], U[c], tau);
  if (e != cudaSuccess) return e;
  e = timed_kernel(P, KC_RDIFF, (double)N * 16.0 * G.terms.n, (double)sizeof(T) * N * 3 * m, [&] {
    poly_kernel<T><<<gr, 256, 0, P->stream>>>(G.terms, q, N, 1);
    return cudaGetLastError();
  });
  if (e != cudaSuccess) return e;
  const double c2 = ldexp(tau, d - 1);
  for (int c = 0; c < m && e == cudaSuccess; ++c) e = tucker(c, 2, G.w[c], U[c], G.u2[c], c2);
  return e;
}

cudaError_t general_step(adr_plan P, void* const* U) {
  return P->prec == ADR_FP64 ? step_general<double>(P, U) : step_general<float>(P, U);
}

void general_free(adr_plan P) {
  delete P->gen;
  P->gen = nullptr;
}

int general_components(const adr_plan_s* P) { return P->gen ? P->gen->m : 0; }

const double* general_master(const adr_plan_s* P, int c, int mu, int which) {
  return P->gen ? P->gen->master[c][mu][which] : nullptr;
}

}  // namespace adr

using namespace adr;

static adr_status gfail(adr_status s, const std::string& msg) {
  set_error(msg);
  return s;
}

extern "C" adr_status adr_plan_create_general(const adr_general_problem* gp, void* stream,
                                              adr_plan* out) {
  if (!gp || !out) return gfail(ADR_EINVAL, "adr_plan_create_general: NULL argument");
  const int d = gp->d, m = gp->m;
  if (d != 2 && d != 3) return gfail(ADR_EINVAL, "adr_plan_create_general: d must be 2 or 3");
  if (m < 1 || m > 4) return gfail(ADR_EINVAL, "adr_plan_create_general: m must be in [1, 4]");
  if (gp->precision != ADR_FP64 && gp->precision != ADR_FP32)
    return gfail(ADR_EUNSUPPORTED, "adr_plan_create_general: ADR_FP64 or ADR_FP32 products only");
  if (!(gp->tau > 0.0) || !isfinite(gp->tau))
    return gfail(ADR_EINVAL, "adr_plan_create_general: tau must be finite and > 0");
  if (gp->nterms < 0 || gp->nterms > kMaxTerms || (gp->nterms > 0 && !gp->terms))
    return gfail(ADR_EINVAL, "adr_plan_create_general: 0 <= nterms <= 64 terms needed");
  int64_t N = 1;
  for (int mu = 0; mu < d; ++mu) {
    if (gp->n[mu] < 1 || gp->n[mu] > 4096)
      return gfail(ADR_EINVAL, "adr_plan_create_general: n[mu] must be in [1, 4096]");
    N *= gp->n[mu];
  }
  if (N > ((int64_t)1 << 31)) return gfail(ADR_EINVAL, "adr_plan_create_general: grid too large");
  PolyTerms T{};
  T.n = gp->nterms;
  T.m = m;
  for (int t = 0; t < gp->nterms; ++t) {
    const adr_term& q = gp->terms[t];
    if (q.comp < 0 || q.comp >= m || !isfinite(q.coef))
      return gfail(ADR_EINVAL, "adr_plan_create_general: term component out of range or coefficient not finite");
    T.comp[t] = q.comp;
    T.coef[t] = q.coef;
    for (int j = 0; j < 4; ++j) {
      if (q.pow[j] < 0 || q.pow[j] > 8 || (j >= m && q.pow[j] != 0))
        return gfail(ADR_EINVAL, "adr_plan_create_general: exponents must be in [0, 8] (0 beyond m)");
      T.pw[t][j] = q.pow[j];
    }
  }
  for (int c = 0; c < m; ++c)
    for (int mu = 0; mu < d; ++mu) {
      if (!gp->A[c][mu]) return gfail(ADR_EINVAL, "adr_plan_create_general: NULL matrix");
      const int64_t nn = gp->n[mu] * gp->n[mu];
      for (int64_t e = 0; e < nn; ++e)
        if (!isfinite(gp->A[c][mu][e]))
          return gfail(ADR_EINVAL, "adr_plan_create_general: matrix entries must be finite");
    }

  adr_plan P = new adr_plan_s();
  memset(&P->prob, 0, sizeof(P->prob));
  P->prob.d = d;
  P->prob.precision = gp->precision;
  P->prob.scheme = ADR_ETD2RKDS;
  P->prob.tau = gp->tau;
  P->stream = (cudaStream_t)stream;
  P->d = d;
  P->N = N;
  for (int mu = 0; mu < 3; ++mu) P->n[mu] = mu < d ? gp->n[mu] : 1;
  for (int mu = 0; mu < d; ++mu) P->prob.n[mu] = gp->n[mu];
  P->prec = gp->precision;
  P->scheme = ADR_ETD2RKDS;
  P->esize = P->prec == ADR_FP64 ? 8 : 4;
  memset(&P->pw, 0, sizeof(P->pw));
  memset(P->master, 0, sizeof(P->master));
  memset(P->op, 0, sizeof(P->op));
  memset(P->opT, 0, sizeof(P->opT));
  P->u2 = P->v2 = nullptr;
  P->bufA[0] = P->bufA[1] = P->bufB[0] = P->bufB[1] = nullptr;
  P->dstate[0] = P->dstate[1] = nullptr;
  P->ind = nullptr;
  P->launches = P->steps = 0;
  P->timing = false;
  P->capturing = false;
  memset(P->acc_ms, 0, sizeof(P->acc_ms));
  memset(P->acc_flops, 0, sizeof(P->acc_flops));
  memset(P->acc_bytes, 0, sizeof(P->acc_bytes));
  memset(P->acc_count, 0, sizeof(P->acc_count));
  P->event_next = 0;
  P->use_graphs = 0;
  P->cap_stream = nullptr;
  P->gexec = P->gexec_timed = nullptr;
  P->g_u = P->g_v = P->gt_u = P->gt_v = nullptr;
  P->g_launches = 0;
  P->tc_variant = -1;
  P->batch_refs = 0;
  P->shared_hits = 0;
  tc_init(&P->tc);
  P->gen = new GeneralState();
  GeneralState& G = *P->gen;
  memset(G.master, 0, sizeof(G.master));
  memset(G.op, 0, sizeof(G.op));
  memset(G.opT, 0, sizeof(G.opT));
  G.m = m;
  G.terms = T;
  cudaStream_t s = P->stream;
  cudaError_t e = cudaSuccess;
  auto alloc = [&](void** q, size_t bytes) -> cudaError_t {
    cudaError_t r = cudaMalloc(q, bytes < 16 ? 16 : bytes);
    if (r == cudaSuccess) P->allocs.push_back(*q);
    return r;
  };
  for (int c = 0; c < m && e == cudaSuccess; ++c)
    for (int mu = 0; mu < d && e == cudaSuccess; ++mu) {
      const int64_t n = gp->n[mu];
      const size_t nn = (size_t)n * n;
      for (int w = 0; w < 4 && e == cudaSuccess; ++w) e = alloc((void**)&G.master[c][mu][w], nn * 8);
      if (e != cudaSuccess) break;
      e = cudaMemcpyAsync(G.master[c][mu][0], gp->A[c][mu], nn * 8, cudaMemcpyHostToDevice, s);
      double norm1 = 0.0;  // ||A||_1: the largest absolute column sum
      for (int64_t j = 0; j < n; ++j) {
        double cs = 0.0;
        for (int64_t i = 0; i < n; ++i) cs += fabs(gp->A[c][mu][i * n + j]);
        norm1 = cs > norm1 ? cs : norm1;
      }
      if (e == cudaSuccess)
        e = matfun_phi_dense((int)n, G.master[c][mu][0], norm1, gp->tau, G.master[c][mu][1],
                             G.master[c][mu][2], G.master[c][mu][3], s);
      if (e == cudaSuccess && n > 0) {
        // A (for K U), phi_1 and phi_2 in the state type, row-major and transposed
        const int k2w[3] = {0, 2, 3};
        for (int k = 0; k < 3 && e == cudaSuccess; ++k) {
          e = alloc(&G.op[c][mu][k], nn * P->esize);
          if (e == cudaSuccess) e = alloc(&G.opT[c][mu][k], nn * P->esize);
          if (e == cudaSuccess)
            e = launch_convert(G.master[c][mu][k2w[k]], G.op[c][mu][k], (int64_t)nn,
                               P->prec == ADR_FP64, 0, s);
          if (e == cudaSuccess)
            e = launch_convert(G.master[c][mu][k2w[k]], G.opT[c][mu][k], (int64_t)nn,
                               P->prec == ADR_FP64, (int)n, s);
        }
      }
    }
  for (int c = 0; c < m && e == cudaSuccess; ++c) {
    const size_t sb = (size_t)N * P->esize;
    e = alloc(&G.w[c], sb);
    if (e == cudaSuccess) e = alloc(&G.u2[c], sb);
    if (e == cudaSuccess) e = alloc(&G.t0[c], sb);
    if (e == cudaSuccess) e = alloc(&G.t1[c], sb);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) {
    const bool nomem = e == cudaErrorMemoryAllocation;
    set_error(std::string("adr_plan_create_general: ") + cudaGetErrorString(e));
    adr_plan_destroy(P);
    return nomem ? ADR_ENOMEM : ADR_ECUDA;
  }
  *out = P;
  return ADR_OK;
}

extern "C" adr_status adr_step_general(adr_plan plan, void* const* states, int64_t nsteps) {
  if (!plan || !states || nsteps < 0) return gfail(ADR_EINVAL, "adr_step_general: bad argument");
  if (!plan->gen) return gfail(ADR_EINVAL, "adr_step_general: not a general plan");
  const int m = plan->gen->m;
  for (int c = 0; c < m; ++c) {
    if (!states[c]) return gfail(ADR_EINVAL, "adr_step_general: NULL state");
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, states[c]) != cudaSuccess ||
        (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)) {
      cudaGetLastError();
      return gfail(ADR_EINVAL, "adr_step_general: states must be device pointers");
    }
    for (int j = 0; j < c; ++j)
      if (states[j] == states[c]) return gfail(ADR_EINVAL, "adr_step_general: states must be distinct");
  }
  for (int64_t k = 0; k < nsteps; ++k) {
    cudaError_t e = general_step(plan, states);
    if (e != cudaSuccess)
      return gfail(ADR_ECUDA, std::string("adr_step_general: ") + cudaGetErrorString(e));
    plan->steps++;
  }
  return ADR_OK;
}

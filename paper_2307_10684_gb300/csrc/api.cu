// C ABI of the ETD2RKds library: plans, steps, solves and queries.
//
// A plan holds, for each component c in {u, v} and direction mu, the FP64
// matrices A_mu^c, e^(tau A_mu^c), phi_1(tau A_mu^c), phi_2(tau A_mu^c)
// (computed on the GPU by matfun.cu) plus their operand copies for the step
// kernels, and the step workspace.  One ETD2RKds step (Sec. 3, Eq. 11) is
//   W^c  = sum_mu U^c x_mu A_mu^c + G^c(U, V)          (rhs kernel)
//   U2^c = U^c + tau W^c x_1 phi_1 ... x_d phi_1        (d mode products)
//   D^c  = G^c(U2, V2) - G^c(U, V)                      (rdiff kernel)
//   U+^c = U2^c + 2^(d-1) tau D^c x_1 phi_2 ... x_d phi_2
// with both components handled by each launch.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "adr_internal.h"

namespace adr {

static thread_local std::string g_last_error;
void set_error(const std::string& msg) { g_last_error = msg; }

}  // namespace adr

using namespace adr;

// ---------------------------------------------------------------- helpers
static adr_status fail(adr_status s, const std::string& msg) {
  set_error(msg);
  return s;
}

static cudaError_t plan_alloc(adr_plan P, void** out, size_t bytes) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, bytes < 16 ? 16 : bytes);
  if (e != cudaSuccess) return e;
  P->allocs.push_back(q);
  *out = q;
  return cudaSuccess;
}

static adr_status validate(const adr_problem* p) {
  if (!p) return fail(ADR_EINVAL, "problem is NULL");
  if (p->d != 2 && p->d != 3) return fail(ADR_EINVAL, "d must be 2 or 3");
  if (p->scheme != ADR_ETD2RKDS && p->scheme != ADR_LAWSON2B)
    return fail(ADR_EINVAL, "unknown scheme");
  if (p->model < 0 || p->model > ADR_DIB) return fail(ADR_EINVAL, "unknown model");
  if (p->precision < 0 || p->precision > ADR_BF16X3)
    return fail(ADR_EINVAL, "unknown precision");
  if (!(p->tau > 0.0) || !isfinite(p->tau)) return fail(ADR_EINVAL, "tau must be finite and > 0");
  if (p->state < ADR_STATE_AUTO || p->state > ADR_STATE_COMPENSATED || p->reserved != 0)
    return fail(ADR_EINVAL, "unknown state mode (or reserved field not 0)");
  if (p->state == ADR_STATE_COMPENSATED &&
      ((p->precision != ADR_BF16X3 && p->precision != ADR_TF32X3) || p->scheme != ADR_ETD2RKDS))
    return fail(ADR_EUNSUPPORTED, "compensated state: tensor-core ETD2RKds plans only");
  int64_t N = 1;
  for (int m = 0; m < p->d; ++m) {
    if (p->n[m] < 3 || p->n[m] > 4096) return fail(ADR_EINVAL, "n[mu] must be in [3, 4096]");
    if (!(p->hi[m] > p->lo[m]) || !isfinite(p->hi[m]) || !isfinite(p->lo[m]))
      return fail(ADR_EINVAL, "domain needs lo < hi, finite");
    N *= p->n[m];
  }
  if (N > ((int64_t)1 << 31)) return fail(ADR_EINVAL, "grid too large (N > 2^31)");
  for (int c = 0; c < 2; ++c) {
    if (!(p->diff[c] > 0.0) || !isfinite(p->diff[c]))
      return fail(ADR_EINVAL, "diffusion must be finite and > 0");
    for (int m = 0; m < p->d; ++m)
      if (!isfinite(p->adv[c][m])) return fail(ADR_EINVAL, "advection must be finite");
  }
  for (int i = 0; i < 16; ++i)
    if (!isfinite(p->params[i])) return fail(ADR_EINVAL, "params must be finite");
  return ADR_OK;
}

// Centred second-order FD coefficients of delta d2/dx2 - alpha d/dx on the
// vertex grid with mirrored ghost values at both ends (Sec. 4 text).
static Tridiag fd_coefficients(int64_t n, double lo, double hi, double delta, double alpha) {
  const double h = (hi - lo) / (double)(n - 1);
  Tridiag t;
  t.lo = delta / (h * h) + alpha / (2.0 * h);
  t.di = -2.0 * delta / (h * h);
  t.up = delta / (h * h) - alpha / (2.0 * h);
  t.b0 = 2.0 * delta / (h * h);
  t.bn = 2.0 * delta / (h * h);
  return t;
}

// How a (validated) problem carries its state: 0 = plain FP32, 2 = hi + lo
// FP32 words carried across calls, with the reactions in double-float.
static int compensated(const adr_problem* p) {
  const bool tc = p->precision == ADR_BF16X3 || p->precision == ADR_TF32X3;
  return (tc && p->scheme == ADR_ETD2RKDS && p->state == ADR_STATE_COMPENSATED) ? 2 : 0;
}

static bool same_operator(const Tridiag& a, const Tridiag& b) {
  return a.lo == b.lo && a.di == b.di && a.up == b.up && a.b0 == b.b0 && a.bn == b.bn;
}

// ---------------------------------------------------------------- step (SIMT)
template <typename T>
static cudaError_t mode_product_simt(adr_plan P, int mu, int ell, void* const in[2], void* const out[2],
                                     void* const base[2], double alpha) {
  const int64_t n = P->n[mu];
  int64_t Q = 1;
  for (int m = 0; m < mu; ++m) Q *= P->n[m];
  const int64_t Pb = P->N / (n * Q);
  GemmArgs g{};
  g.ncomp = 2;
  g.alpha = alpha;
  g.beta = 1.0;
  for (int c = 0; c < 2; ++c) {
    g.C[c] = out[c];
    g.base[c] = base ? base[c] : nullptr;
    g.base2[c] = nullptr;
  }
  if (mu == 0) {  // Y[p][i] = sum_j X[p][j] Phi[i][j]  ->  Y = X Phi^T
    for (int c = 0; c < 2; ++c) {
      g.A[c] = in[c];
      g.B[c] = P->opT[c][mu][ell];
    }
    g.M = (int)Pb;
    g.N = (int)n;
    g.K = (int)n;
    g.lda = n;
    g.ldb = n;
    g.ldc = n;
    g.batch = 1;
  } else {  // Y[p] = Phi X[p], X[p] an n x Q row-major slab
    for (int c = 0; c < 2; ++c) {
      g.A[c] = P->op[c][mu][ell];
      g.B[c] = in[c];
    }
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
  const double flops = 2.0 * 2.0 * (double)n * (double)P->N;
  const double bytes = (double)sizeof(T) * 2.0 * (2.0 * P->N + (base ? P->N : 0) + n * n);
  return timed_kernel(P, KC_MODE_SIMT, flops, bytes,
                      [&] { return launch_gemm_simt<T>(g, P->stream); });
}

template <typename T>
static cudaError_t tucker_simt(adr_plan P, int ell, void* const in[2], void* const out[2],
                               void* const base[2], double alpha) {
  // in -> bufB -> bufA -> ... -> out, last product with the AXPY epilogue
  void* cur[2] = {in[0], in[1]};
  for (int mu = 0; mu < P->d; ++mu) {
    const bool last = (mu == P->d - 1);
    void* dst[2];
    if (last) {
      dst[0] = out[0];
      dst[1] = out[1];
    } else {
      void* const* pick = (cur[0] == P->bufA[0]) ? P->bufB : P->bufA;
      dst[0] = pick[0];
      dst[1] = pick[1];
    }
    cudaError_t e = mode_product_simt<T>(P, mu, ell, cur, dst, last ? base : nullptr,
                                         last ? alpha : 1.0);
    if (e != cudaSuccess) return e;
    cur[0] = dst[0];
    cur[1] = dst[1];
  }
  return cudaSuccess;
}

template <typename T>
static const PointwiseArgsT<T>& pw_for(adr_plan P);
template <>
const PointwiseArgsT<double>& pw_for<double>(adr_plan P) {
  return P->pw;
}
template <>
const PointwiseArgsT<float>& pw_for<float>(adr_plan P) {
  return P->pwf;
}

template <typename T>
static cudaError_t step_simt(adr_plan P, T* u, T* v) {
  const double tau = P->prob.tau;
  const double N = (double)P->N;
  cudaError_t e = timed_kernel(P, KC_RHS, N * 2.0 * (6.0 * P->d + 10.0), sizeof(T) * N * 4.0, [&] {
    return launch_rhs<T>(pw_for<T>(P), u, v, (T*)P->bufA[0], (T*)P->bufA[1], P->stream);
  });
  if (e != cudaSuccess) return e;
  void* uv[2] = {u, v};
  void* st2[2] = {P->u2, P->v2};
  e = tucker_simt<T>(P, 1, P->bufA, st2, uv, tau);
  if (e != cudaSuccess) return e;
  e = timed_kernel(P, KC_RDIFF, N * 2.0 * 12.0, sizeof(T) * N * 6.0, [&] {
    return launch_rdiff<T>(pw_for<T>(P), u, v, (const T*)P->u2, (const T*)P->v2, (T*)P->bufA[0],
                           (T*)P->bufA[1], P->stream);
  });
  if (e != cudaSuccess) return e;
  const double c2 = ldexp(tau, P->d - 1);
  return tucker_simt<T>(P, 2, P->bufA, uv, st2, c2);
}

// Lawson2b, Eq. 7:  U2 = (U + tau G(U,V)) x_mu e^(tau A_mu),
//                   U+ = (U + tau/2 G(U,V)) x_mu e^(tau A_mu) + tau/2 G(U2, V2).
template <typename T>
static cudaError_t step_lawson_simt(adr_plan P, T* u, T* v) {
  const T tau = (T)P->prob.tau;
  const double N = (double)P->N;
  void* uv[2] = {u, v};
  void* st2[2] = {P->u2, P->v2};
  auto pre = [&](T scale) {
    return timed_kernel(P, KC_LAWSON_PW, N * 2.0 * 12.0, sizeof(T) * N * 4.0, [&] {
      return launch_lawson_pre<T>(pw_for<T>(P), u, v, scale, (T*)P->bufA[0], (T*)P->bufA[1],
                                  P->stream);
    });
  };
  cudaError_t e = pre(tau);
  if (e != cudaSuccess) return e;
  e = tucker_simt<T>(P, 0, P->bufA, st2, nullptr, 1.0);
  if (e != cudaSuccess) return e;
  e = pre(tau / (T)2);
  if (e != cudaSuccess) return e;
  e = tucker_simt<T>(P, 0, P->bufA, uv, nullptr, 1.0);
  if (e != cudaSuccess) return e;
  return timed_kernel(P, KC_LAWSON_PW, N * 2.0 * 12.0, sizeof(T) * N * 6.0, [&] {
    return launch_lawson_post<T>(pw_for<T>(P), (const T*)P->u2, (const T*)P->v2, tau / (T)2, u,
                                 v, P->stream);
  });
}

// ---------------------------------------------------------------- plan
static void plan_free(adr_plan P) {
  if (!P) return;
  if (P->stream) cudaStreamSynchronize(P->stream);
  for (void* q : P->allocs) cudaFree(q);
  // the operand pieces first: they are keyed by the FP64 matrices' addresses
  tc_free(&P->tc);
  for (void* q : P->shared) shared_release(q);
  general_free(P);
  for (cudaEvent_t e : P->event_pool) cudaEventDestroy(e);
  if (P->gexec) cudaGraphExecDestroy(P->gexec);
  if (P->gexec_timed) cudaGraphExecDestroy(P->gexec_timed);
  if (P->cap_stream) cudaStreamDestroy(P->cap_stream);
  delete P;
}

extern "C" adr_status adr_plan_create(const adr_problem* problem, void* stream, adr_plan* out) {
  return adr_plan_create_tuned(problem, nullptr, stream, out);
}

extern "C" adr_status adr_plan_create_tuned(const adr_problem* problem, const adr_tuning* tuning,
                                            void* stream, adr_plan* out) {
  if (!out) return fail(ADR_EINVAL, "out is NULL");
  if (tuning && (tuning->kernel < -1 || tuning->kernel > 4))
    return fail(ADR_EINVAL, "adr_tuning.kernel must be -1 or 0..4");
  adr_status st = validate(problem);
  if (st != ADR_OK) return st;
  adr_plan P = new adr_plan_s();
  P->gen = nullptr;
  memset(&P->pw, 0, sizeof(P->pw));
  memset(P->master, 0, sizeof(P->master));
  memset(P->op, 0, sizeof(P->op));
  memset(P->opT, 0, sizeof(P->opT));
  P->prob = *problem;
  P->stream = (cudaStream_t)stream;
  P->d = problem->d;
  P->N = 1;
  for (int m = 0; m < 3; ++m) P->n[m] = m < P->d ? problem->n[m] : 1;
  for (int m = 0; m < P->d; ++m) P->N *= P->n[m];
  P->prec = problem->precision;
  P->scheme = problem->scheme;
  P->esize = P->prec == ADR_FP64 ? sizeof(double) : sizeof(float);
  P->launches = 0;
  P->steps = 0;
  P->timing = false;
  P->event_next = 0;
  P->u2 = P->v2 = nullptr;
  P->dstate[0] = P->dstate[1] = nullptr;
  P->gexec = nullptr;
  P->g_u = P->g_v = nullptr;
  P->gexec_timed = nullptr;
  P->gt_u = P->gt_v = nullptr;
  P->capturing = false;
  memset(P->acc_ms, 0, sizeof(P->acc_ms));
  memset(P->acc_flops, 0, sizeof(P->acc_flops));
  memset(P->acc_bytes, 0, sizeof(P->acc_bytes));
  memset(P->acc_count, 0, sizeof(P->acc_count));
  P->g_launches = 0;
  P->tc_variant = tuning ? tuning->kernel : -1;
  P->cap_stream = nullptr;
  P->shared_hits = 0;
  P->use_graphs = 1;
  if (const char* ev = getenv("ADR_GRAPHS")) P->use_graphs = atoi(ev) != 0;
  tc_init(&P->tc);

  PointwiseArgs& pw = P->pw;
  pw.d = P->d;
  pw.N = P->N;
  for (int m = 0; m < 3; ++m) pw.n[m] = P->n[m];
  pw.rx.model = problem->model;
  for (int i = 0; i < 16; ++i) pw.rx.p[i] = problem->params[i];
  for (int c = 0; c < 2; ++c)
    for (int m = 0; m < P->d; ++m)
      pw.A[c][m] = fd_coefficients(P->n[m], problem->lo[m], problem->hi[m], problem->diff[c],
                                   problem->adv[c][m]);

  P->pwf = cast_args<float>(pw);
  cudaError_t e = cudaSuccess;
#define PLAN_TRY(x)                                                            \
  do {                                                                         \
    e = (x);                                                                   \
    if (e != cudaSuccess) {                                                    \
      set_error(std::string("adr_plan_create: ") + #x + ": " + cudaGetErrorString(e)); \
      plan_free(P);                                                            \
      return e == cudaErrorMemoryAllocation ? ADR_ENOMEM : ADR_ECUDA;          \
    }                                                                          \
  } while (0)

  // matrices, shared between (c, mu) pairs with identical operators
  for (int c = 0; c < 2; ++c) {
    for (int m = 0; m < P->d; ++m) {
      const int64_t n = P->n[m];
      bool found = false;
      for (int c2 = 0; c2 <= c && !found; ++c2)
        for (int m2 = 0; m2 < P->d && !found; ++m2) {
          if (c2 == c && m2 >= m) break;
          if (P->n[m2] == n && same_operator(pw.A[c2][m2], pw.A[c][m])) {
            for (int w = 0; w < 4; ++w) P->master[c][m][w] = P->master[c2][m2][w];
            for (int l = 0; l < 3; ++l) {
              P->op[c][m][l] = P->op[c2][m2][l];
              P->opT[c][m][l] = P->opT[c2][m2][l];
            }
            found = true;
          }
        }
      if (found) continue;
      const size_t nn = (size_t)n * n;
      // A, e^(tau A), phi_1, phi_2 of this operator and step: from the
      // process-wide cache, computed here on a miss
      const Tridiag& op = pw.A[c][m];
      const std::vector<uint64_t> key = {0, (uint64_t)n, key_bits(op.lo), key_bits(op.di),
                                         key_bits(op.up), key_bits(op.b0), key_bits(op.bn),
                                         key_bits(problem->tau)};
      void* mats[4] = {};
      bool hit = false;
      PLAN_TRY(shared_acquire(key, 4, nn * 8, [&](void* const* b) {
        cudaError_t r = launch_build_dense((int)n, op, 1.0, (double*)b[0], P->stream);
        if (r == cudaSuccess)
          r = matfun_phi((int)n, op, problem->tau, (double*)b[1], (double*)b[2], (double*)b[3],
                         P->stream);
        return r;
      }, P->stream, mats, &hit));
      P->shared.push_back(mats[0]);
      P->shared_hits += hit ? 1 : 0;
      for (int w = 0; w < 4; ++w) P->master[c][m][w] = (double*)mats[w];
      // SIMT operands (FP32/FP64 plans): e^(tau A), phi_1, phi_2 and transposes
      for (int l = 0; l < 3 && P->prec <= ADR_FP32; ++l) {
        PLAN_TRY(plan_alloc(P, &P->op[c][m][l], nn * P->esize));
        PLAN_TRY(plan_alloc(P, &P->opT[c][m][l], nn * P->esize));
        PLAN_TRY(launch_convert(P->master[c][m][1 + l], P->op[c][m][l], (int64_t)nn,
                                P->prec == ADR_FP64, 0, P->stream));
        PLAN_TRY(launch_convert(P->master[c][m][1 + l], P->opT[c][m][l], (int64_t)nn,
                                P->prec == ADR_FP64, (int)n, P->stream));
      }
    }
  }
  const size_t sb = (size_t)P->N * P->esize;
  PLAN_TRY(plan_alloc(P, &P->u2, sb));
  PLAN_TRY(plan_alloc(P, &P->v2, sb));
  for (int c = 0; c < 2; ++c) {
    PLAN_TRY(plan_alloc(P, &P->bufA[c], sb));
    PLAN_TRY(plan_alloc(P, &P->bufB[c], sb));
  }
  if (P->prec == ADR_TF32X3 || P->prec == ADR_BF16X3) {
    e = tc_prepare(&P->tc, P->prec, P->scheme, P->d, P->n, P->master, P->stream, P->tc_variant,
                   compensated(problem));
    if (e != cudaSuccess) {
      const bool unsup = (e == cudaErrorNotSupported);
      set_error(std::string("adr_plan_create: tensor-core operands: ") + cudaGetErrorString(e));
      plan_free(P);
      return unsup ? ADR_EUNSUPPORTED : ADR_ECUDA;
    }
  }
  PLAN_TRY(plan_alloc(P, (void**)&P->ind, 4 * sizeof(double)));
  PLAN_TRY(cudaStreamCreateWithFlags(&P->cap_stream, cudaStreamNonBlocking));
  PLAN_TRY(cudaStreamSynchronize(P->stream));
  PLAN_TRY(cudaGetLastError());
#undef PLAN_TRY
  *out = P;
  return ADR_OK;
}

extern "C" adr_status adr_plan_set_stream(adr_plan plan, void* stream) {
  if (!plan) return fail(ADR_EINVAL, "plan is NULL");
  ADR_CUDA_TRY(cudaStreamSynchronize(plan->stream));
  plan->stream = (cudaStream_t)stream;
  return ADR_OK;
}

extern "C" adr_status adr_plan_destroy(adr_plan plan) {
  if (plan && __atomic_load_n(&plan->batch_refs, __ATOMIC_ACQUIRE) > 0)
    return fail(ADR_EBUSY, "adr_plan_destroy: a live batch uses this plan; destroy the batch first");
  plan_free(plan);
  return ADR_OK;
}

static bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

static cudaError_t step_direct(adr_plan P, void* u, void* v, int64_t nsteps) {
  for (int64_t s = 0; s < nsteps; ++s) {
    cudaError_t e;
    const bool lawson = P->scheme == ADR_LAWSON2B;
    if (P->prec == ADR_FP64)
      e = lawson ? step_lawson_simt<double>(P, (double*)u, (double*)v)
                 : step_simt<double>(P, (double*)u, (double*)v);
    else if (P->prec == ADR_FP32)
      e = lawson ? step_lawson_simt<float>(P, (float*)u, (float*)v)
                 : step_simt<float>(P, (float*)u, (float*)v);
    else
      e = tc_step(&P->tc, P, u, v);
    if (e != cudaSuccess) return e;
    P->steps++;
  }
  return cudaSuccess;
}

// Steps per captured graph.  A step is 5-8 launches, so a chunk replays a few
// hundred kernels per cudaGraphLaunch.
static constexpr int64_t kGraphChunk = 32;

// Capture kGraphChunk steps on (u, v) into P->gexec (P->gexec_timed when
// timing: the capture then also records the event-record nodes around every
// kernel).  On any failure graphs are switched off for this plan and the
// caller launches directly.
static void build_graph(adr_plan P, void* u, void* v) {
  const bool timed = P->timing;
  cudaGraphExec_t& ge = timed ? P->gexec_timed : P->gexec;
  if (ge) {
    cudaGraphExecDestroy(ge);
    ge = nullptr;
  }
  const int64_t l0 = P->launches, s0 = P->steps;
  cudaStream_t saved = P->stream;
  P->stream = P->cap_stream;
  if (timed) P->graph_timed.clear();
  P->capturing = true;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(P->cap_stream, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaError_t e1 = step_direct(P, u, v, kGraphChunk);
    cudaError_t e2 = cudaStreamEndCapture(P->cap_stream, &g);
    e = e1 != cudaSuccess ? e1 : e2;
  }
  P->capturing = false;
  P->stream = saved;
  P->g_launches = P->launches - l0;
  P->launches = l0;
  P->steps = s0;
  if (e == cudaSuccess && g) e = cudaGraphInstantiate(&ge, g, 0);
  if (g) cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    cudaGetLastError();
    ge = nullptr;
    P->use_graphs = 0;
    return;
  }
  if (timed) {
    P->gt_u = u;
    P->gt_v = v;
  } else {
    P->g_u = u;
    P->g_v = v;
  }
}

static adr_status step_impl(adr_plan P, void* u, void* v, int64_t nsteps) {
  int64_t done = 0;
  if (P->gen) return fail(ADR_EINVAL, "a general plan steps with adr_step_general");
  if (nsteps == 0) return ADR_OK;
  if (P->prec == ADR_TF32X3 || P->prec == ADR_BF16X3) {
    if ((((uintptr_t)u) | ((uintptr_t)v)) & 15)
      return fail(ADR_EINVAL, "adr_step: BF16X3 state buffers must be 16-byte aligned");
    cudaError_t e = tc_bind(&P->tc, P, u, v);
    if (e != cudaSuccess)
      return fail(ADR_ECUDA, std::string("adr_step: binding state buffers: ") + cudaGetErrorString(e));
  }
  if (P->use_graphs && nsteps >= kGraphChunk) {
    const bool timed = P->timing;
    if (timed ? (!P->gexec_timed || P->gt_u != u || P->gt_v != v)
              : (!P->gexec || P->g_u != u || P->g_v != v))
      build_graph(P, u, v);
    cudaGraphExec_t ge = timed ? P->gexec_timed : P->gexec;
    if (ge) {
      for (; done + kGraphChunk <= nsteps; done += kGraphChunk) {
        cudaError_t e = cudaGraphLaunch(ge, P->stream);
        if (e != cudaSuccess)
          return fail(ADR_ECUDA, std::string("adr_step: cudaGraphLaunch: ") + cudaGetErrorString(e));
        P->launches += P->g_launches;
        P->steps += kGraphChunk;
        if (timed) {  // the replay's events are re-recorded by the next replay
          e = cudaStreamSynchronize(P->stream);
          if (e != cudaSuccess)
            return fail(ADR_ECUDA, std::string("adr_step: ") + cudaGetErrorString(e));
          harvest_timing(P, P->graph_timed);
        }
      }
    }
  }
  cudaError_t e = step_direct(P, u, v, nsteps - done);
  if (e != cudaSuccess)
    return fail(e == cudaErrorNotSupported ? ADR_EUNSUPPORTED : ADR_ECUDA,
                std::string("adr_step: ") + cudaGetErrorString(e));
  return ADR_OK;
}

adr_status plan_step_continue(adr_plan plan, void* u, void* v, int64_t nsteps) {
  if (!plan) return fail(ADR_EINVAL, "plan is NULL");
  if (!u || !v || u == v) return fail(ADR_EINVAL, "u, v must be distinct non-NULL device pointers");
  if (nsteps < 0) return fail(ADR_EINVAL, "nsteps < 0");
  if (!is_device_ptr(u) || !is_device_ptr(v))
    return fail(ADR_EINVAL, "adr_step needs device pointers");
  return step_impl(plan, u, v, nsteps);
}

extern "C" adr_status adr_step(adr_plan plan, void* u, void* v, int64_t nsteps) {
  if (plan && u && v && u != v && nsteps > 0) {  // the start of a call (compensated state)
    cudaError_t e = tc_begin_call(&plan->tc, u, v, plan->stream);
    if (e != cudaSuccess) return fail(ADR_ECUDA, std::string("adr_step: ") + cudaGetErrorString(e));
  }
  return plan_step_continue(plan, u, v, nsteps);
}

extern "C" adr_status adr_plan_time_mode_products(adr_plan plan, void* u, void* v, int32_t reps,
                                                  double* ms_per_launch, int32_t* launches_per_step) {
  if (!plan || !u || !v || u == v || !ms_per_launch || !launches_per_step)
    return fail(ADR_EINVAL, "adr_plan_time_mode_products: bad argument");
  if (reps < 1 || reps > 4096) return fail(ADR_EINVAL, "adr_plan_time_mode_products: reps in [1, 4096]");
  if (plan->prec != ADR_BF16X3 && plan->prec != ADR_TF32X3)
    return fail(ADR_EUNSUPPORTED, "adr_plan_time_mode_products: tensor-core plans only");
  if (!is_device_ptr(u) || !is_device_ptr(v) || ((((uintptr_t)u) | ((uintptr_t)v)) & 15))
    return fail(ADR_EINVAL, "adr_plan_time_mode_products: 16-byte aligned device buffers needed");
  float ms = 0.f;
  int passes = 0;
  cudaError_t e = tc_time_passes(&plan->tc, plan, u, v, reps, &ms, &passes);
  if (e != cudaSuccess)
    return fail(ADR_ECUDA, std::string("adr_plan_time_mode_products: ") + cudaGetErrorString(e));
  *ms_per_launch = ms;
  *launches_per_step = passes;
  return ADR_OK;
}

extern "C" adr_status adr_plan_mode_product_macs(adr_plan plan, double* dense, double* computed) {
  if (!plan || !dense || !computed) return fail(ADR_EINVAL, "adr_plan_mode_product_macs: bad argument");
  if (!plan->gen && (plan->prec == ADR_BF16X3 || plan->prec == ADR_TF32X3)) {
    tc_mode_macs(&plan->tc, dense, computed);
    return ADR_OK;
  }
  // FP32 / FP64 products and general plans: two Tucker operators per
  // component and step, each a full contraction along every direction
  const int m = plan->gen ? general_components(plan) : 2;
  double sum_n = 0.0;
  for (int mu = 0; mu < plan->d; ++mu) sum_n += (double)plan->n[mu];
  *dense = *computed = 2.0 * m * (double)plan->N * sum_n;
  return ADR_OK;
}

static bool tc_etd2rkds(adr_plan P) {
  return (P->prec == ADR_BF16X3 || P->prec == ADR_TF32X3) && P->scheme == ADR_ETD2RKDS;
}

static void drop_graphs(adr_plan P) {
  if (P->gexec) cudaGraphExecDestroy(P->gexec);
  if (P->gexec_timed) cudaGraphExecDestroy(P->gexec_timed);
  P->gexec = P->gexec_timed = nullptr;
  P->g_u = P->g_v = P->gt_u = P->gt_v = nullptr;
}

extern "C" adr_status adr_plan_set_indicators(adr_plan plan, int enable) {
  if (!plan) return fail(ADR_EINVAL, "plan is NULL");
  if (!tc_etd2rkds(plan))
    return fail(ADR_EUNSUPPORTED, "fused indicators: tensor-core ETD2RKds plans only");
  if (__atomic_load_n(&plan->batch_refs, __ATOMIC_ACQUIRE) > 0)
    return fail(ADR_EBUSY, "adr_plan_set_indicators: a live batch uses this plan");
  ADR_CUDA_TRY(cudaStreamSynchronize(plan->stream));
  drop_graphs(plan);  // the captured launches carry the old descriptors
  ADR_CUDA_TRY(tc_set_indicators(&plan->tc, enable != 0, plan->stream));
  return ADR_OK;
}

extern "C" adr_status adr_plan_indicator_log(adr_plan plan, double* out, int64_t max_steps,
                                             int64_t* count) {
  if (!plan || !out || !count || max_steps < 0) return fail(ADR_EINVAL, "bad argument");
  if (!tc_etd2rkds(plan)) return fail(ADR_EUNSUPPORTED, "fused indicators: tensor-core ETD2RKds plans only");
  cudaError_t e = tc_indicator_log(&plan->tc, plan->stream, out, max_steps, count);
  if (e == cudaErrorNotSupported) return fail(ADR_EINVAL, "indicators are off (adr_plan_set_indicators)");
  if (e != cudaSuccess) return fail(ADR_ECUDA, std::string("adr_plan_indicator_log: ") + cudaGetErrorString(e));
  return ADR_OK;
}

extern "C" adr_status adr_run(adr_plan plan, void* u, void* v, double t_end, double tol,
                              int64_t check_every, int64_t* steps_done, double ind_last[4]) {
  if (!plan || !u || !v || u == v || !steps_done || !ind_last || check_every < 1 ||
      !(t_end >= 0.0) || !isfinite(t_end) || !(tol >= 0.0))
    return fail(ADR_EINVAL, "adr_run: bad argument");
  if (!tc_etd2rkds(plan)) return fail(ADR_EUNSUPPORTED, "adr_run: tensor-core ETD2RKds plans only");
  *steps_done = 0;
  const double tau = plan->prob.tau;
  const int64_t total = (int64_t)ceil(t_end / tau - 1e-9);  // steps to reach t_end
  if (total > 0) {
    cudaError_t e = tc_begin_call(&plan->tc, u, v, plan->stream);
    if (e != cudaSuccess) return fail(ADR_ECUDA, std::string("adr_run: ") + cudaGetErrorString(e));
  }
  for (int m = 0; m < 4; ++m) ind_last[m] = 0.0;
  while (*steps_done < total) {
    const int64_t n = std::min<int64_t>(check_every, total - *steps_done);
    adr_status st = plan_step_continue(plan, u, v, n);
    if (st != ADR_OK) return st;
    *steps_done += n;
    int64_t got = 0;
    cudaError_t e = tc_indicator_log(&plan->tc, plan->stream, ind_last, 1, &got);
    if (e == cudaErrorNotSupported) return fail(ADR_EINVAL, "adr_run: indicators are off (adr_plan_set_indicators)");
    if (e != cudaSuccess) return fail(ADR_ECUDA, std::string("adr_run: ") + cudaGetErrorString(e));
    if (int* ew = tc_error_word(&plan->tc)) {
      int h = 0;
      ADR_CUDA_TRY(cudaMemcpy(&h, ew, sizeof(int), cudaMemcpyDeviceToHost));
      if (h != 0) return fail(ADR_ETIMEOUT, "adr_run: a kernel gave up a bounded wait");
    }
    if (tol > 0.0 && std::max(ind_last[2], ind_last[3]) <= tol) break;
  }
  return ADR_OK;
}

extern "C" adr_status adr_plan_reset_state(adr_plan plan) {
  if (!plan) return fail(ADR_EINVAL, "plan is NULL");
  ADR_CUDA_TRY(tc_reset_state(&plan->tc, plan->stream));
  return ADR_OK;
}

extern "C" adr_status adr_solve(adr_plan plan, const void* u0, const void* v0, void* uT, void* vT,
                                int64_t nsteps) {
  if (!plan) return fail(ADR_EINVAL, "plan is NULL");
  if (plan->gen) return fail(ADR_EINVAL, "a general plan steps with adr_step_general");
  if (!u0 || !v0 || !uT || !vT) return fail(ADR_EINVAL, "NULL state pointer");
  if (uT == vT) return fail(ADR_EINVAL, "uT and vT must differ");
  if (nsteps < 0) return fail(ADR_EINVAL, "nsteps < 0");
  adr_plan P = plan;
  const size_t sb = (size_t)P->N * P->esize;
  const bool dev_in = is_device_ptr(u0) && is_device_ptr(v0);
  const bool dev_out = is_device_ptr(uT) && is_device_ptr(vT);
  void* wu;
  void* wv;
  if (dev_out) {
    wu = uT;
    wv = vT;
  } else {
    if (!P->dstate[0]) {
      if (plan_alloc(P, &P->dstate[0], sb) != cudaSuccess ||
          plan_alloc(P, &P->dstate[1], sb) != cudaSuccess)
        return fail(ADR_ENOMEM, "adr_solve: device state allocation failed");
    }
    wu = P->dstate[0];
    wv = P->dstate[1];
  }
  // a solve starts from (u0, v0) alone
  ADR_CUDA_TRY(tc_reset_state(&P->tc, P->stream));
  const cudaMemcpyKind kin = dev_in ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if (wu != u0) ADR_CUDA_TRY(cudaMemcpyAsync(wu, u0, sb, kin, P->stream));
  if (wv != v0) ADR_CUDA_TRY(cudaMemcpyAsync(wv, v0, sb, kin, P->stream));
  adr_status st = step_impl(P, wu, wv, nsteps);
  if (st != ADR_OK) return st;
  if (!dev_out) {
    ADR_CUDA_TRY(cudaMemcpyAsync(uT, wu, sb, cudaMemcpyDeviceToHost, P->stream));
    ADR_CUDA_TRY(cudaMemcpyAsync(vT, wv, sb, cudaMemcpyDeviceToHost, P->stream));
  }
  if (!dev_out || !dev_in) {
    ADR_CUDA_TRY(cudaStreamSynchronize(P->stream));
    if (int* ew = tc_error_word(&P->tc)) {
      int h = 0;
      ADR_CUDA_TRY(cudaMemcpy(&h, ew, sizeof(int), cudaMemcpyDeviceToHost));
      if (h != 0) return fail(ADR_ETIMEOUT, "adr_solve: a kernel gave up a bounded wait");
    }
  }
  return ADR_OK;
}

extern "C" adr_status adr_plan_bytes(const adr_problem* problem, size_t* state_bytes,
                                     size_t* cache_bytes) {
  adr_status st = validate(problem);
  if (st != ADR_OK) return st;
  const size_t es = problem->precision == ADR_FP64 ? 8 : 4;
  size_t N = 1, mats = 0;
  for (int m = 0; m < problem->d; ++m) {
    N *= (size_t)problem->n[m];
    const size_t nn = (size_t)problem->n[m] * problem->n[m];
    mats += 2 * (4 * 8 * nn + 4 * es * nn);
    if (problem->precision >= ADR_TF32X3) mats += 2 * 2 * 3 * 4 * nn;
  }
  if (state_bytes) *state_bytes = 2 * N * es;
  if (cache_bytes) *cache_bytes = mats + 6 * N * es + (compensated(problem) ? 2 * N * 4 : 0);
  return ADR_OK;
}

extern "C" adr_status adr_plan_matrix(adr_plan plan, int which, int component, int mu, double* out) {
  if (!plan || !out) return fail(ADR_EINVAL, "NULL argument");
  const int ncomp = plan->gen ? general_components(plan) : 2;
  if (which < 0 || which > 3 || component < 0 || component >= ncomp || mu < 0 || mu >= plan->d)
    return fail(ADR_EINVAL, "matrix index out of range");
  const int64_t n = plan->n[mu];
  const double* src = plan->gen ? general_master(plan, component, mu, which)
                                 : plan->master[component][mu][which];
  ADR_CUDA_TRY(cudaMemcpyAsync(out, src, (size_t)n * n * 8, cudaMemcpyDeviceToHost, plan->stream));
  ADR_CUDA_TRY(cudaStreamSynchronize(plan->stream));
  return ADR_OK;
}

extern "C" adr_status adr_plan_set_timing(adr_plan plan, int enable) {
  if (!plan) return fail(ADR_EINVAL, "plan is NULL");
  ADR_CUDA_TRY(cudaStreamSynchronize(plan->stream));
  plan->timing = enable != 0;
  if (int* ew = tc_error_word(&plan->tc)) ADR_CUDA_TRY(cudaMemset(ew, 0, sizeof(int)));
  plan->timed.clear();
  plan->graph_timed.clear();
  if (plan->gexec_timed) {  // holds pool events that are handed out again
    cudaGraphExecDestroy(plan->gexec_timed);
    plan->gexec_timed = nullptr;
  }
  plan->gt_u = plan->gt_v = nullptr;
  memset(plan->acc_ms, 0, sizeof(plan->acc_ms));
  memset(plan->acc_flops, 0, sizeof(plan->acc_flops));
  memset(plan->acc_bytes, 0, sizeof(plan->acc_bytes));
  memset(plan->acc_count, 0, sizeof(plan->acc_count));
  plan->event_next = 0;
  plan->launches = 0;
  plan->steps = 0;
  return ADR_OK;
}

extern "C" adr_status adr_plan_stats(adr_plan plan, adr_stats* out) {
  if (!plan || !out) return fail(ADR_EINVAL, "NULL argument");
  memset(out, 0, sizeof(*out));
  out->launches = plan->launches;
  out->steps = plan->steps;
  out->timing = plan->timing ? 1 : 0;
  out->nkernels = KC_COUNT;
  out->shared_matrices = plan->shared_hits;
  ADR_CUDA_TRY(cudaStreamSynchronize(plan->stream));
  if (int* ew = tc_error_word(&plan->tc)) {
    int h = 0;
    ADR_CUDA_TRY(cudaMemcpy(&h, ew, sizeof(int), cudaMemcpyDeviceToHost));
    out->device_error = h;
  }
  for (int k = 0; k < KC_COUNT; ++k) snprintf(out->name[k], 32, "%s", kClassNames[k]);
  if (plan->timing) {
    ADR_CUDA_TRY(cudaStreamSynchronize(plan->stream));
    harvest_timing(plan, plan->timed);  // direct launches since the last call
    plan->timed.clear();
    for (int k = 0; k < KC_COUNT; ++k) {
      out->count[k] = plan->acc_count[k];
      out->ms[k] = plan->acc_ms[k];
      out->flops[k] = plan->acc_flops[k];
      out->bytes[k] = plan->acc_bytes[k];
    }
  }
  return ADR_OK;
}

extern "C" adr_status adr_indicators(adr_plan plan, const void* u_prev, const void* v_prev,
                                     const void* u, const void* v, double out[4]) {
  if (!plan || !u_prev || !v_prev || !u || !v || !out) return fail(ADR_EINVAL, "NULL argument");
  if (!is_device_ptr(u_prev) || !is_device_ptr(v_prev) || !is_device_ptr(u) || !is_device_ptr(v))
    return fail(ADR_EINVAL, "adr_indicators needs device pointers");
  adr_plan P = plan;
  double h[4];
  ADR_CUDA_TRY(cudaMemsetAsync(P->ind, 0, 4 * sizeof(double), P->stream));
  ADR_CUDA_TRY(launch_indicators(P->pw, u_prev, v_prev, u, v, P->prec == ADR_FP64, P->ind,
                                 P->stream));
  ADR_CUDA_TRY(cudaMemcpyAsync(h, P->ind, sizeof(h), cudaMemcpyDeviceToHost, P->stream));
  ADR_CUDA_TRY(cudaStreamSynchronize(P->stream));
  double wsum = 1.0;
  for (int m = 0; m < P->d; ++m) wsum *= (double)(P->n[m] - 1);
  out[0] = h[0] / wsum;
  out[1] = h[1] / wsum;
  out[2] = sqrt(h[2]);
  out[3] = sqrt(h[3]);
  return ADR_OK;
}

extern "C" adr_status adr_max_abs_diff(void* stream, const void* x, int x_is_double,
                                       const double* ref, int64_t count, double out[2]) {
  if (!x || !ref || !out || count < 0) return fail(ADR_EINVAL, "bad argument");
  cudaStream_t s = (cudaStream_t)stream;
  unsigned long long* d = nullptr;
  ADR_CUDA_TRY(cudaMalloc(&d, 2 * sizeof(unsigned long long)));
  unsigned long long h[2] = {0, 0};
  cudaError_t e = cudaMemsetAsync(d, 0, sizeof(h), s);
  if (e == cudaSuccess && count > 0) e = launch_max_abs_diff(x, x_is_double, ref, count, d, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, d, sizeof(h), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(d);
  if (e != cudaSuccess) return fail(ADR_ECUDA, std::string("adr_max_abs_diff: ") + cudaGetErrorString(e));
  memcpy(&out[0], &h[0], 8);
  memcpy(&out[1], &h[1], 8);
  return ADR_OK;
}

extern "C" const char* adr_status_str(adr_status s) {
  switch (s) {
    case ADR_OK: return "ADR_OK";
    case ADR_EINVAL: return "ADR_EINVAL";
    case ADR_ENOMEM: return "ADR_ENOMEM";
    case ADR_ECUDA: return "ADR_ECUDA";
    case ADR_EUNSUPPORTED: return "ADR_EUNSUPPORTED";
    case ADR_ETIMEOUT: return "ADR_ETIMEOUT";
    case ADR_ENUMERIC: return "ADR_ENUMERIC";
    case ADR_EBUSY: return "ADR_EBUSY";
  }
  return "ADR_UNKNOWN";
}

extern "C" const char* adr_last_error(void) { return g_last_error.c_str(); }

extern "C" adr_status adr_plan_set_kernel(adr_plan P, int32_t kernel) {
  if (!P) return fail(ADR_EINVAL, "plan is NULL");
  if (kernel < -1 || kernel > 4) return fail(ADR_EINVAL, "kernel must be -1 or 0..4");
  if (__atomic_load_n(&P->batch_refs, __ATOMIC_ACQUIRE) > 0)
    return fail(ADR_EBUSY, "adr_plan_set_kernel: a live batch uses this plan; destroy the batch first");
  if (P->prec != ADR_BF16X3 && P->prec != ADR_TF32X3) return ADR_OK;
  ADR_CUDA_TRY(cudaStreamSynchronize(P->stream));
  if (P->gexec) cudaGraphExecDestroy(P->gexec);
  if (P->gexec_timed) cudaGraphExecDestroy(P->gexec_timed);
  P->gexec = P->gexec_timed = nullptr;
  P->g_u = P->g_v = P->gt_u = P->gt_v = nullptr;
  tc_free(&P->tc);
  tc_init(&P->tc);
  P->tc_variant = kernel;
  cudaError_t e = tc_prepare(&P->tc, P->prec, P->scheme, P->d, P->n, P->master, P->stream, kernel,
                             compensated(&P->prob));
  if (e != cudaSuccess)
    return fail(e == cudaErrorNotSupported ? ADR_EUNSUPPORTED : ADR_ECUDA,
                std::string("adr_plan_set_kernel: ") + cudaGetErrorString(e));
  return ADR_OK;
}

// ---------------------------------------------------------------- autotuner
extern "C" adr_status adr_autotune(const adr_problem* problem, void* stream, int32_t nsteps,
                                   adr_tuning* best, float ms_per_step[8]) {
  if (!problem || !best || !ms_per_step) return fail(ADR_EINVAL, "NULL argument");
  if (nsteps < 1 || nsteps > 1024) return fail(ADR_EINVAL, "adr_autotune: nsteps must be in [1, 1024]");
  adr_status st = validate(problem);
  if (st != ADR_OK) return st;
  memset(best, 0, sizeof(*best));
  best->kernel = -1;
  for (int k = 0; k < 8; ++k) ms_per_step[k] = -1.f;
  const int prec = problem->precision;
  if (prec != ADR_BF16X3 && prec != ADR_TF32X3) return ADR_OK;  // nothing to tune
  size_t N = 1;
  for (int m = 0; m < problem->d; ++m) N *= (size_t)problem->n[m];
  cudaStream_t s = (cudaStream_t)stream;
  void* u = nullptr;
  void* v = nullptr;
  ADR_CUDA_TRY(cudaMalloc(&u, N * sizeof(float)));
  if (cudaMalloc(&v, N * sizeof(float)) != cudaSuccess) {
    cudaFree(u);
    return fail(ADR_ENOMEM, "adr_autotune: scratch state");
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best_ms = -1.f;
  const int candidates[5] = {0, 1, 2, 3, 4};
  const int ncand = prec == ADR_TF32X3 ? 1 : 5;
  for (int c = 0; c < ncand; ++c) {
    const int k = prec == ADR_TF32X3 ? 1 : candidates[c];
    adr_tuning t;
    memset(&t, 0, sizeof(t));
    t.kernel = k;
    adr_plan P = nullptr;
    if (adr_plan_create_tuned(problem, &t, stream, &P) != ADR_OK) continue;
    bool ok = cudaMemsetAsync(u, 0, N * sizeof(float), s) == cudaSuccess &&
              cudaMemsetAsync(v, 0, N * sizeof(float), s) == cudaSuccess &&
              adr_step(P, u, v, 2) == ADR_OK && cudaEventRecord(e0, s) == cudaSuccess &&
              adr_step(P, u, v, nsteps) == ADR_OK && cudaEventRecord(e1, s) == cudaSuccess &&
              cudaEventSynchronize(e1) == cudaSuccess;
    float ms = 0.f;
    if (ok) ok = cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
    if (ok && tc_error_word(&P->tc)) {
      int h = 0;
      ok = cudaMemcpy(&h, tc_error_word(&P->tc), sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess &&
           h == 0;
    }
    adr_plan_destroy(P);
    if (!ok) {
      cudaGetLastError();
      continue;
    }
    ms_per_step[k] = ms / (float)nsteps;
    if (best_ms < 0.f || ms_per_step[k] < best_ms) {
      best_ms = ms_per_step[k];
      best->kernel = k;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(u);
  cudaFree(v);
  if (best->kernel < 0) return fail(ADR_EUNSUPPORTED, "adr_autotune: no kernel ran");
  return ADR_OK;
}

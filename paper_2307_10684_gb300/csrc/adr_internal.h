// Internal declarations shared by the translation units of libadr_gb300.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <functional>
#include <string>
#include <vector>

#include "../../include/adr.h"

namespace adr {

// Per-thread error message for adr_last_error().
void set_error(const std::string& msg);

#define ADR_CUDA_TRY(expr)                                                        \
  do {                                                                            \
    cudaError_t e_ = (expr);                                                      \
    if (e_ != cudaSuccess) {                                                      \
      ::adr::set_error(std::string(#expr) + ": " + cudaGetErrorString(e_));       \
      return ADR_ECUDA;                                                           \
    }                                                                             \
  } while (0)

// Tridiagonal directional operator with Neumann rows (interior row i:
// lo x_{i-1} + di x_i + up x_{i+1}; row 0: di x_0 + b0 x_1; row n-1:
// bn x_{n-2} + di x_{n-1}).  Row sums are zero, so the kernels evaluate
// lo (x_{i-1} - x_i) + up (x_{i+1} - x_i), which is the same value with
// far less cancellation in single precision.
template <typename T>
struct TridiagT {
  T lo, di, up, b0, bn;
};
using Tridiag = TridiagT<double>;

template <typename T>
struct ReactionT {
  int model;
  T p[16];
  T plo[16];  // low-order parts: p + plo is the double-precision parameter
              // (zero when T is double)
};

// Stencil + reaction description for one problem, passed by value.  The
// coefficients are held in the kernel's arithmetic type so that no kernel
// converts from double on the (slow) FP64 pipe.
template <typename T>
struct PointwiseArgsT {
  int d;
  int64_t n[3];
  int64_t N;
  TridiagT<T> A[2][3];    // [component][mu]
  TridiagT<T> Alo[2][3];  // low-order parts: A + Alo is the double-precision operator
                          // (zero when T is double)
  ReactionT<T> rx;
};
using PointwiseArgs = PointwiseArgsT<double>;

template <typename T>
inline PointwiseArgsT<T> cast_args(const PointwiseArgs& a) {
  PointwiseArgsT<T> r;
  r.d = a.d;
  r.N = a.N;
  for (int m = 0; m < 3; ++m) r.n[m] = a.n[m];
  for (int c = 0; c < 2; ++c)
    for (int m = 0; m < 3; ++m) {
      const Tridiag& x = a.A[c][m];
      r.A[c][m] = TridiagT<T>{(T)x.lo, (T)x.di, (T)x.up, (T)x.b0, (T)x.bn};
      const TridiagT<T>& h = r.A[c][m];
      r.Alo[c][m] = TridiagT<T>{(T)(x.lo - (double)h.lo), (T)(x.di - (double)h.di),
                                (T)(x.up - (double)h.up), (T)(x.b0 - (double)h.b0),
                                (T)(x.bn - (double)h.bn)};
    }
  r.rx.model = a.rx.model;
  for (int i = 0; i < 16; ++i) {
    r.rx.p[i] = (T)a.rx.p[i];
    r.rx.plo[i] = (T)(a.rx.p[i] - (double)r.rx.p[i]);
  }
  return r;
}

// Batched GEMM with per-component operand sets.  blockIdx.z = comp * batch
// + p.  C[p] = alpha * A[p] B[p] (+ beta * base[p]) (+ beta2 * base2[p]),
// A row-major M x K (lda), B row-major K x N (ldb), C/base/base2 row-major
// M x N (ldc).  *_bs are batch strides in elements.
struct GemmArgs {
  const void* A[2];
  const void* B[2];
  void* C[2];
  const void* base[2];
  const void* base2[2];
  int64_t lda, ldb, ldc;
  int64_t a_bs, b_bs, c_bs;
  int M, N, K;
  int batch;   // p range
  int ncomp;   // 1 or 2
  double alpha, beta, beta2;
};

// Kernel launchers (simt.cu).
template <typename T>
cudaError_t launch_gemm_simt(const GemmArgs& g, cudaStream_t s);
template <typename T>
cudaError_t launch_rhs(const PointwiseArgsT<T>& a, const T* u, const T* v, T* wu, T* wv,
                       cudaStream_t s);
template <typename T>
cudaError_t launch_lawson_pre(const PointwiseArgsT<T>& a, const T* u, const T* v, T scale, T* xu,
                              T* xv, cudaStream_t s);
template <typename T>
cudaError_t launch_lawson_post(const PointwiseArgsT<T>& a, const T* u2, const T* v2, T scale, T* u,
                               T* v, cudaStream_t s);
template <typename T>
cudaError_t launch_rdiff(const PointwiseArgsT<T>& a, const T* u, const T* v, const T* u2,
                         const T* v2, T* du, T* dv, cudaStream_t s);

// Matrix-function helpers (matfun.cu).
cudaError_t matfun_phi(int n, const Tridiag& A, double tau, double* E, double* P1, double* P2,
                       cudaStream_t s);
// The same for a dense row-major A (device), norm1_A = ||A||_1.
cudaError_t matfun_phi_dense(int n, const double* A, double norm1_A, double tau, double* E,
                             double* P1, double* P2, cudaStream_t s);
cudaError_t launch_build_dense(int n, const Tridiag& A, double scale, double* X, cudaStream_t s);
cudaError_t launch_convert(const double* src, void* dst, int64_t count, int to_double,
                           int transpose_n, cudaStream_t s);
cudaError_t launch_indicators(const PointwiseArgs& a, const void* up, const void* vp,
                              const void* u, const void* v, int is_double, double* acc,
                              cudaStream_t s);
cudaError_t launch_max_abs_diff(const void* x, int x_is_double, const double* ref, int64_t count,
                                unsigned long long* out2, cudaStream_t s);


// Refcounted process-wide cache of device buffer sets (cache.cu): nbuf
// buffers of `bytes` each, keyed by the values that determine their
// contents (plus the device).  On a miss the buffers are allocated, filled
// by fill() on stream s, and inserted once s has completed.  *hit tells
// whether the set was found.  shared_release takes the first buffer.
cudaError_t shared_acquire(std::vector<uint64_t> key, int nbuf, size_t bytes,
                           const std::function<cudaError_t(void* const*)>& fill, cudaStream_t s,
                           void** out, bool* hit);
void shared_release(void* first);
int64_t shared_sets_live();

inline uint64_t key_bits(double x) {
  uint64_t b;
  static_assert(sizeof(b) == sizeof(x), "64-bit double");
  memcpy(&b, &x, sizeof(b));
  return b;
}

struct GeneralState;  // general plans (general.cu): m components, dense A_mu

// Tensor-core operand set of a plan (tc.cu).
struct TcOperands {
  int prec;        // ADR_TF32X3 or ADR_BF16X3; 0 when unused
  void* mats[2][3][2];   // split operand matrices per [c][mu][ell-1]
  void* work[4];         // tensor-core workspace
  void* tmaps;           // device copy of tensor maps (opaque)
  int ready;
};

}  // namespace adr

enum KernelClass {
  KC_RHS = 0,
  KC_RDIFF = 1,
  KC_MODE_SIMT = 2,
  KC_MODE_TC = 3,
  KC_LAWSON_PW = 4,
  KC_COUNT = 5
};

struct TimedLaunch {
  int cls;
  cudaEvent_t e0, e1;
  double flops, bytes;
};

struct adr_plan_s {
  adr_problem prob;
  cudaStream_t stream;
  int d;
  int64_t n[3];
  int64_t N;
  int prec;
  int scheme;    // adr_scheme
  size_t esize;  // bytes per state element
  adr::PointwiseArgs pw;            // FP64 master
  adr::PointwiseArgsT<float> pwf;   // single-precision copy for FP32-state kernels
  // FP64 masters [c][mu][which], which: 0 = A, 1 = e^(tau A), 2 = phi_1, 3 = phi_2
  double* master[2][3][4];
  // SIMT operands: phi_ell row-major and transposed, in the state type
  void* op[2][3][3];    // [c][mu][ell]: ell 0 = e^(tau A), 1 = phi_1, 2 = phi_2
  void* opT[2][3][3];
  // tensor-core operands
  adr::TcOperands tc;
  // workspace
  void* u2;
  void* v2;
  void* bufA[2];
  void* bufB[2];
  void* dstate[2];  // device state for adr_solve with host buffers
  double* ind;      // 4 accumulators of adr_indicators
  std::vector<void*> allocs;
  adr::GeneralState* gen;     // non-null for plans of adr_plan_create_general
  std::vector<void*> shared;  // matrix sets held in the process-wide cache
  int32_t shared_hits;        // of them, found there (computed by another plan)
  // counters
  int64_t launches;
  int64_t steps;
  bool timing;
  std::vector<TimedLaunch> timed;        // directly launched, not yet harvested
  std::vector<TimedLaunch> graph_timed;  // captured in the timed graph; harvested per replay
  bool capturing;                        // a graph capture is recording the launches
  double acc_ms[KC_COUNT], acc_flops[KC_COUNT], acc_bytes[KC_COUNT];
  int64_t acc_count[KC_COUNT];
  std::vector<cudaEvent_t> event_pool;
  size_t event_next;
  // CUDA graph of kGraphChunk steps for one (u, v) pair, replayed by adr_step
  int use_graphs;
  cudaStream_t cap_stream;   // internal stream used only for capture
  cudaGraphExec_t gexec;
  void* g_u;
  void* g_v;
  int64_t g_launches;        // kernels per replay
  int tc_variant;            // requested tensor-core kernel (-1: the library's choice)
  int batch_refs;            // live batches over this plan (atomic; destroy and
                             // kernel changes are refused while non-zero)
  // timing mode: the same chunk captured with an event-record node before and
  // after every kernel, so that per-kernel times exclude host launch gaps
  cudaGraphExec_t gexec_timed;
  void* gt_u;
  void* gt_v;
};


namespace adr {
static const char* const kClassNames[KC_COUNT] = {"rhs_stencil_reaction", "reaction_diff",
                                                  "mode_product_simt", "mode_product_tc",
                                                  "lawson_pointwise"};
void tc_init(TcOperands* t);
void tc_free(TcOperands* t);
// variant_req: -1 = the library's choice, else a kernel variant (adr_tuning)
// comp: 2 = carry the state as hi + lo FP32 words across calls on the same
// (u, v) pair and evaluate the reactions in double-float
// (ADR_STATE_COMPENSATED); 0 = plain
cudaError_t tc_prepare(TcOperands* t, int prec, int scheme, int d, const int64_t n[3],
                       double* const master[2][3][4], cudaStream_t s, int variant_req, int comp);
// Clear the low-order state words (no-op without compensation).
cudaError_t tc_reset_state(TcOperands* t, cudaStream_t s);
// Start of a stepping call on (u, v): restarts the low-order words of a
// compensated state when the call needs it (enqueued on s).
cudaError_t tc_begin_call(TcOperands* t, void* u, void* v, cudaStream_t s);
cudaError_t tc_bind(TcOperands* t, adr_plan_s* P, void* u, void* v);
cudaError_t tc_step(TcOperands* t, adr_plan_s* P, void* u, void* v);
int* tc_error_word(TcOperands* t);
// Indicators of Sec. 4 accumulated by the last product of every step.
cudaError_t tc_set_indicators(TcOperands* t, int enable, cudaStream_t s);
cudaError_t tc_indicator_log(TcOperands* t, cudaStream_t s, double* out, int64_t max_steps,
                             int64_t* count);
cudaError_t tc_time_passes(TcOperands* t, adr_plan_s* P, void* u, void* v, int reps, float* ms,
                           int* passes);
// multiply-adds of one step's mode products: dense, and as the tiles run them
void tc_mode_macs(const TcOperands* t, double* dense, double* computed);

inline cudaEvent_t pool_event(adr_plan_s* P) {
  if (P->event_next < P->event_pool.size()) return P->event_pool[P->event_next++];
  cudaEvent_t e;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  P->event_pool.push_back(e);
  P->event_next++;
  return e;
}

// Inside a capture the event becomes an event-record node of the graph.
inline void record_event(adr_plan_s* P, cudaEvent_t e) {
  if (P->capturing)
    cudaEventRecordWithFlags(e, P->stream, cudaEventRecordExternal);
  else
    cudaEventRecord(e, P->stream);
}

// Launch wrapper: counts launches and, when timing is on, brackets the
// launch with events on the plan's stream.
template <typename F>
inline cudaError_t timed_kernel(adr_plan_s* P, int cls, double flops, double bytes, F&& fn) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (P->timing) {
    e0 = pool_event(P);
    e1 = pool_event(P);
    if (e0) record_event(P, e0);
  }
  cudaError_t err = fn();
  P->launches++;
  if (P->timing && e0 && e1) {
    record_event(P, e1);
    (P->capturing ? P->graph_timed : P->timed).push_back(TimedLaunch{cls, e0, e1, flops, bytes});
  }
  return err;
}

// Add the elapsed times of `v`'s launches (completed) to the plan's totals.
inline void harvest_timing(adr_plan_s* P, const std::vector<TimedLaunch>& v) {
  for (const TimedLaunch& t : v) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, t.e0, t.e1) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    P->acc_count[t.cls]++;
    P->acc_ms[t.cls] += ms;
    P->acc_flops[t.cls] += t.flops;
    P->acc_bytes[t.cls] += t.bytes;
  }
}
}  // namespace adr

// Advance a plan's (u, v) by nsteps, continuing its compensated state as it
// stands (api.cu; the batch path uses it for plans it steps one by one).
adr_status plan_step_continue(adr_plan plan, void* u, void* v, int64_t nsteps);

namespace adr {
// General plans (general.cu).
cudaError_t general_step(adr_plan P, void* const* U);
void general_free(adr_plan P);
int general_components(const adr_plan_s* P);
const double* general_master(const adr_plan_s* P, int c, int mu, int which);
}  // namespace adr

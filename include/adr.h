/*
 * adr.h - C ABI of the GB300 ETD2RKds time stepper.
 *
 * The library advances two-component advection-diffusion-reaction systems
 *     u_t = K^u u + g^u(u, v),   v_t = K^v v + g^v(u, v)
 * (Caliari & Cassini, arXiv:2307.10684, Sec. 1, Eq. 1-2) on a box grid of
 * n_1 x ... x n_d points (d = 2 or 3) with homogeneous Neumann boundaries,
 * using the directional split exponential integrator ETD2RKds
 * (Sec. 3, Eq. 11).  K^c = A_d^c (+) ... (+) A_1^c is a Kronecker sum
 * (Eq. 3) of tridiagonal second-order centred finite-difference matrices
 * (Sec. 4, opening text).  Each step is four Tucker operators (Eq. 5, Eq.
 * 10b) with the small dense matrices phi_1(tau A_mu^c), phi_2(tau A_mu^c)
 * plus two Kronecker-sum actions (Eq. 6) and the pointwise reactions.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * State layout: a state tensor is a dense array of n_1 * ... * n_d values
 *   with x_1 fastest (C array [n_d]...[n_2][n_1]); this is the column-major
 *   vec() ordering of Sec. 2.  Element type: double for ADR_FP64, float for
 *   every other precision.
 * Grid: vertex-centred, x_i = lo + i (hi - lo)/(n - 1), i = 0..n-1.
 *   Neumann rows mirror a ghost value across the boundary (u_{-1} = u_1).
 * Pointers: "device" means memory the GPU of the plan can address (cudaMalloc
 *   or managed); "host or device" arguments are classified with
 *   cudaPointerGetAttributes.
 * Streams: every call is enqueued on the plan's CUDA stream (the one given
 *   to adr_plan_create, 0 = legacy default stream) and is asynchronous with
 *   respect to the host unless it says otherwise.
 * Errors: every call returns an adr_status; no exception crosses the ABI.
 *   On ADR_EINVAL nothing was enqueued and user buffers are untouched.
 *   adr_last_error() gives a human-readable message for the calling thread.
 * Ownership: the caller owns state buffers; a plan owns its matrices and
 *   workspace, which adr_plan_destroy frees.
 * Threads: a plan may be used from one host thread at a time.
 */
#ifndef ADR_H
#define ADR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  ADR_OK = 0,
  ADR_EINVAL = 1,        /* invalid argument (problem, pointer, size)      */
  ADR_ENOMEM = 2,        /* device allocation failed                       */
  ADR_ECUDA = 3,         /* a CUDA runtime call failed                     */
  ADR_EUNSUPPORTED = 4,  /* valid but not implemented for this shape/prec. */
  ADR_ETIMEOUT = 5,      /* a bounded device wait gave up                  */
  ADR_ENUMERIC = 6,      /* non-finite value detected                      */
  ADR_EBUSY = 7          /* resource busy (admission refused)              */
} adr_status;

/* Reaction models g^u, g^v and the meaning of adr_problem.params[]
 * (unused entries must be 0):
 *  ADR_SCHNAKENBERG (Sec. 4.1, Eq. 12): params {gamma, a, b}
 *     g^u = gamma (a - u + u^2 v),  g^v = gamma (b - u^2 v)
 *  ADR_FHN, FitzHugh-Nagumo with linear recovery: params {eps, a1, a0}
 *     g^u = u - u^3 - v,            g^v = eps (u - a1 v - a0)
 *  ADR_BRUSSELATOR (Sec. 4.6, Eq. 17): params {a, b}
 *     g^u = a - (b + 1) u + u^2 v,  g^v = b u - u^2 v
 *  ADR_NO_REACTION: g^u = g^v = 0 (linear advection-diffusion). */
typedef enum {
  ADR_SCHNAKENBERG = 0,
  ADR_FHN = 1,
  ADR_BRUSSELATOR = 2,
  ADR_NO_REACTION = 3,
  ADR_FHN_RHO = 4,   /* FitzHugh-Nagumo as in Sec. 4.2-4.3, Eq. 13-14:
                        params {rho, a1, a2}: g^u = rho (u - u^3 - v),
                        g^v = rho a1 (u - a2 v)                             */
  ADR_DIB = 5        /* morpho-chemical DIB model, Sec. 4.4, Eq. 15: params
                        {rho, a1u, a2u, a3u, a4u, a1v, a2v, a3v, a4v, a5v}:
                        g^u = rho (a1u (1 - v) u - a2u u^3 - a3u (v - a4u)),
                        g^v = rho (a1v (1 + a2v u) (1 - v) (1 - a3v (1 - v))
                                   - a4v v (1 + a5v u) (1 + a3v v))         */
} adr_model;

/* Arithmetic of the mode products (the Tucker operators).
 *  ADR_FP64   : double state, double SIMT products.
 *  ADR_FP32   : float state, float SIMT products (FP32 FMA).
 *  ADR_TF32X3 : float state, tcgen05 kind::tf32 products with operands split
 *               into two TF32 parts, hi + lo (three MMAs: the lo x lo term is
 *               dropped), FP32 accumulation.  About 22 significant bits per
 *               operand: less accurate than ADR_BF16X3, at the same MMA cost
 *               and more operand bytes.  Same grid rule as ADR_BF16X3.
 *  ADR_BF16X3 : float state, tcgen05 tensor-core products with operands
 *               split into three BF16 parts (6 MMAs, FP32 accumulation);
 *               needs every n[mu] to be a multiple of 8, else
 *               ADR_EUNSUPPORTED.
 * Matrix functions are always evaluated in FP64 on the GPU. */
typedef enum {
  ADR_FP64 = 0,
  ADR_FP32 = 1,
  ADR_TF32X3 = 2,
  ADR_BF16X3 = 3
} adr_precision;

/* Time-stepping scheme.
 *  ADR_ETD2RKDS : directional split ETD2RK, Sec. 3, Eq. 11 (the default).
 *  ADR_LAWSON2B : second-order Lawson scheme in tensor form, Eq. 7: two
 *                 Tucker operators of e^(tau A_mu) per component and step;
 *                 no splitting error, so exact to rounding when g = 0. */
typedef enum {
  ADR_ETD2RKDS = 0,
  ADR_LAWSON2B = 1
} adr_scheme;

/* How a single-precision state is carried from step to step.
 *  ADR_STATE_AUTO        : the library's choice: plain (below).
 *  ADR_STATE_PLAIN       : the caller's buffers are the whole state; each
 *                          stage update U + tau T of Eq. 11 is rounded to
 *                          FP32 and the reactions are evaluated in FP32.
 *                          Over long horizons these roundings accumulate, by
 *                          ~1e-7 relative per step and more where the
 *                          dynamics amplify them.
 *  ADR_STATE_COMPENSATED : the accurate mode for long or unstable horizons.
 *                          The state is hi + lo: hi in the caller's buffer
 *                          (the FP32 value nearest the state) and lo, a
 *                          low-order FP32 word per point and component, in
 *                          plan memory.  The stage updates of Eq. 11 add the
 *                          increment to hi + lo with its exact rounding
 *                          error (TwoSum) and renormalise, so the state
 *                          keeps about 48 bits; the right-hand sides are
 *                          evaluated from hi, with the reactions (and the
 *                          stage-2 reaction difference) in double-float
 *                          arithmetic and double-float parameters, since an
 *                          FP32 reaction whose terms cancel loses digits
 *                          every step.  Costs 16 bytes of traffic per point
 *                          and step and more pointwise arithmetic.  The lo
 *                          words carry over from one call to the next while
 *                          the plan (alone or in a batch) steps the same
 *                          (u, v) pair; they restart at zero when it steps
 *                          another pair, when adr_solve starts, and on
 *                          adr_plan_reset_state.  A caller that writes new
 *                          values into buffers the plan has stepped calls
 *                          adr_plan_reset_state.
 * Compensation applies to tensor-core ETD2RKds plans only: other plans
 * asking for ADR_STATE_COMPENSATED get ADR_EUNSUPPORTED. */
typedef enum {
  ADR_STATE_AUTO = 0,
  ADR_STATE_PLAIN = 1,
  ADR_STATE_COMPENSATED = 2
} adr_state_mode;

/* One problem.  Direction mu = 0 is x_1 (the contiguous axis). */
typedef struct {
  int32_t d;            /* 2 or 3                                           */
  int32_t model;        /* adr_model                                        */
  int32_t precision;    /* adr_precision                                    */
  int32_t scheme;       /* adr_scheme                                       */
  int64_t n[3];         /* grid points per direction, 3 <= n[mu] <= 4096    */
  double lo[3], hi[3];  /* domain [lo_mu, hi_mu], hi > lo                   */
  double diff[2];       /* diffusion delta^u, delta^v (> 0)                 */
  double adv[2][3];     /* velocity of the term -adv[c] . grad(c)           */
  double params[16];    /* model constants, see adr_model                   */
  double tau;           /* constant time step (> 0)                         */
  int32_t state;        /* adr_state_mode (0 = the library's choice)        */
  int32_t reserved;     /* must be 0                                        */
} adr_problem;

typedef struct adr_plan_s* adr_plan;

/* Create a plan: validates the problem, builds the directional matrices
 * A_mu^c, evaluates e^(tau A_mu^c), phi_1(tau A_mu^c), phi_2(tau A_mu^c) in
 * FP64 on the GPU (Pade [13/13] scaling and squaring of the augmented matrix
 * [[X, I, 0], [0, 0, I], [0, 0, 0]], X = tau A_mu^c; phi_ell is Eq. 9),
 * converts them to the kernel operand format and allocates the step
 * workspace.  Synchronises the stream before returning.
 *   problem : host pointer, read only.
 *   stream  : cudaStream_t (as void*), 0 for the default stream.
 *   out     : receives the plan; untouched on failure. */
adr_status adr_plan_create(const adr_problem* problem, void* stream, adr_plan* out);

/* Kernel choice of a tensor-core plan (ADR_BF16X3 / ADR_TF32X3), as chosen
 * by adr_autotune.  The paper has no counterpart: it concerns only how the
 * mode products of Eq. 11 are tiled on the GPU, not what they compute.
 *   kernel : -1 = the library's choice from the grid size;
 *            0 = one CTA per 128 x 128 tile, 64-byte swizzle, 4 stages;
 *            1 = one CTA per 128 x 128 tile, 128-byte swizzle, 2 stages;
 *            2 = one CTA per 128 x 64 tile, 64-byte swizzle;
 *            3 / 4 = two-SM (cta_group::2) 256 x 128 tiles, 64- / 128-byte
 *            swizzle.  TF32X3 plans always use 1.
 * Every kernel computes the same products in the same order per output. */
typedef struct {
  int32_t kernel;
  int32_t reserved[7];
} adr_tuning;

/* adr_plan_create with an explicit kernel choice (tuning may be NULL: the
 * library's choice).  Other precisions ignore it. */
adr_status adr_plan_create_tuned(const adr_problem* problem, const adr_tuning* tuning,
                                 void* stream, adr_plan* out);

/* Switch an existing tensor-core plan to another kernel (adr_tuning.kernel)
 * without recomputing its FP64 matrix functions: synchronises the plan's
 * stream and rebuilds only the kernel operands, tensor maps and graphs.
 * ADR_EBUSY (nothing changed) while a batch created over the plan is alive.
 * FP32 / FP64 plans: no-op.
 * On failure the plan cannot step until a later call succeeds. */
adr_status adr_plan_set_kernel(adr_plan plan, int32_t kernel);

/* Self-test of the bounded waits that every tensor-core and staging kernel
 * uses (no counterpart in the paper: it checks this library's failure
 * detection).  One kernel on `stream` waits on a shared-memory mbarrier
 * that a thread of another warp arrives on (arrive != 0) or that nothing
 * arrives on (arrive == 0), gives up after limit_ns nanoseconds of
 * %globaltimer (1e6 <= limit_ns <= 2e9), and records the timeout code in a
 * device error word, as a kernel of a step does.  Synchronises the stream;
 * *code = the error word (0, or 1 = a wait gave up), *waited_ns = the wait's
 * length measured on the device.  ADR_OK when the kernel ran, whatever the
 * code; the CUDA context stays usable either way. */
adr_status adr_selftest_bounded_wait(void* stream, int32_t arrive, int64_t limit_ns, int32_t* code,
                                     int64_t* waited_ns);

/* Autotuner: for a tensor-core problem, builds a plan with each candidate
 * kernel, advances scratch state (allocated here, zero-filled) by 2 + nsteps
 * steps on `stream` and times the last nsteps with CUDA events.  best
 * receives the fastest kernel; ms_per_step[k] the time per step of kernel k
 * (-1 when k is not a candidate or failed).  For FP32 / FP64 problems there
 * is nothing to tune: best->kernel = -1 and every entry is -1.  Synchronous;
 * allocates and frees device memory.  nsteps in [1, 1024]. */
adr_status adr_autotune(const adr_problem* problem, void* stream, int32_t nsteps,
                        adr_tuning* best, float ms_per_step[8]);

/* Move a plan to another CUDA stream (as void*, 0 = default stream): later
 * calls enqueue there.  Synchronises the old stream first, so work already
 * enqueued is complete.  Lets a plan be built on one stream (for instance
 * on a planner thread) and stepped on another. */
adr_status adr_plan_set_stream(adr_plan plan, void* stream);

/* Free a plan (synchronises its stream first).  NULL is accepted.
 * ADR_EBUSY (nothing freed) while a batch created over the plan is alive. */
adr_status adr_plan_destroy(adr_plan plan);

/* Advance (u, v) by nsteps ETD2RKds steps in place (Eq. 11):
 *   U2 = U + tau (sum_mu U x_mu A_mu^u + G^u(U,V)) x_mu phi_1(tau A_mu^u)
 *   U+ = U2 + 2^(d-1) tau (G^u(U2,V2) - G^u(U,V)) x_mu phi_2(tau A_mu^u)
 * and likewise for V.  u, v: device pointers to state tensors (layout
 * above), distinct, not aliasing plan memory; for ADR_BF16X3 plans both
 * 16-byte aligned (ADR_EINVAL otherwise).  nsteps >= 0.  Asynchronous. */
adr_status adr_step(adr_plan plan, void* u, void* v, int64_t nsteps);

/* Restart the compensation of a plan's state (adr_state_mode): the
 * low-order words are cleared, so the next step continues from the
 * caller's buffers alone.  Call it after writing new values into buffers
 * the plan has already stepped under ADR_STATE_COMPENSATED.  Enqueued on
 * the plan's stream; a no-op for plain plans.  No counterpart in the paper. */
adr_status adr_plan_reset_state(adr_plan plan);

/* Solve from (u0, v0) for nsteps steps into (uT, vT).  Each pointer may be
 * host or device memory; host inputs are copied to the device, host outputs
 * copied back, and in that case the call returns after the copy-back has
 * completed (returning ADR_ETIMEOUT if a kernel gave up a bounded wait).
 * With device pointers only it is asynchronous.  u0/v0 may equal uT/vT. */
adr_status adr_solve(adr_plan plan, const void* u0, const void* v0, void* uT, void* vT,
                     int64_t nsteps);

/* Bytes a plan for `problem` would hold: state_bytes = one (u, v) pair in
 * the run precision; cache_bytes = matrices + workspace.  Host only. */
adr_status adr_plan_bytes(const adr_problem* problem, size_t* state_bytes, size_t* cache_bytes);

/* Copy one FP64 plan matrix to host memory `out` (n_mu * n_mu doubles,
 * row-major, out[i * n + j] = M[i][j]).  which: 0 = A_mu^c, 1 = e^(tau A),
 * 2 = phi_1(tau A), 3 = phi_2(tau A).  component: 0 = u, 1 = v.  mu: 0..d-1.
 * Synchronous. */
adr_status adr_plan_matrix(adr_plan plan, int which, int component, int mu, double* out);

/* Measurement aid (no counterpart in the paper): the duration of one
 * tensor-core mode-product launch as it runs inside a step.  The launches
 * of `reps` steps' Tucker operators are captured back to back in one CUDA
 * graph (per ETD2RKds step: 2 on 2D grids and 4 on 3D grids with BF16x3
 * products, where the first two directions of an operator share one
 * launch; 4 d with one launch per direction), with programmatic
 * dependent launch between them and no timing node in between, and the
 * graph is replayed
 * once to warm up and once between two CUDA events on the plan's stream.
 * *ms_per_launch = that replay's time / (reps x *launches_per_step).
 * u, v: device scratch state buffers of the plan's shape, 16-byte aligned;
 * their contents are overwritten (the last product of each Tucker operator
 * writes the state).  reps in [1, 4096].  Tensor-core plans only
 * (ADR_EUNSUPPORTED otherwise).  Synchronous. */
adr_status adr_plan_time_mode_products(adr_plan plan, void* u, void* v, int32_t reps,
                                       double* ms_per_launch, int32_t* launches_per_step);

/* Measurement aid: multiply-adds of the mode products of one time step.
 * *dense counts them as the Tucker operators of Eq. 5 state them: per
 * component, two operators of d full contractions, N n_mu multiply-adds
 * each (4 N sum_mu n_mu for two components).  *computed counts what the
 * kernels run.  On the tensor-core path every 128-row group of
 * phi(tau A_mu) contracts only over the column support of its rows: the
 * union of each row's narrowest column range whose left-out entries weigh
 * at most 2^-40 of the row's absolute sum (from the FP64 matrix at plan
 * time), widened to multiples of 64 columns, the same for every kernel
 * choice.  The left-out part of a product is then below
 * 2^-40 max|x| sum_j |phi_ij| per row, far below the products' own 2^-24
 * rounding.  (The environment variable ADR_KSUPPORT=0, read at plan
 * creation, runs every tile over all of K.)  Other plans: *computed =
 * *dense.  Host-only, never fails on a valid plan. */
adr_status adr_plan_mode_product_macs(adr_plan plan, double* dense, double* computed);

/* Counters of a plan since creation (or the last reset). */
typedef struct {
  int64_t launches;        /* kernels launched by adr_step / adr_solve     */
  int64_t steps;           /* ETD2RKds steps enqueued                      */
  int32_t timing;          /* 1 if per-kernel event timing is on           */
  int32_t nkernels;        /* entries used in the arrays below             */
  int32_t device_error;    /* 0, or the code a bounded device wait left    */
  int32_t shared_matrices; /* directional matrix sets (A, e^(tau A), phi_1,
                              phi_2 of one operator) this plan took from the
                              library's cache instead of computing: plans
                              whose operators and step coincide share one
                              refcounted copy (as do their split operand
                              pieces)                                         */
  char    name[16][32];    /* kernel class names                           */
  int64_t count[16];       /* timed launches per class                     */
  double  ms[16];          /* summed CUDA-event time per class (ms)        */
  double  flops[16];       /* algorithmic flops per class (summed)         */
  double  bytes[16];       /* algorithmic bytes per class (summed)         */
} adr_stats;

/* Turn per-kernel CUDA-event timing on (1) or off (0); clears counters. */
adr_status adr_plan_set_timing(adr_plan plan, int enable);
/* Fetch counters; synchronises the plan's stream.  device_error != 0 means
 * a kernel gave up a bounded wait (its results are invalid); the plan stays
 * usable and the word is cleared by adr_plan_set_timing. */
adr_status adr_plan_stats(adr_plan plan, adr_stats* out);

/* ---------------------------------------------------------------- batches
 * Many independent solves (say hundreds of grids of different sizes)
 * advanced together.  When every plan is ADR_BF16X3 with the same d, one
 * step of the whole batch is a fixed set of grouped launches: one stencil
 * launch, one launch per mode-product pass covering every solve's tiles (a
 * persistent tcgen05 kernel reading per-solve descriptors; the first two
 * directions of an operator form one pass), one
 * reaction-difference launch; runs of 16 steps
 * replay a captured CUDA graph.  Other batches step their plans in turn.
 * The batch uses the plans' matrices and workspaces: while a batch steps, do
 * not step its plans on their own.  The plans must outlive the batch:
 * adr_plan_destroy and adr_plan_set_kernel return ADR_EBUSY for a plan that
 * a live batch uses. */
typedef struct adr_batch_s* adr_batch;

/* Build a batch of `count` plans (host array, copied); launches go to
 * `stream`.  Synchronous. */
adr_status adr_batch_create(const adr_plan* plans, int count, void* stream, adr_batch* out);
adr_status adr_batch_destroy(adr_batch batch);
/* Advance solve i's device state (u[i], v[i]) by nsteps[i] steps (its own
 * horizon, >= 0); u, v and nsteps are host arrays of `count` entries.  The
 * solves advance in lock-step while they run: between consecutive distinct
 * horizons the solves that are still running form one grouped launch
 * sequence (a batch over that subset, built on first use and kept with the
 * batch), so a solve that has finished drops out of the work of the rest.
 * The first call with a new set of pointers (per subset) uploads the
 * per-solve descriptors; calls are asynchronous. */
adr_status adr_batch_step(adr_batch batch, void* const* u, void* const* v, const int64_t* nsteps);
/* Timing and counters of the batch's launches (as for plans). */
adr_status adr_batch_set_timing(adr_batch batch, int enable);
adr_status adr_batch_stats(adr_batch batch, adr_stats* out);
/* 1 when the batch runs grouped tensor-core launches, 0 when it steps its
 * plans in turn. */
int adr_batch_is_grouped(adr_batch batch);

/* Error reduction (FP64 on the GPU): out[0] = max_i |x_i - ref_i|,
 * out[1] = max_i |ref_i| over `count` elements.  x: device array of float
 * (x_is_double = 0) or double (1); ref: device array of double.  out: host.
 * Enqueued on `stream` and synchronised before returning. */
adr_status adr_max_abs_diff(void* stream, const void* x, int x_is_double, const double* ref,
                            int64_t count, double out[2]);

/* Same result as adr_max_abs_diff, but allocates no device memory.  The
 * paper has no counterpart: this is a service for callers that cannot
 * allocate at the point where they check a result (a serving loop whose
 * device-memory budget is fully committed, a host application that owns the
 * CUDA allocator, code that must avoid cudaFree's implicit synchronisation).
 * Scratch is a 256 KB device array inside the library image, held by every
 * GPU that loads the library until the process exits.  Limit: count <=
 * 67,108,864 (2^26) elements; larger counts return ADR_EINVAL and enqueue
 * nothing.  The first call on a device resolves the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  The resolved address is kept for the life of
 * the process: it belongs to the device's primary context, so after a
 * cudaDeviceReset of that device in this process it is stale and this entry
 * point must not be called again.  All calls share the one array, so calls that
 * overlap on the GPU (different streams, or different host threads) race and
 * may return each other's results.  Enqueued on `stream`, synchronised before
 * returning; out: host. */
adr_status adr_max_abs_diff_noalloc(void* stream, const void* x, int x_is_double,
                                    const double* ref, int64_t count, double out[2]);

/* Dynamics indicators of Sec. 4 for the state (u, v) after a step from
 * (u_prev, v_prev): out[0], out[1] = spatial means <U>, <V> (trapezoid
 * weights on the vertex grid, divided by the weights' sum, i.e. by |Omega|
 * in grid units); out[2], out[3] = ||U - U_prev||_F, ||V - V_prev||_F.  All
 * four pointers are device state tensors of the plan's shape and type; out
 * is host memory.  Accumulates in FP64 on the GPU into plan-owned scratch;
 * synchronous. */
adr_status adr_indicators(adr_plan plan, const void* u_prev, const void* v_prev, const void* u,
                          const void* v, double out[4]);

/* Indicators of Sec. 4 fused into the step: with them on, the last product
 * of every ETD2RKds step also accumulates, in FP64, the trapezoid-weighted
 * spatial means <U_{n+1}>, <V_{n+1}> and the increments ||U_{n+1} - U_n||_F,
 * ||V_{n+1} - V_n||_F (reading the previous state before overwriting it: 8
 * bytes more traffic per point and step), into a ring of the last 4096 steps
 * in plan memory.  Tensor-core ETD2RKds plans only (ADR_EUNSUPPORTED
 * otherwise), not while a live batch uses the plan (ADR_EBUSY).  Enabling
 * clears the history; the state results are the same with them on or off.
 * Synchronises the plan's stream. */
adr_status adr_plan_set_indicators(adr_plan plan, int enable);
/* The indicators of the last min(max_steps, steps since enabling, 4096)
 * steps, oldest first: out[4 k + 0..3] = <U>, <V>, ||dU||_F, ||dV||_F of
 * step k.  *count = the number of steps written.  Synchronous. */
adr_status adr_plan_indicator_log(adr_plan plan, double* out, int64_t max_steps, int64_t* count);
/* Step-count-free run (the pattern and equilibrium runs of Sec. 4): advance
 * (u, v) in place (device pointers) until the physical time t_end, that is
 * ceil(t_end / tau) steps, or, when tol > 0, until the increment indicator
 * of a checked step, max(||U_{n+1} - U_n||_F, ||V_{n+1} - V_n||_F), is at
 * most tol (a stationary state).  The indicators are checked every
 * check_every >= 1 steps, each check synchronising the plan's stream.
 * *steps_done = steps taken; ind_last = the indicators of the last step.
 * Needs adr_plan_set_indicators(plan, 1).  Synchronous. */
adr_status adr_run(adr_plan plan, void* u, void* v, double t_end, double tol, int64_t check_every,
                   int64_t* steps_done, double ind_last[4]);

/* ---------------------------------------------------------------- general
 * Plans beyond the finite-difference two-component setting: the method
 * needs nothing of the directional matrices but their size (Sec. 1, Eq. 3-4:
 * any A_mu in the Kronecker sum) and extends to more than two components
 * (Sec. 3, closing remark).  A general plan has m = 1..4 components, caller
 * matrices A_mu^c (dense, any entries), and a polynomial reaction: each term
 * adds coef * prod_j u_j^pow[j] to g^comp.  One step is Eq. 11 per
 * component, with K^c U_c = sum_mu U_c x_mu A_mu^c as d dense mode products;
 * every stage value is formed before any stage-2 reaction.  Products in
 * FP64 or FP32 (ADR_FP64 / ADR_FP32; other precisions: ADR_EUNSUPPORTED);
 * matrix functions in FP64 on the GPU as for the other plans (Pade [13/13]
 * scaling and squaring, dense powers and LU). */
typedef struct {
  int32_t comp;     /* component the term adds to, 0..m-1                  */
  int32_t pow[4];   /* exponents of u_0..u_3, 0..8 (0 beyond m)             */
  double coef;      /* finite                                              */
} adr_term;

typedef struct {
  int32_t d;                 /* 2 or 3                                     */
  int32_t m;                 /* components, 1..4                           */
  int32_t precision;         /* ADR_FP64 or ADR_FP32                       */
  int32_t nterms;            /* 0..64                                      */
  int64_t n[3];              /* grid points per direction, 1..4096          */
  const double* A[4][3];     /* host, A[c][mu]: n[mu] x n[mu] row-major,
                                read during the call only                   */
  const adr_term* terms;     /* host, nterms entries, read during the call  */
  double tau;                /* constant step (> 0)                        */
} adr_general_problem;

/* Create a general plan (copies everything it needs).  Synchronises the
 * stream.  adr_step / adr_solve / batches refuse general plans
 * (ADR_EINVAL); adr_plan_matrix, adr_plan_stats, adr_plan_set_timing and
 * adr_plan_destroy work as for other plans (component 0..m-1). */
adr_status adr_plan_create_general(const adr_general_problem* problem, void* stream,
                                   adr_plan* out);
/* Advance the m device state tensors states[0..m-1] (layout as above,
 * double for ADR_FP64, float for ADR_FP32, distinct) by nsteps steps in
 * place.  Asynchronous. */
adr_status adr_step_general(adr_plan plan, void* const* states, int64_t nsteps);

/* Short name of a status code (static storage). */
const char* adr_status_str(adr_status s);
/* Message describing the last failure on the calling host thread. */
const char* adr_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* ADR_H */

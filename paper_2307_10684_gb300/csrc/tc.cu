// Tensor-core (tcgen05) path of the ETD2RKds step, BF16x3 split precision.
//
// Every mu-mode product of a Tucker operator (Sec. 2, Eq. 5; Eq. 10b) is one
// GEMM of the same shape,
//     out[n][m] = sum_k Phi[n][k] X[m][k],       X = [M rows][K = n_mu],
// i.e. out = (X Phi^T)^T.  Writing the product transposed rotates the axes:
// a state stored [i3][i2][i1] (x_1 fastest) becomes [i1][i3][i2] after the
// x_1 product, [i2][i1][i3] after the x_2 product and [i3][i2][i1] again after
// the x_3 product (2D: [i2][i1] -> [i1][i2] -> [i2][i1]).  So every operand is
// K-major, loaded by TMA with 128-byte swizzle, and the transposed store is
// coalesced because the accumulator's TMEM lanes are the m index.
//
// Split precision: each FP32 operand x is held as three BF16 pieces
// x = b0 + b1 + b2 (round to nearest at each level, ~24 significant bits);
// the product sum_k a_k c_k is formed from the six piece products whose
// order is <= 2^-16 relative: (0,0) (0,1) (1,0) (1,1) (0,2) (2,0), all
// accumulated in one FP32 TMEM accumulator by tcgen05.mma kind::f16.
//
// Kernel roles (192 threads): warp 0 issues TMA loads, warp 1 owns TMEM and
// issues MMAs (one elected thread), warps 2-5 run the epilogue (warp w reads
// TMEM lanes 32 (w % 4) .. +31).  Every wait is bounded (about 2 s of
// %globaltimer); on timeout the kernel records an error code, drains what it
// issued and frees TMEM before returning.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>

#include <map>
#include <mutex>

#include "adr_internal.h"
#include "pointwise.cuh"

namespace adr {

namespace {

constexpr int kBM = 128;       // rows per tile (TMEM lanes)
constexpr int kPieces = 3;     // BF16 pieces of an FP32 value

// Operand formats of the tensor-core path: three BF16 pieces per value with
// six products (kind::f16), or two TF32 pieces (stored as FP32 words whose
// low 13 mantissa bits are zero) with three products (kind::tf32).  Both
// take 32 bytes of K per MMA, so the shared-memory layouts are the same.
enum { kFmtBF16 = 0, kFmtTF32 = 1 };
template <int F>
struct Fmt {
  static constexpr int P = F == kFmtTF32 ? 2 : 3;     // pieces
  static constexpr int ESZ = F == kFmtTF32 ? 4 : 2;   // bytes per piece element
};
constexpr uint64_t kWaitNs = 2000000000ull;    // bounded waits: 2 s

// Tile configuration: SW = bytes of K per stage row (the swizzle width: 64
// or 128, i.e. 32 or 64 BF16 values), BN = output columns per tile.
template <int SW, int BN, int F = kFmtBF16>
struct TcCfg {
  static constexpr int P = Fmt<F>::P;
  static constexpr int BK = SW / Fmt<F>::ESZ;        // K elements per stage
  static constexpr int KSTEPS = SW / 32;             // 32-byte MMA K steps per stage
  static constexpr int TILE_A = kBM * SW;            // bytes of one A piece tile
  static constexpr int TILE_B = BN * SW;             // bytes of one B piece tile
  static constexpr int STAGE = P * (TILE_A + TILE_B);
  static constexpr int STAGES = (224 * 1024) / STAGE > 8 ? 8 : (224 * 1024) / STAGE;
  static constexpr int SMEM = STAGES * STAGE + 1024 + 512;  // + alignment, barriers
  static constexpr int TMEM_COLS = 2 * BN;           // two accumulators
  static constexpr uint32_t LAYOUT = SW == 128 ? 2u : 4u;   // descriptor swizzle code
  static constexpr uint32_t SBO = 8 * SW;            // bytes between 8-row groups
};

// error codes written to the plan's device error word
constexpr int kErrTimeoutFull = 1, kErrTimeoutEmpty = 2, kErrTimeoutDone = 3;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for a phase expected to take a while (an epilogue waiting for its
// accumulator): polls with a back-off, leaving the issue slots to the
// producer and MMA warps; false after kWaitNs.
__device__ __forceinline__ bool mbar_wait_sleep(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer();
  while (!mbar_try_wait(bar, parity)) {
    __nanosleep(256);
    if (globaltimer() - t0 > kWaitNs) return false;
  }
  return true;
}
// Wait with acquire semantics at cluster scope (the phase is completed by
// arrivals from the other CTA of the cluster); false after kWaitNs.
__device__ __forceinline__ bool mbar_try_wait_cluster(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_cluster(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait_cluster(bar, parity)) return true;
  const uint64_t t0 = globaltimer();
  while (!mbar_try_wait_cluster(bar, parity)) {
    if (globaltimer() - t0 > kWaitNs) return false;
  }
  return true;
}
// Wait for the phase with the given parity; false after limit_ns.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint64_t limit_ns = kWaitNs) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer();
  while (!mbar_try_wait(bar, parity)) {
    if (globaltimer() - t0 > limit_ns) return false;
  }
  return true;
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int x, int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(smem_u32(dst)),
      "l"((uint64_t)map), "r"(smem_u32(bar)), "r"(x), "r"(y), "r"(z)
      : "memory");
}
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   smem_u32(dst)),
               "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// The A operand collector: kColFill reads A from shared memory and keeps it,
// kColUse / kColLast reuse the kept A (the last use releases it), kColNone
// reads A and keeps nothing.  Consecutive MMAs on the same A tile then read
// it from shared memory once.
enum { kColNone = 0, kColFill = 1, kColUse = 2, kColLast = 3 };
template <int COL>
__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t acc) {
  if constexpr (COL == kColFill) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16.collector::a::fill [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
  } else if constexpr (COL == kColUse) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16.collector::a::use [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
  } else if constexpr (COL == kColLast) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16.collector::a::lastuse [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
  } else {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
  }
}
// kind::tf32 (A and B TF32 in shared memory, FP32 accumulate), same collector use.
template <int COL>
__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t acc) {
  if constexpr (COL == kColFill) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32.collector::a::fill [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
  } else if constexpr (COL == kColLast) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32.collector::a::lastuse [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
  } else {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
  }
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}
// 32 lanes x 32 bit, 16 consecutive columns per thread.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// tmem_ld16 without the wait: the registers are valid only after
// tmem_wait_ld() and tmem_fence16() on them.
__device__ __forceinline__ void tmem_ld16_nw(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
// Orders every later use of r after the preceding tmem_wait_ld().
__device__ __forceinline__ void tmem_fence16(uint32_t (&r)[16]) {
  asm volatile(""
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]),
                 "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]),
                 "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15])
               :
               : "memory");
}

// Shared-memory matrix descriptor of a K-major tile with SW-byte swizzle
// (SW = 64 or 128): rows of SW bytes, 8-row groups 8*SW bytes apart (stride
// byte offset), descriptor version 1 (bit 46), swizzle code at bits 61-63
// (2 = 128-byte, 4 = 64-byte).  The leading byte offset is not used by
// swizzled K-major layouts whose K step (32 bytes) fits in one swizzle row.
template <int SW>
__device__ __forceinline__ uint64_t kmajor_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)((8 * SW) >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)(SW == 128 ? 2 : 4) << 61;
  return d;
}

// Shared-memory matrix descriptor of an MN-major tile with 128-byte swizzle:
// atoms of 64 M values (128 bytes) by 8 K rows, consecutive atoms along K
// `sbo` bytes apart and the second 64 M values `lbo` bytes from the first.
__device__ __forceinline__ uint64_t mnmajor_desc128(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}
// A operand of a stage in the MMA issue loops: the descriptor of piece 0 at
// the stage's first K step, and the descriptor increments (16-byte units)
// from one piece to the next and from one K16 step to the next.
struct AOperand {
  uint64_t d;
  uint32_t piece, kstep;
};
// K-major A tile of P pieces of 128 rows x SW bytes, or (amn) MN-major:
// [M half][piece][bk K rows][128 bytes] as two TMA boxes of 64 M values.
template <int SW>
__device__ __forceinline__ AOperand a_operand(uint32_t stage, bool amn) {
  constexpr int BK = SW / 2;  // BF16 values of K per stage
  if (amn) return {mnmajor_desc128(stage, kPieces * BK * 128, 1024), (uint32_t)(BK * 128 >> 4), 128u};
  return {kmajor_desc<SW>(stage), (uint32_t)(kBM * SW >> 4), 2u};
}

// Instruction descriptor, kind::f16: D = F32 (bits 4-5 = 1), A = B = BF16
// (bits 7-9 = 1, 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bits
// 17-22, M >> 4 at bits 24-28.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

// Instruction descriptor, kind::tf32: as above with A = B = TF32 (code 2).
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

// x = hi + lo with hi, lo TF32 (round to nearest, ties away, at each level);
// about 22 significant bits of x.
__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}
__device__ __forceinline__ void split2_tf32(float x, float& hi, float& lo) {
  hi = tf32_rna(x);
  lo = tf32_rna(x - hi);
}

__device__ __forceinline__ void split3(float x, __nv_bfloat16& b0, __nv_bfloat16& b1,
                                       __nv_bfloat16& b2) {
  b0 = __float2bfloat16_rn(x);
  const float r1 = x - __bfloat162float(b0);
  b1 = __float2bfloat16_rn(r1);
  const float r2 = r1 - __bfloat162float(b1);
  b2 = __float2bfloat16_rn(r2);
}

// ---------------------------------------------------------------- descriptors
// Everything one unit of the mode-product kernel needs about its solve for
// one pass.  Lives in device memory; a launch covers one or many solves
// (a batch), each with its own sizes, tensor maps, outputs and step size.
struct alignas(128) TcPassDesc {
  CUtensorMap amap[2];      // X pieces [3][M][K] per component
  CUtensorMap bmap[2];      // Phi pieces [3][N][K] per component
  __nv_bfloat16* outp[2];   // [3][N][M] per component (kPieces3, kStage1)
  float* outf[2];           // FP32 output per component (kStage1, kAxpy)
  const float* base[2];     // FP32 base per component (kStage1, kAxpy)
  float* lo[2];             // kAxpy of a compensated state: low-order words, read and
                            // rewritten in place (null: plain FP32 update)
  const int2* kband[2];     // per component: column support [lo, hi) of each 128-row group
                            // of Phi (null: every tile runs the whole K)
  // fused two-mode pass (modes 1 and 2 in one launch): amap = Phi_a pieces,
  // bmap = W pieces (box of kFRowsW rows), cmap = Phi_b pieces, kband /
  // kband2 = the supports of Phi_a / Phi_b; slabs = n3 (1 in 2D)
  CUtensorMap cmap[2];
  const int2* kband2[2];
  int n1, n2, slabs;
  int bunit;                // fused pass: j2 tiles per unit (all of them when n2 <= 256, else 1)
  // 1: the A pieces are MN-major, [piece][K rows][M] (the mode-3 product of a
  // 3D operator after the fused pass, K = x3): two boxes of 64 M values per
  // stage, 128-byte swizzle
  int amn;
  double* ind;              // last product of a step: indicator ring [ind_k][4] (null: off)
  const int64_t* ind_ctr;   // the step's slot: *ind_ctr % ind_k
  int ind_k;
  int ind_n1, ind_n2;       // n_1 and (3D) n_2, for the trapezoid weights of row m
  int M, N, K;
  int tiles_m, tiles_n;
  int pair;                 // 1: unit = (u, v) tile pair; 0: unit = one tile of one component
  int mode;                 // TcMode
  float alpha;
  ReactionT<float> rx;
};

// Kernel parameter of one pass launch.  A launch for one solve carries its
// descriptor (tensor maps included) in the parameter itself; a grouped
// launch reads the solves' descriptors from device memory.
struct TcLaunch {
  TcPassDesc one;           // used when desc is null (one solve)
  const TcPassDesc* desc;   // [nsolves] in device memory, or null
  const int* ustart;        // [nsolves + 1] prefix sums of units (desc non-null)
  int nsolves;
  int nunits;
  int* err;
};

// Programmatic dependent launch: a kernel lets the next kernel of the step
// be scheduled early (its set-up then overlaps this kernel's tail) and
// waits for its predecessors' completion before touching the data they
// write.  Both are no-ops for launches without the programmatic attribute.
__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Stage update of a compensated state.  The state is b + lo_in (two FP32
// words); (hi, lo) receives b + lo_in + inc with hi the FP32 value nearest
// the sum and |lo| <= ulp(hi) / 2.  Knuth's TwoSum gives the exact rounding
// error of b + inc; a second TwoSum renormalises after the low-order words
// are added.  The _rn intrinsics keep the compiler from contracting or
// reordering the error terms.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void comp_update(float b, float lo_in, float inc, float& hi, float& lo) {
  float s, e;
  two_sum(b, inc, s, e);
  two_sum(s, __fadd_rn(lo_in, e), hi, lo);
}

__device__ __forceinline__ double trap_w(int i, int n) { return (i == 0 || i == n - 1) ? 0.5 : 1.0; }

// Epilogue of a kAxpy pass with its options, for one epilogue warp: lane =
// output row m, NCH chunks of 16 columns from n0; out = base + alpha acc.
//  lp  : compensated state; the low-order words are read and rewritten in
//        place and hi + lo takes the exact sum (comp_update).
//  ind : the step's indicator slot of this component: adds the
//        trapezoid-weighted sum of the new state and the squared increment
//        against the value the output buffer held (the previous state), in
//        FP64, one atomic per warp and sum.
// Per chunk the base, low-order and previous values are loaded before the
// TMEM read, so their latency overlaps it.
template <int NCH>
__device__ __forceinline__ void axpy_epilogue(uint32_t ta, float* __restrict__ of,
                                              const float* __restrict__ bsrc, float* lp,
                                              float alpha, int M, int N, int n0, int m, bool mrow,
                                              double* ind, int n1, int n2) {
  double wm = 0.0;  // trapezoid weight of row m (the directions before the last)
  if (ind && mrow) wm = n2 > 0 ? trap_w(m % n1, n1) * trap_w(m / n1, n2) : trap_w(m, n1);
  double sw = 0.0, sd = 0.0;
#pragma unroll 1
  for (int bt = 0; bt < NCH; ++bt) {
    float bb[16], lv[16], pv[16];
    uint32_t r[16];
#pragma unroll
    for (int jj = 0; jj < 16; ++jj) {
      const int col = n0 + bt * 16 + jj;
      const bool ok = mrow && col < N;
      const int64_t o = (int64_t)col * M + m;
      bb[jj] = (ok && bsrc) ? __ldg(bsrc + o) : 0.f;
      lv[jj] = (ok && lp) ? __ldcg(lp + o) : 0.f;
      pv[jj] = (ok && ind) ? __ldcg(of + o) : 0.f;
    }
    tmem_ld16_nw(ta + (uint32_t)(bt * 16), r);
    tmem_wait_ld();
    tmem_fence16(r);
#pragma unroll
    for (int jj = 0; jj < 16; ++jj) {
      const int col = n0 + bt * 16 + jj;
      if (mrow && col < N) {
        const int64_t o = (int64_t)col * M + m;
        const float a = __uint_as_float(r[jj]);
        float hi;
        if (lp) {
          float lo;
          comp_update(bb[jj], lv[jj], __fmul_rn(alpha, a), hi, lo);
          lp[o] = lo;
        } else {
          hi = __fmaf_rn(alpha, a, bb[jj]);
        }
        of[o] = hi;
        if (ind) {
          sw += wm * trap_w(col, N) * (double)hi;
          const double dd = (double)hi - (double)pv[jj];
          sd += dd * dd;
        }
      }
    }
  }
  if (ind) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      sw += __shfl_xor_sync(0xffffffffu, sw, off);
      sd += __shfl_xor_sync(0xffffffffu, sd, off);
    }
    if ((threadIdx.x & 31) == 0) {
      atomicAdd(ind, sw);
      atomicAdd(ind + 2, sd);
    }
  }
}

// The indicator slot of component c for the unit's step (null when off).
__device__ __forceinline__ double* indicator_slot(const struct TcPassDesc* D, int c);

// Epilogue of one mode-product pass.
enum TcMode : int {
  kPieces3 = 0,   // out pieces [3][N][M] of acc
  kStage1 = 1,    // pair units only: U2 = U + alpha acc_u, V2 = V + alpha acc_v
                  // (FP32 out) and D = G(U2, V2) - G(U, V) as pieces
  kAxpy = 2,      // out = base + alpha acc (FP32)
  kStage1X = 3    // as kStage1 with one component per CTA: the two CTAs of a
                  // cluster hold u and v of the same tile and exchange U2, V2
};

__device__ __forceinline__ double* indicator_slot(const TcPassDesc* D, int c) {
  if (D->ind == nullptr) return nullptr;
  const int64_t s = __ldcg(D->ind_ctr);
  return D->ind + 4 * (s % D->ind_k) + c;
}

// The six piece pairs (i, j), A piece i times B piece j, grouped by A piece
// so that each A piece is read from shared memory once per K step (A
// collector), smaller A pieces first: (2,0), (1,1), (1,0), (0,2), (0,1), (0,0).

constexpr int kEpiWarps = 8;                  // two warps per TMEM lane quarter
constexpr int kThreads = 64 + 32 * kEpiWarps;  // producer warp, MMA warp, epilogue

// Largest s with start[s] <= x (start[0] = 0, start[n] = total > x).
__device__ __forceinline__ int find_segment(const int* __restrict__ start, int n, int x) {
  int lo = 0, hi = n;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(start + mid) <= x)
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

// K-blocks [kb0, kb1) that a tile of Phi rows starting at n0 contracts over.
// The support table holds one column range per 128-row group of Phi, with
// both ends on multiples of 64 (the end clipped to K); tiles of 64 or 128
// rows (starting at multiples of their height) take their group's range.
// Every kernel variant's K-block (32 or 64 values) divides 64, so all
// variants accumulate each output over the same K values in the same order.
// Without a table, all of K.  The table is plan data, so it may be read
// before the programmatic dependency on the previous kernel is resolved.
__device__ __forceinline__ void k_blocks(const TcPassDesc* d, int c, int n0, int bk, int& kb0,
                                         int& kb1) {
  const int nk = (d->K + bk - 1) / bk;
  const int2* t = d->kband[c];
  kb0 = 0;
  kb1 = nk;
  if (t == nullptr) return;
  const int2 r = __ldg(t + (n0 >> 7));
  if (r.x < r.y) {
    kb0 = r.x / bk;
    kb1 = min(nk, (r.y + bk - 1) / bk);
  }
}

struct Unit {
  const TcPassDesc* d;
  int m0, n0, c_lo, c_hi;
};

template <int BN>
__device__ __forceinline__ Unit decode_unit(const TcLaunch& L, int u) {
  Unit w;
  int r = u;
  if (L.desc == nullptr) {
    w.d = &L.one;
  } else {
    const int s = find_segment(L.ustart, L.nsolves, u);
    w.d = L.desc + s;
    r -= __ldg(L.ustart + s);
  }
  if (w.d->pair) {
    w.c_lo = 0;
    w.c_hi = 2;
  } else if (w.d->mode == kStage1X) {  // unit 2 t + c: component c of tile t
    w.c_lo = r & 1;
    w.c_hi = w.c_lo + 1;
    r >>= 1;
  } else {
    const int per = w.d->tiles_m * w.d->tiles_n;
    w.c_lo = r / per;
    w.c_hi = w.c_lo + 1;
    r -= w.c_lo * per;
  }
  w.m0 = (r / w.d->tiles_n) * kBM;
  w.n0 = (r % w.d->tiles_n) * BN;
  return w;
}

// ---- cluster helpers (CTA rank, addresses in the other CTA, barriers)
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// Address of the same shared-memory location in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t mapa_shared(uint32_t addr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
  return r;
}
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n barrier.cluster.wait.acquire.aligned;" ::
                   : "memory");
}
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t cluster_addr) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr)
               : "memory");
}
// Arrival that orders no memory: for "these TMEM columns have been read"
// (tcgen05.wait::ld has completed the reads).  A release at cluster scope
// would first wait for every preceding global store of the thread.
__device__ __forceinline__ void mbar_arrive_cluster_relaxed(uint32_t cluster_addr) {
  asm volatile("mbarrier.arrive.relaxed.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr)
               : "memory");
}
// Persistent kernel.  CTA b handles units b, b + gridDim.x, ... of the
// launch's unit list (all solves' tiles, solve-major, n-tile fastest within
// a solve so that CTAs running together share A tiles in L2).  For each unit
// the MMA warp accumulates into one of two TMEM slots of 2 x BN columns, so
// the epilogue of one unit overlaps the MMAs of the next; pair units put u
// and v of the same tile in one slot, which the fused stage-1 epilogue needs.
// Epilogue warp w owns TMEM lane quarter w % 4 and half (w - 2) / 4 of the
// columns; it prefetches its FP32 base values two 16-column chunks ahead,
// starting before the accumulator is ready.
//
// IND instantiation: the last product of a step with the indicators of
// Sec. 4 on (a separate instantiation, so that the other launches carry none
// of its code).
//
// XCHG instantiation (launched in clusters of two, for the kStage1X pass):
// CTA 2k + c holds component c of the tile, forms U2 (or V2) in its
// epilogue, stores it, then each epilogue warp signals its counterpart in
// the other CTA through that CTA's `xready` barrier and waits for its own;
// it then reads the other component's base and stage values (L2) and writes
// its component of D = G(U2, V2) - G(U, V) as BF16 pieces.
template <int SW, int BN, bool PAIR, bool XCHG, int F = kFmtBF16, bool IND = false>
__global__ void __launch_bounds__(kThreads, 1) tc_mode_kernel(const __grid_constant__ TcLaunch L) {
  using C = TcCfg<SW, BN, F>;
  static_assert(F == kFmtBF16 || (!PAIR && !XCHG), "TF32 pieces: plain epilogues only");
  static_assert(4 * BN <= 512, "four accumulators must fit in TMEM");
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(smem + C::STAGES * C::STAGE);
  uint64_t* empty = full + C::STAGES;
  uint64_t* acc_full = empty + C::STAGES;   // [2]
  uint64_t* acc_empty = acc_full + 2;       // [2]
  uint64_t* drain = acc_empty + 2;
  uint32_t* tmem_slot = (uint32_t*)(drain + 1);
  int* abort_flag = (int*)(tmem_slot + 1);
  uint64_t* xready = drain + 3;  // [2 slots][kEpiWarps] (XCHG), after tmem_slot and abort_flag

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  pdl_trigger();

  if (threadIdx.x == 0) {
    for (int s = 0; s < C::STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], kEpiWarps);
    }
    mbar_init(drain, 1);
    if (XCHG)
      for (int b = 0; b < 2 * kEpiWarps; ++b) mbar_init(&xready[b], 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    tmem_alloc(tmem_slot, 4 * BN);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  if (XCHG) cluster_sync_all();  // the other CTA's exchange barriers are initialised
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  volatile int* abort_v = abort_flag;

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer
    uint32_t g = 0;  // k-block counter of this CTA
    bool stop = false;
    bool waited = false;
    for (int u = blockIdx.x; u < L.nunits && !stop; u += gridDim.x) {
      const Unit w = decode_unit<BN>(L, u);
      for (int comp = w.c_lo; comp < w.c_hi; ++comp) {
        asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&w.d->amap[comp]) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&w.d->bmap[comp]) : "memory");
      }
      for (int comp = w.c_lo; comp < w.c_hi && !stop; ++comp) {
        const CUtensorMap* ma = &w.d->amap[comp];
        const CUtensorMap* mb = &w.d->bmap[comp];
        int kb0, kb1;
        k_blocks(w.d, comp, w.n0, C::BK, kb0, kb1);
        for (int kb = kb0; kb < kb1; ++kb, ++g) {
          const int s = g % C::STAGES;
          const uint32_t it = g / C::STAGES;
          if (*abort_v || (it > 0 && !mbar_wait(&empty[s], (it - 1) & 1))) {
            atomicCAS(L.err, 0, kErrTimeoutEmpty);
            *abort_v = 1;
            stop = true;
            break;
          }
          uint8_t* st = smem + s * C::STAGE;
          if (!waited) {  // the A pieces are the previous launch's output
            pdl_wait();
            waited = true;
          }
          mbar_arrive_expect_tx(&full[s], C::STAGE);
          if (w.d->amn) {  // MN-major A: two boxes of 64 M values
            tma_load_3d(st, ma, &full[s], w.m0, kb * C::BK, 0);
            tma_load_3d(st + kPieces * C::BK * 128, ma, &full[s], w.m0 + 64, kb * C::BK, 0);
          } else {
            tma_load_3d(st, ma, &full[s], kb * C::BK, w.m0, 0);                 // 3 A pieces
          }
          tma_load_3d(st + C::P * C::TILE_A, mb, &full[s], kb * C::BK, w.n0, 0);  // B pieces
        }
      }
    }
    // drain: the last STAGES issued loads must have landed before exit
    const uint32_t first = g > (uint32_t)C::STAGES ? g - C::STAGES : 0;
    for (uint32_t q = first; q < g; ++q) mbar_wait(&full[q % C::STAGES], (q / C::STAGES) & 1);
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer
    const uint32_t idesc = F == kFmtTF32 ? idesc_tf32(kBM, BN) : idesc_bf16(kBM, BN);
    const uint64_t dA0 = kmajor_desc<SW>(smem_u32(smem));  // stage 0, A piece 0
    uint32_t g = 0;
    int i = 0;  // local unit counter
    bool stop = false;
    for (int u = blockIdx.x; u < L.nunits && !stop; u += gridDim.x, ++i) {
      const int slot = i & 1;
      const uint32_t use = i >> 1;
      if (use > 0 && !mbar_wait(&acc_empty[slot], (use - 1) & 1)) {
        atomicCAS(L.err, 0, kErrTimeoutDone);
        *abort_v = 1;
        break;
      }
      tc_fence_after();
      const Unit w = decode_unit<BN>(L, u);
      for (int comp = w.c_lo; comp < w.c_hi && !stop; ++comp) {
        const uint32_t dt = tmem + (uint32_t)((slot * 2 + comp - w.c_lo) * BN);
        int kb0, kb1;
        k_blocks(w.d, comp, w.n0, C::BK, kb0, kb1);
        for (int kb = kb0; kb < kb1; ++kb, ++g) {
          const int s = g % C::STAGES;
          if (!mbar_wait(&full[s], (g / C::STAGES) & 1)) {
            atomicCAS(L.err, 0, kErrTimeoutFull);
            *abort_v = 1;
            stop = true;
            break;
          }
          // (TMA -> MMA hand-off through the mbarrier needs no tcgen05 fence)
          const uint64_t db = dA0 + (uint64_t)((s * C::STAGE + C::P * C::TILE_A) >> 4);
          uint64_t da = dA0 + (uint64_t)((s * C::STAGE) >> 4);
          uint32_t apiece = C::TILE_A >> 4, akstep = 2, idk = idesc;
          if (F == kFmtBF16 && w.d->amn) {
            const AOperand ao = a_operand<SW>(smem_u32(smem) + s * C::STAGE, true);
            da = ao.d;
            apiece = ao.piece;
            akstep = ao.kstep;
            idk |= 1u << 15;  // A is MN-major
          }
#pragma unroll
          for (int kk = 0; kk < C::KSTEPS; ++kk) {
            const uint64_t a0 = da + (uint64_t)(kk * akstep);
            const uint64_t a1 = a0 + (uint64_t)apiece;
            const uint64_t b0 = db + (uint64_t)(kk * 2);
            const uint64_t b1 = b0 + (uint64_t)(C::TILE_B >> 4);
            if constexpr (F == kFmtTF32) {
              // (lo, hi), (hi, lo), (hi, hi): the lo x lo term (2^-22) is dropped
              mma_tf32<kColNone>(dt, a1, b0, idesc, (kb != kb0 || kk != 0));
              mma_tf32<kColFill>(dt, a0, b1, idesc, 1);
              mma_tf32<kColLast>(dt, a0, b0, idesc, 1);
            } else {
              const uint64_t a2 = a0 + (uint64_t)(2 * apiece);
              const uint64_t b2 = b0 + (uint64_t)(2 * C::TILE_B >> 4);
              mma_bf16<kColNone>(dt, a2, b0, idk, (kb != kb0 || kk != 0));
              mma_bf16<kColFill>(dt, a1, b1, idk, 1);
              mma_bf16<kColLast>(dt, a1, b0, idk, 1);
              mma_bf16<kColFill>(dt, a0, b2, idk, 1);
              mma_bf16<kColUse>(dt, a0, b1, idk, 1);
              mma_bf16<kColLast>(dt, a0, b0, idk, 1);
            }
          }
          mma_commit(&empty[s]);  // frees the stage once these MMAs have read it
        }
      }
      if (stop) break;
      mma_commit(&acc_full[slot]);  // the accumulators of this slot are complete
    }
    // every MMA this thread issued has completed once `drain` fires
    mma_commit(drain);
    mbar_wait(drain, 0);
  } else if (warp >= 2) {
    // ---------------- epilogue
    pdl_wait();
    const int q = warp & 3;                   // TMEM lane quarter
    const int half = (warp - 2) >> 2;         // column half
    constexpr int HC = BN / 2;                // columns per epilogue warp
    constexpr int NCH = HC / 16;              // 16-column chunks
    int i = 0;
    for (int u = blockIdx.x; u < L.nunits; u += gridDim.x, ++i) {
      const int slot = i & 1;
      const Unit w = decode_unit<BN>(L, u);
      const TcPassDesc* D = w.d;
      const int M = D->M, N = D->N, mode = D->mode;
      const float alpha = D->alpha;
      const bool fp32_in = mode != kPieces3;
      const int nc = w.c_hi - w.c_lo;
      const int n0 = w.n0 + half * HC;
      const int m = w.m0 + q * 32 + lane;
      const bool mrow = m < M;
      const int64_t plane = (int64_t)N * M;
      const float* bsrc0 = D->base[w.c_lo];
      const float* bsrc1 = nc == 2 ? D->base[w.c_lo + 1] : nullptr;
      auto chunk_cols = [&](int ch) { return min(16, N - (n0 + ch * 16)); };
      if constexpr (XCHG) {
        // kStage1X: this CTA's component c; the other CTA of the cluster has 1 - c
        const int c = w.c_lo;
        float bv[HC];  // own base U^c
        const float* bsrc = D->base[c];
#pragma unroll
        for (int j = 0; j < HC; ++j) {
          const int col = n0 + j;
          bv[j] = (mrow && col < N) ? __ldg(bsrc + (int64_t)col * M + m) : 0.f;
        }
        if (!mbar_wait_sleep(&acc_full[slot], (i >> 1) & 1)) {
          if (lane == 0) atomicCAS(L.err, 0, kErrTimeoutDone);
          *abort_v = 1;
          break;
        }
        tc_fence_after();
        if (*abort_v) break;
        const uint32_t ta = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(slot * 2 * BN + half * HC);
        float* of = D->outf[c];
#pragma unroll
        for (int bt = 0; bt < NCH; bt += 2) {  // U2^c = U^c + alpha acc, stored
          uint32_t r[2][16];
          tmem_ld16_nw(ta + (uint32_t)(bt * 16), r[0]);
          tmem_ld16_nw(ta + (uint32_t)((bt + 1) * 16), r[1]);
          tmem_wait_ld();
          tmem_fence16(r[0]);
          tmem_fence16(r[1]);
#pragma unroll
          for (int jj = 0; jj < 32; ++jj) {
            const int col = n0 + bt * 16 + jj;
            if (mrow && col < N)
              of[(int64_t)col * M + m] = __fmaf_rn(alpha, __uint_as_float(r[jj / 16][jj % 16]), bv[bt * 16 + jj]);
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0)  // the accumulator slot is free again
          asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acc_empty[slot]))
                       : "memory");
        // publish U2^c to the other CTA's counterpart warp, wait for its U2^(1-c)
        __threadfence();
        __syncwarp();
        uint64_t* mine = &xready[slot * kEpiWarps + (warp - 2)];
        if (lane == 0) mbar_arrive_cluster(mapa_shared(smem_u32(mine), cluster_rank() ^ 1u));
        if (!mbar_wait_cluster(mine, (i >> 1) & 1)) {
          if (lane == 0) atomicCAS(L.err, 0, kErrTimeoutDone);
          *abort_v = 1;
          break;
        }
        __syncwarp();
        // D^c = g^c(U2, V2) - g^c(U, V) as pieces
        const float* ob = D->base[1 - c];
        const float* os = D->outf[1 - c];
        __nv_bfloat16* op = D->outp[c];
        const ReactionT<float> rx = D->rx;
        constexpr int XC = 8;  // columns per exchange chunk (register budget)
#pragma unroll 1
        for (int ch = 0; ch < HC / XC; ++ch) {
          float x2[XC], yb[XC], y2[XC];
#pragma unroll
          for (int j = 0; j < XC; ++j) {
            const int col = n0 + ch * XC + j;
            const bool ok = mrow && col < N;
            const int64_t o = (int64_t)col * M + m;
            x2[j] = ok ? __ldcg(of + o) : 0.f;
            yb[j] = ok ? __ldcg(ob + o) : 0.f;
            y2[j] = ok ? __ldcg(os + o) : 0.f;
          }
#pragma unroll
          for (int j = 0; j < XC; ++j) {
            const int col = n0 + ch * XC + j;
            if (mrow && col < N) {
              float xb = 0.f;
#pragma unroll
              for (int t = 0; t < HC / XC; ++t)
                if (t == ch) xb = bv[t * XC + j];  // register-indexed select
              const float u0 = c == 0 ? xb : yb[j], v0 = c == 0 ? yb[j] : xb;
              const float u2 = c == 0 ? x2[j] : y2[j], v2 = c == 0 ? y2[j] : x2[j];
              float du, dv;
              react_diff<float>(rx, u0, v0, u2, v2, du, dv);
              const int64_t o = (int64_t)col * M + m;
              __nv_bfloat16 b0, b1, b2;
              split3(c == 0 ? du : dv, b0, b1, b2);
              op[o] = b0;
              op[plane + o] = b1;
              op[2 * plane + o] = b2;
            }
          }
        }
      } else if constexpr (!PAIR) {
        // One component: load this warp's whole FP32 base strip (HC columns)
        // before the accumulator is ready, read all its TMEM columns with one
        // wait, then write.
        float bv[HC];
        const float* bsrc = D->base[w.c_lo];
        float* lp = mode == kAxpy ? D->lo[w.c_lo] : nullptr;  // compensated state update
        double* ind = (IND && mode == kAxpy) ? indicator_slot(D, w.c_lo) : nullptr;
#pragma unroll
        for (int j = 0; j < HC; ++j) {
          const int col = n0 + j;
          bv[j] = (fp32_in && !lp && !ind && bsrc && mrow && col < N)
                      ? __ldg(bsrc + (int64_t)col * M + m) : 0.f;
        }
        if (!mbar_wait_sleep(&acc_full[slot], (i >> 1) & 1)) {
          if (lane == 0) atomicCAS(L.err, 0, kErrTimeoutDone);
          *abort_v = 1;
          break;
        }
        tc_fence_after();
        if (*abort_v) break;
        const uint32_t ta = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(slot * 2 * BN + half * HC);
        // TMEM columns in batches of two 16-column chunks, one wait per batch
        if (lp || ind) {
          axpy_epilogue<NCH>(ta, D->outf[w.c_lo], bsrc, lp, alpha, M, N, n0, m, mrow, ind,
                             D->ind_n1, D->ind_n2);
        } else {
#pragma unroll
        for (int bt = 0; bt < NCH; bt += 2) {
          constexpr int NB = NCH >= 2 ? 2 : 1;
          uint32_t r[NB][16];
#pragma unroll
          for (int c = 0; c < NB; ++c) tmem_ld16_nw(ta + (uint32_t)((bt + c) * 16), r[c]);
          tmem_wait_ld();
#pragma unroll
          for (int c = 0; c < NB; ++c) tmem_fence16(r[c]);
          if (mrow) {
            if (mode == kPieces3 && F == kFmtTF32) {  // two TF32 pieces, FP32 words
              float* op = reinterpret_cast<float*>(D->outp[w.c_lo]);
#pragma unroll
              for (int jj = 0; jj < 16 * NB; ++jj) {
                const int col = n0 + bt * 16 + jj;
                if (col < N) {
                  const int64_t o = (int64_t)col * M + m;
                  float hi, lo;
                  split2_tf32(__uint_as_float(r[jj / 16][jj % 16]), hi, lo);
                  op[o] = hi;
                  op[plane + o] = lo;
                }
              }
            } else if (mode == kPieces3) {
              __nv_bfloat16* op = D->outp[w.c_lo];
#pragma unroll
              for (int jj = 0; jj < 16 * NB; ++jj) {
                const int col = n0 + bt * 16 + jj;
                if (col < N) {
                  const int64_t o = (int64_t)col * M + m;
                  __nv_bfloat16 b0, b1, b2;
                  split3(__uint_as_float(r[jj / 16][jj % 16]), b0, b1, b2);
                  op[o] = b0;
                  op[plane + o] = b1;
                  op[2 * plane + o] = b2;
                }
              }
            } else {
              float* of = D->outf[w.c_lo];
#pragma unroll
              for (int jj = 0; jj < 16 * NB; ++jj) {
                const int col = n0 + bt * 16 + jj;
                if (col < N)
                  of[(int64_t)col * M + m] = __fmaf_rn(alpha, __uint_as_float(r[jj / 16][jj % 16]), bv[bt * 16 + jj]);
              }
            }
          }
        }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0)
          asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acc_empty[slot]))
                       : "memory");
      } else {
      // base prefetch, two chunks deep: pb[buffer][component slot][column]
      float pb[2][2][16];
      auto prefetch = [&](int ch, int buf) {
        const int jm = chunk_cols(ch);
        const int64_t o0 = (int64_t)(n0 + ch * 16) * M + m;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const bool ok = mrow && j < jm;
          pb[buf][0][j] = (ok && bsrc0) ? __ldg(bsrc0 + o0 + (int64_t)j * M) : 0.f;
          pb[buf][1][j] = (ok && bsrc1) ? __ldg(bsrc1 + o0 + (int64_t)j * M) : 0.f;
        }
      };
      if (fp32_in) {
        prefetch(0, 0);
        if (NCH > 1) prefetch(1, 1);
      }
      if (!mbar_wait_sleep(&acc_full[slot], (i >> 1) & 1)) {
        if (lane == 0) atomicCAS(L.err, 0, kErrTimeoutDone);
        *abort_v = 1;
        break;
      }
      tc_fence_after();
      if (*abort_v) break;
      const uint32_t ta = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(slot * 2 * BN + half * HC);
#pragma unroll
      for (int ch = 0; ch < NCH; ++ch) {
        float acc[2][16];
        tmem_ld16(ta + (uint32_t)(ch * 16), acc[0]);
        if (nc == 2) tmem_ld16(ta + (uint32_t)(BN + ch * 16), acc[1]);
        const int jm = chunk_cols(ch);
        const int64_t o0 = (int64_t)(n0 + ch * 16) * M + m;
        const int buf = ch & 1;
        if (mrow && jm > 0) {
          if (mode == kStage1) {
            __nv_bfloat16* op0 = D->outp[0];
            __nv_bfloat16* op1 = D->outp[1];
            float* of0 = D->outf[0];
            float* of1 = D->outf[1];
            const ReactionT<float> rx = D->rx;
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              if (j >= jm) break;
              const int64_t o = o0 + (int64_t)j * M;
              const float u0 = pb[buf][0][j], v0 = pb[buf][1][j];
              const float u2 = u0 + alpha * acc[0][j];
              const float v2 = v0 + alpha * acc[1][j];
              of0[o] = u2;
              of1[o] = v2;
              float du, dv;
              react_diff<float>(rx, u0, v0, u2, v2, du, dv);
              __nv_bfloat16 b0, b1, b2;
              split3(du, b0, b1, b2);
              op0[o] = b0;
              op0[plane + o] = b1;
              op0[2 * plane + o] = b2;
              split3(dv, b0, b1, b2);
              op1[o] = b0;
              op1[plane + o] = b1;
              op1[2 * plane + o] = b2;
            }
          } else {
            auto emit = [&](int c, const float(&a)[16], const float(&bsv)[16]) {
              if (mode == kPieces3) {
                __nv_bfloat16* op = D->outp[w.c_lo + c];
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                  if (j >= jm) break;
                  const int64_t o = o0 + (int64_t)j * M;
                  __nv_bfloat16 b0, b1, b2;
                  split3(a[j], b0, b1, b2);
                  op[o] = b0;
                  op[plane + o] = b1;
                  op[2 * plane + o] = b2;
                }
              } else {
                float* of = D->outf[w.c_lo + c];
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                  if (j >= jm) break;
                  of[o0 + (int64_t)j * M] = __fmaf_rn(alpha, a[j], bsv[j]);
                }
              }
            };
            emit(0, acc[0], pb[buf][0]);
            if (nc == 2) emit(1, acc[1], pb[buf][1]);
          }
        }
        if (fp32_in && ch + 2 < NCH) prefetch(ch + 2, buf);
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0)
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acc_empty[slot]))
                     : "memory");
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (XCHG) cluster_sync_all();  // no exchange arrival can still target this CTA
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, 4 * BN);
  }
}

// ---------------------------------------------------------------- CTA-pair kernel
// The same mode product with 2-SM tensor-core instructions (cta_group::2): a
// cluster of two CTAs computes a 256 x BN tile as one M = 256 MMA.  Each CTA
// stages its own 128 rows of A and half (BN / 2 rows) of B; the MMA, issued
// by the even CTA, reads both CTAs' shared memory and writes each CTA's 128
// accumulator rows into that CTA's TMEM.  Per SM this halves the B traffic
// (TMA and shared-memory reads) of the one-CTA kernel.
//
// Synchronisation: both CTAs' TMA loads complete on the even CTA's `full`
// barrier (which expects both CTAs' bytes); the MMA commits arrive on the
// `empty` and `acc_full` barriers of both CTAs (multicast); both CTAs'
// epilogue warps arrive on the even CTA's `acc_empty`.
template <int SW>
struct Tc2Cfg {
  static constexpr int BN = 128;                     // output columns per tile
  static constexpr int BK = SW / 2;
  static constexpr int KSTEPS = SW / 32;
  static constexpr int TILE_A = kBM * SW;            // this CTA's 128 A rows
  static constexpr int TILE_B = (BN / 2) * SW;       // this CTA's half of the B rows
  static constexpr int STAGE = kPieces * (TILE_A + TILE_B);
  static constexpr int STAGES = (216 * 1024) / STAGE > 8 ? 8 : (216 * 1024) / STAGE;
  static constexpr int SMEM = STAGES * STAGE + 1024 + 256;
};

__device__ __forceinline__ void tma_load_3d_pair(void* dst, const CUtensorMap* map, uint32_t bar,
                                                 int x, int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes.cta_group::2"
      " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(smem_u32(dst)),
      "l"((uint64_t)map), "r"(bar), "r"(x), "r"(y), "r"(z)
      : "memory");
}
__device__ __forceinline__ void tmem_alloc_pair(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   smem_u32(dst)),
               "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish_pair() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc_pair(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}
template <int COL>
__device__ __forceinline__ void mma_bf16_pair(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                              uint32_t acc) {
  if constexpr (COL == kColFill) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::2.kind::f16.collector::a::fill [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
  } else if constexpr (COL == kColUse) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::2.kind::f16.collector::a::use [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
  } else if constexpr (COL == kColLast) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::2.kind::f16.collector::a::lastuse [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
  } else {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
  }
}
// Arrive on the barrier at this offset in every CTA of `mask` once the
// preceding pair MMAs of this thread have completed.
__device__ __forceinline__ void mma_commit_pair(uint64_t* bar, uint16_t mask) {
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64"
      " [%0], %1;" ::"r"(smem_u32(bar)),
      "h"(mask)
      : "memory");
}

// One stage of the split-precision product: KSTEPS K16 steps, six MMAs each,
// grouped by A piece for the A collector.  da / db are the descriptors of
// piece 0 of the stage's A and B tiles; pieces and K steps are fixed offsets
// of the descriptor's address field (16-byte units), so the issue loop adds
// immediates only.  acc0 = 0 starts a new accumulation.
template <int SW, int TILE_A, int TILE_B, bool CTA2>
__device__ __forceinline__ void issue_stage(uint32_t dt, uint64_t da, uint64_t db, uint32_t idesc,
                                            uint32_t acc0, uint32_t apiece = TILE_A >> 4,
                                            uint32_t akstep = 2) {
#pragma unroll
  for (int kk = 0; kk < SW / 32; ++kk) {
    const uint64_t a0 = da + (uint64_t)(kk * akstep);
    const uint64_t a1 = a0 + (uint64_t)apiece;
    const uint64_t a2 = a0 + (uint64_t)(2 * apiece);
    const uint64_t b0 = db + (uint64_t)(kk * 2);
    const uint64_t b1 = b0 + (uint64_t)(TILE_B >> 4);
    const uint64_t b2 = b0 + (uint64_t)(2 * TILE_B >> 4);
    if constexpr (CTA2) {
      mma_bf16_pair<kColNone>(dt, a2, b0, idesc, kk == 0 ? acc0 : 1u);
      mma_bf16_pair<kColFill>(dt, a1, b1, idesc, 1);
      mma_bf16_pair<kColLast>(dt, a1, b0, idesc, 1);
      mma_bf16_pair<kColFill>(dt, a0, b2, idesc, 1);
      mma_bf16_pair<kColUse>(dt, a0, b1, idesc, 1);
      mma_bf16_pair<kColLast>(dt, a0, b0, idesc, 1);
    } else {
      mma_bf16<kColNone>(dt, a2, b0, idesc, kk == 0 ? acc0 : 1u);
      mma_bf16<kColFill>(dt, a1, b1, idesc, 1);
      mma_bf16<kColLast>(dt, a1, b0, idesc, 1);
      mma_bf16<kColFill>(dt, a0, b2, idesc, 1);
      mma_bf16<kColUse>(dt, a0, b1, idesc, 1);
      mma_bf16<kColLast>(dt, a0, b0, idesc, 1);
    }
  }
}

// Unit of the pair kernel: one component's 256 x BN tile.
struct Unit2 {
  const TcPassDesc* d;
  int m0, n0, c;
};
__device__ __forceinline__ Unit2 decode_unit2(const TcLaunch& L, int u, int bn) {
  Unit2 w;
  int r = u;
  if (L.desc == nullptr) {
    w.d = &L.one;
  } else {
    const int s = find_segment(L.ustart, L.nsolves, u);
    w.d = L.desc + s;
    r -= __ldg(L.ustart + s);
  }
  const int per = w.d->tiles_m * w.d->tiles_n;  // tiles_m counts 256-row tiles
  w.c = r / per;
  r -= w.c * per;
  w.m0 = (r / w.d->tiles_n) * (2 * kBM);
  w.n0 = (r % w.d->tiles_n) * bn;
  return w;
}

template <int SW, bool IND = false>
__global__ void __launch_bounds__(kThreads, 1) tc_pair_kernel(const __grid_constant__ TcLaunch L) {
  using C = Tc2Cfg<SW>;
  constexpr int BN = C::BN;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(smem + C::STAGES * C::STAGE);
  uint64_t* empty = full + C::STAGES;
  uint64_t* acc_full = empty + C::STAGES;   // [2]
  uint64_t* acc_empty = acc_full + 2;       // [2]; used in the even CTA
  uint64_t* drain = acc_empty + 2;
  uint32_t* tmem_slot = (uint32_t*)(drain + 1);
  int* abort_flag = (int*)(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = cluster_rank();     // 0: issues the MMAs
  const int cid = (int)(blockIdx.x >> 1), ncl = (int)(gridDim.x >> 1);
  pdl_trigger();

  if (threadIdx.x == 0) {
    for (int s = 0; s < C::STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], 2 * kEpiWarps);
    }
    mbar_init(drain, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    tmem_alloc_pair(tmem_slot, 2 * BN);
    tmem_relinquish_pair();
  }
  tc_fence_before();
  cluster_sync_all();  // barriers initialised and TMEM allocated in both CTAs
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  volatile int* abort_v = abort_flag;

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer (both CTAs)
    uint32_t g = 0;
    bool stop = false, waited = false;
    for (int u = cid; u < L.nunits && !stop; u += ncl) {
      const Unit2 w = decode_unit2(L, u, BN);
      const CUtensorMap* ma = &w.d->amap[w.c];
      const CUtensorMap* mb = &w.d->bmap[w.c];
      asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)ma) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)mb) : "memory");
      const int ya = w.m0 + (int)rank * kBM, yb = w.n0 + (int)rank * (BN / 2);
      int kb0, kb1;  // the same range in both CTAs: the whole tile's BN rows
      k_blocks(w.d, w.c, w.n0, C::BK, kb0, kb1);
      for (int kb = kb0; kb < kb1; ++kb, ++g) {
        const int s = g % C::STAGES;
        const uint32_t it = g / C::STAGES;
        if (*abort_v || (it > 0 && !mbar_wait(&empty[s], (it - 1) & 1))) {
          atomicCAS(L.err, 0, kErrTimeoutEmpty);
          *abort_v = 1;
          stop = true;
          break;
        }
        if (!waited) {  // the A pieces are the previous launch's output
          pdl_wait();
          waited = true;
        }
        if (rank == 0) mbar_arrive_expect_tx(&full[s], 2 * C::STAGE);
        const uint32_t fb = mapa_shared(smem_u32(&full[s]), 0);
        uint8_t* st = smem + s * C::STAGE;
        if (w.d->amn) {  // MN-major A: two boxes of 64 M values
          tma_load_3d_pair(st, ma, fb, ya, kb * C::BK, 0);
          tma_load_3d_pair(st + kPieces * C::BK * 128, ma, fb, ya + 64, kb * C::BK, 0);
        } else {
          tma_load_3d_pair(st, ma, fb, kb * C::BK, ya, 0);                      // 3 A pieces
        }
        tma_load_3d_pair(st + kPieces * C::TILE_A, mb, fb, kb * C::BK, yb, 0);  // 3 B pieces
      }
    }
    if (rank == 0) {
      // the last STAGES k-blocks (both CTAs' bytes) must have landed before exit
      const uint32_t first = g > (uint32_t)C::STAGES ? g - C::STAGES : 0;
      for (uint32_t q = first; q < g; ++q) mbar_wait(&full[q % C::STAGES], (q / C::STAGES) & 1);
    } else if (stop) {
      // loads of this CTA still in flight complete on the even CTA's barrier;
      // give them time to land before the exit rendezvous
      const uint64_t t0 = globaltimer();
      while (globaltimer() - t0 < 50000ull) {
      }
    }
  } else if (warp == 1 && lane == 0 && rank == 0) {
    // ---------------- MMA issuer (even CTA)
    const uint32_t idesc = idesc_bf16(2 * kBM, BN);
    const uint64_t dA0 = kmajor_desc<SW>(smem_u32(smem));
    uint32_t g = 0;
    int i = 0;
    bool stop = false;
    for (int u = cid; u < L.nunits && !stop; u += ncl, ++i) {
      const int slot = i & 1;
      const uint32_t use = i >> 1;
      if (use > 0 && !mbar_wait(&acc_empty[slot], (use - 1) & 1)) {
        atomicCAS(L.err, 0, kErrTimeoutDone);
        *abort_v = 1;
        break;
      }
      tc_fence_after();
      const Unit2 w = decode_unit2(L, u, BN);
      const uint32_t dt = tmem + (uint32_t)(slot * BN);
      int kb0, kb1;
      k_blocks(w.d, w.c, w.n0, C::BK, kb0, kb1);
      for (int kb = kb0; kb < kb1; ++kb, ++g) {
        const int s = g % C::STAGES;
        if (!mbar_wait(&full[s], (g / C::STAGES) & 1)) {
          atomicCAS(L.err, 0, kErrTimeoutFull);
          *abort_v = 1;
          stop = true;
          break;
        }
        const uint64_t db = dA0 + (uint64_t)((s * C::STAGE + kPieces * C::TILE_A) >> 4);
        if (w.d->amn) {
          const AOperand ao = a_operand<SW>(smem_u32(smem) + s * C::STAGE, true);
          issue_stage<SW, C::TILE_A, C::TILE_B, true>(dt, ao.d, db, idesc | (1u << 15), kb != kb0,
                                                      ao.piece, ao.kstep);
        } else {
          const uint64_t da = dA0 + (uint64_t)((s * C::STAGE) >> 4);
          issue_stage<SW, C::TILE_A, C::TILE_B, true>(dt, da, db, idesc, kb != kb0);
        }
        mma_commit_pair(&empty[s], 0x3);  // frees stage s in both CTAs
      }
      if (stop) break;
      mma_commit_pair(&acc_full[slot], 0x3);
    }
    mma_commit_pair(drain, 0x1);
    mbar_wait(drain, 0);
  } else if (warp >= 2) {
    // ---------------- epilogue (both CTAs)
    pdl_wait();
    const int q = warp & 3;
    const int half = (warp - 2) >> 2;
    constexpr int HC = BN / 2;
    constexpr int NCH = HC / 16;
    const uint32_t ae0 = mapa_shared(smem_u32(&acc_empty[0]), 0);
    const uint32_t ae1 = mapa_shared(smem_u32(&acc_empty[1]), 0);
    int i = 0;
    for (int u = cid; u < L.nunits; u += ncl, ++i) {
      const int slot = i & 1;
      const Unit2 w = decode_unit2(L, u, BN);
      const TcPassDesc* D = w.d;
      const int M = D->M, N = D->N, mode = D->mode;
      const float alpha = D->alpha;
      const bool fp32_in = mode != kPieces3;
      const int n0 = w.n0 + half * HC;
      const int m = w.m0 + (int)rank * kBM + q * 32 + lane;
      const bool mrow = m < M;
      const int64_t plane = (int64_t)N * M;
      float bv[HC];
      const float* bsrc = D->base[w.c];
      float* lp = mode == kAxpy ? D->lo[w.c] : nullptr;  // compensated state update
      double* ind = (IND && mode == kAxpy) ? indicator_slot(D, w.c) : nullptr;
#pragma unroll
      for (int j = 0; j < HC; ++j) {
        const int col = n0 + j;
        bv[j] = (fp32_in && !lp && !ind && bsrc && mrow && col < N)
                    ? __ldg(bsrc + (int64_t)col * M + m) : 0.f;
      }
      if (!mbar_wait_sleep(&acc_full[slot], (i >> 1) & 1)) {
        if (lane == 0) atomicCAS(L.err, 0, kErrTimeoutDone);
        *abort_v = 1;
        break;
      }
      tc_fence_after();
      if (*abort_v) break;
      const uint32_t ta = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(slot * BN + half * HC);
      if (lp || ind) {
        axpy_epilogue<NCH>(ta, D->outf[w.c], bsrc, lp, alpha, M, N, n0, m, mrow, ind, D->ind_n1,
                           D->ind_n2);
      } else {
#pragma unroll
      for (int bt = 0; bt < NCH; bt += 2) {
        uint32_t r[2][16];
        tmem_ld16_nw(ta + (uint32_t)(bt * 16), r[0]);
        tmem_ld16_nw(ta + (uint32_t)((bt + 1) * 16), r[1]);
        tmem_wait_ld();
        tmem_fence16(r[0]);
        tmem_fence16(r[1]);
        if (mrow) {
          if (mode == kPieces3) {
            __nv_bfloat16* op = D->outp[w.c];
#pragma unroll
            for (int jj = 0; jj < 32; ++jj) {
              const int col = n0 + bt * 16 + jj;
              if (col < N) {
                const int64_t o = (int64_t)col * M + m;
                __nv_bfloat16 b0, b1, b2;
                split3(__uint_as_float(r[jj / 16][jj % 16]), b0, b1, b2);
                op[o] = b0;
                op[plane + o] = b1;
                op[2 * plane + o] = b2;
              }
            }
          } else {
            float* of = D->outf[w.c];
#pragma unroll
            for (int jj = 0; jj < 32; ++jj) {
              const int col = n0 + bt * 16 + jj;
              if (col < N)
                of[(int64_t)col * M + m] = __fmaf_rn(alpha, __uint_as_float(r[jj / 16][jj % 16]), bv[bt * 16 + jj]);
            }
          }
        }
      }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive_cluster_relaxed(slot ? ae1 : ae0);
    }
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync_all();  // neither CTA's shared memory or TMEM is in use any more
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc_pair(tmem, 2 * BN);
  }
}

// ---------------------------------------------------------------- fused two-mode kernel
// T = W x_1 Phi_a x_2 Phi_b, the first two factors of the Tucker operator of
// Eq. 5, in one launch without storing the intermediate.  A unit is one
// component and one x3 slab (the whole field in 2D), one 128-row tile a of
// output rows j1 of Phi_a, and the 128-row tiles of output rows j2 of Phi_b
// in [b0, b0 + nb): all of them when n2 <= 256 (the tiles then share one
// intermediate), else one.
//   MMA1  D1[j1][i2] = sum_{i1} Phi_a[j1][i1] W[i2][i1] for the i2 of the
//         union of the tiles' Phi_b column supports, in groups of up to 256
//         i2 (the D1 columns), over the K-blocks of the Phi_a rows' support;
//   split the epilogue warps read D1 back 64 i2 (a chunk) at a time and
//         store its three BF16 pieces into TMEM;
//   MMA2  per tile: D2[j1][j2] += sum_{i2} P[j1][i2] Phi_b[j2][i2] over the
//         chunks in the tile's support, the pieces P read as the A operand
//         from TMEM and Phi_b's pieces from shared memory;
//   out   per tile: D2 -> T in the natural layout (x1 contiguous), with the
//         epilogue of the operator's last product, or as pieces.
// Both products take the six piece products of the split form.  With one
// j2 tile per unit MMA1 covers up to 256 i2 for 128 output rows: about twice
// the products of a separate first pass, in exchange for the intermediate's
// round trip through memory and a launch.
//
// Shared memory: a ring of kFStages stages; an MMA1 stage holds one K-block
// (32 values) of Phi_a's 128 rows and of W's kFRowsW rows, an MMA2 stage two
// K-blocks of Phi_b's 128 rows.  TMEM (512 columns): D2 [0, 128), D1
// [128, 384), 128 spare columns [384, 512).  The pieces of all chunks of a
// group coexist (slot_col): each epilogue warp writes only into its half of
// the spare columns and into D1 columns of its own half that it has read.
constexpr int kFBK = 32;                               // K values per K-block (64-byte rows)
constexpr int kFRowsW = 256;                           // W rows per MMA1 stage (D1 columns)
constexpr int kFTileA = kBM * 64;                      // one piece of Phi_a's block: 8 KB
constexpr int kFTileW = kFRowsW * 64;                  // one piece of W's block: 16 KB
constexpr int kFTileC = kBM * 64;                      // one piece of a Phi_b block: 8 KB
constexpr int kFStage = kPieces * (kFTileA + kFTileW);  // 72 KB
constexpr int kFStages = 3;
constexpr int kFSmem = kFStages * kFStage + 1024 + 256;
constexpr uint32_t kFColD2 = 0, kFColD1 = 128, kFColS = 384;
// TMEM column of the 16-column slot holding piece p of chunk ch for the
// epilogue warps of column half h: the 32 i2 values [64 ch + 32 h, +32) of
// the group, two per column, lower i2 in the low half.  The warp's k-th slot
// (k = 3 ch + p): k < 4 its half of the spare columns, then the D1 columns
// of its own half of chunks 0, 1, 2, 3 (32 each), so that chunk ch's pieces
// land only in columns of chunks <= ch that this warp has already read.
__device__ __forceinline__ uint32_t slot_col(int ch, int p, int h) {
  const int k = 3 * ch + p;
  if (k < 4) return kFColS + 64u * h + 16u * k;
  const int r = k - 4;
  return kFColD1 + 64u * (r >> 1) + 32u * h + 16u * (r & 1);
}
// Three BF16 pieces of two FP32 values, each level rounded to nearest (the
// same pieces as split3), packed two per 32-bit word with x0 in the low half.
__device__ __forceinline__ void split3_pair(float x0, float x1, uint32_t& w0, uint32_t& w1,
                                            uint32_t& w2) {
  const __nv_bfloat162 h0 = __floats2bfloat162_rn(x0, x1);
  const float2 f0 = __bfloat1622float2(h0);
  const float r0 = x0 - f0.x, r1 = x1 - f0.y;
  const __nv_bfloat162 h1 = __floats2bfloat162_rn(r0, r1);
  const float2 f1 = __bfloat1622float2(h1);
  const __nv_bfloat162 h2 = __floats2bfloat162_rn(r0 - f1.x, r1 - f1.y);
  w0 = *reinterpret_cast<const uint32_t*>(&h0);
  w1 = *reinterpret_cast<const uint32_t*>(&h1);
  w2 = *reinterpret_cast<const uint32_t*>(&h2);
}
static_assert(2 * kPieces * kFTileC <= kFStage, "an MMA2 stage fits in a ring slot");
static_assert(kFSmem <= 227 * 1024, "shared memory per CTA");

// MMA with the A operand in TMEM (kind::f16, BF16 pieces, FP32 accumulate).
__device__ __forceinline__ void mma_bf16_ts(uint32_t d, uint32_t a, uint64_t b, uint32_t idesc,
                                            uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d),
      "r"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
// 32 lanes x 32 bit, 16 consecutive columns per thread.
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15, %16};" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
      "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
      : "memory");
}
__device__ __forceinline__ void tmem_wait_st() {
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// Unit of the fused kernel: component c, slab s, j1 tile a, j2 tiles
// [b0, b0 + nb).
struct UnitF {
  const TcPassDesc* d;
  int c, s, a, b0, nb;
};
__device__ __forceinline__ UnitF decode_unitf(const TcLaunch& L, int u) {
  UnitF w;
  int r = u;
  if (L.desc == nullptr) {
    w.d = &L.one;
  } else {
    const int sv = find_segment(L.ustart, L.nsolves, u);
    w.d = L.desc + sv;
    r -= __ldg(L.ustart + sv);
  }
  const int nbg = w.d->tiles_n / w.d->bunit;  // groups of j2 tiles
  w.a = r % w.d->tiles_m;
  r /= w.d->tiles_m;
  w.nb = w.d->bunit;
  w.b0 = (r % nbg) * w.nb;
  r /= nbg;
  w.s = r % w.d->slabs;
  w.c = r / w.d->slabs;
  return w;
}
// The i2 range [lo, hi) of j2 tile b: the column support of its Phi_b rows
// (multiples of 64, the end clipped to n2), or all of x2.
__device__ __forceinline__ void x2_range(const TcPassDesc* d, int c, int b, int& lo, int& hi) {
  lo = 0;
  hi = d->n2;
  const int2* t = d->kband2[c];
  if (t == nullptr) return;
  const int2 r = __ldg(t + b);  // 128-row groups: the tile's own
  if (r.x < r.y) {
    lo = r.x;
    hi = r.y;
  }
}
// The union of the ranges of a unit's tiles.
__device__ __forceinline__ void x2_union(const UnitF& w, int& lo, int& hi) {
  x2_range(w.d, w.c, w.b0, lo, hi);
  for (int b = w.b0 + 1; b < w.b0 + w.nb; ++b) {
    int l, h;
    x2_range(w.d, w.c, b, l, h);
    lo = min(lo, l);
    hi = max(hi, h);
  }
}
// Chunks [c0, c1) of the group starting at g2 (nch chunks) that tile b
// contracts over.
__device__ __forceinline__ void tile_chunks(const UnitF& w, int b, int g2, int nch, int& c0,
                                            int& c1) {
  int l, h;
  x2_range(w.d, w.c, b, l, h);
  c0 = max(0, (l - g2) / 64);
  c1 = min(nch, (h - g2 + 63) / 64);
}

template <bool IND = false>
__global__ void __launch_bounds__(kThreads, 1) tc_fused_kernel(const __grid_constant__ TcLaunch L) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(smem + kFStages * kFStage);
  uint64_t* empty = full + kFStages;
  uint64_t* d1_full = empty + kFStages;  // MMA1 of a group complete (commit)
  uint64_t* d1_free = d1_full + 1;       // the group's D1 read by every epilogue warp
  uint64_t* p_full = d1_free + 1;        // [4] chunk ch's pieces stored (every epilogue
                                         // warp), one phase per group that has a chunk ch
  uint64_t* p_done = p_full + 4;         // every MMA2 of a group complete (commit)
  uint64_t* acc_full = p_done + 1;       // D2 of a tile complete (commit)
  uint64_t* acc_empty = acc_full + 1;    // D2 of a tile read by every epilogue warp
  uint64_t* drain = acc_empty + 1;
  uint32_t* tmem_slot = (uint32_t*)(drain + 1);
  int* abort_flag = (int*)(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  pdl_trigger();

  if (threadIdx.x == 0) {
    for (int s = 0; s < kFStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(d1_full, 1);
    mbar_init(d1_free, kEpiWarps);
    for (int ch = 0; ch < 4; ++ch) mbar_init(&p_full[ch], kEpiWarps);
    mbar_init(p_done, 1);
    mbar_init(acc_full, 1);
    mbar_init(acc_empty, kEpiWarps);
    mbar_init(drain, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    tmem_alloc(tmem_slot, 512);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  volatile int* abort_v = abort_flag;

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer: per group the MMA1 K-blocks, then per
    // tile the Phi_b blocks of its chunks, in the order the MMA thread
    // consumes them
    uint32_t g = 0;
    bool stop = false, waited = false;
    auto next_stage = [&](uint32_t bytes) -> uint8_t* {
      const int s = g % kFStages;
      const uint32_t it = g / kFStages;
      if (*abort_v || (it > 0 && !mbar_wait(&empty[s], (it - 1) & 1))) {
        atomicCAS(L.err, 0, kErrTimeoutEmpty);
        *abort_v = 1;
        stop = true;
        return nullptr;
      }
      if (!waited) {  // W is the previous launch's output
        pdl_wait();
        waited = true;
      }
      mbar_arrive_expect_tx(&full[s], bytes);
      return smem + s * kFStage;
    };
    for (int u = blockIdx.x; u < L.nunits && !stop; u += gridDim.x) {
      const UnitF w = decode_unitf(L, u);
      const TcPassDesc* D = w.d;
      const CUtensorMap* ma = &D->amap[w.c];
      const CUtensorMap* mw = &D->bmap[w.c];
      const CUtensorMap* mc = &D->cmap[w.c];
      asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)ma) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)mw) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)mc) : "memory");
      int kb0, kb1, xlo, xhi;
      k_blocks(D, w.c, w.a * kBM, kFBK, kb0, kb1);
      x2_union(w, xlo, xhi);
      for (int g2 = xlo; g2 < xhi && !stop; g2 += kFRowsW) {
        const int nch = (min(kFRowsW, xhi - g2) + 63) / 64;
        for (int kb = kb0; kb < kb1 && !stop; ++kb, ++g) {
          uint8_t* st = next_stage(kFStage);
          if (!st) break;
          tma_load_3d(st, ma, &full[g % kFStages], kb * kFBK, w.a * kBM, 0);
          tma_load_3d(st + kPieces * kFTileA, mw, &full[g % kFStages], kb * kFBK,
                      w.s * D->n2 + g2, 0);
        }
        for (int b = w.b0; b < w.b0 + w.nb && !stop; ++b) {
          int c0, c1;
          tile_chunks(w, b, g2, nch, c0, c1);
          for (int ch = c0; ch < c1 && !stop; ++ch, ++g) {
            uint8_t* st = next_stage(2 * kPieces * kFTileC);
            if (!st) break;
            tma_load_3d(st, mc, &full[g % kFStages], g2 + ch * 64, b * kBM, 0);
            tma_load_3d(st + kPieces * kFTileC, mc, &full[g % kFStages], g2 + ch * 64 + kFBK,
                        b * kBM, 0);
          }
        }
      }
    }
    // the last kFStages loads must have landed before exit
    const uint32_t first = g > (uint32_t)kFStages ? g - kFStages : 0;
    for (uint32_t q = first; q < g; ++q) mbar_wait(&full[q % kFStages], (q / kFStages) & 1);
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer
    const uint64_t dS0 = kmajor_desc<64>(smem_u32(smem));
    const uint32_t idesc2 = idesc_bf16(kBM, kBM);
    uint32_t g = 0, grp = 0, nt = 0;
    uint32_t pu[4] = {0, 0, 0, 0};  // completed phases of p_full[ch]: groups with a chunk ch
    bool stop = false;
    auto fail = [&](int code) {
      atomicCAS(L.err, 0, code);
      *abort_v = 1;
      stop = true;
    };
    for (int u = blockIdx.x; u < L.nunits && !stop; u += gridDim.x) {
      const UnitF w = decode_unitf(L, u);
      const TcPassDesc* D = w.d;
      int kb0, kb1, xlo, xhi;
      k_blocks(D, w.c, w.a * kBM, kFBK, kb0, kb1);
      x2_union(w, xlo, xhi);
      for (int g2 = xlo; g2 < xhi && !stop; g2 += kFRowsW, ++grp) {
        const int nch = (min(kFRowsW, xhi - g2) + 63) / 64;
        const bool first_group = g2 == xlo, last_group = g2 + kFRowsW >= xhi;
        // D1 and the pieces' columns are free once the epilogue warps have
        // read the previous group's D1 and its MMA2 have completed
        if (grp > 0 && (!mbar_wait(d1_free, (grp - 1) & 1) || !mbar_wait(p_done, (grp - 1) & 1))) {
          fail(kErrTimeoutDone);
          break;
        }
        tc_fence_after();
        const uint32_t idesc1 = idesc_bf16(kBM, 64 * nch);
        for (int kb = kb0; kb < kb1; ++kb, ++g) {
          if (!mbar_wait(&full[g % kFStages], (g / kFStages) & 1)) {
            fail(kErrTimeoutFull);
            break;
          }
          const uint64_t da = dS0 + (uint64_t)(((g % kFStages) * kFStage) >> 4);
          const uint64_t db = da + (uint64_t)((kPieces * kFTileA) >> 4);
          issue_stage<64, kFTileA, kFTileW, false>(tmem + kFColD1, da, db, idesc1, kb != kb0);
          mma_commit(&empty[g % kFStages]);
        }
        if (stop) break;
        mma_commit(d1_full);
        uint32_t ready = 0;  // chunks of this group whose pieces are known to be stored
        for (int b = w.b0; b < w.b0 + w.nb && !stop; ++b) {
          int c0, c1;
          tile_chunks(w, b, g2, nch, c0, c1);
          // D2 is free once the epilogue warps have read the previous tile
          if (first_group && nt > 0 && !mbar_wait(acc_empty, (nt - 1) & 1)) {
            fail(kErrTimeoutDone);
            break;
          }
          for (int ch = c0; ch < c1; ++ch, ++g) {
            if (!(ready >> ch & 1u)) {
              if (!mbar_wait(&p_full[ch], pu[ch] & 1)) {
                fail(kErrTimeoutDone);
                break;
              }
              ready |= 1u << ch;
            }
            tc_fence_after();
            if (!mbar_wait(&full[g % kFStages], (g / kFStages) & 1)) {
              fail(kErrTimeoutFull);
              break;
            }
            const uint64_t db0 = dS0 + (uint64_t)(((g % kFStages) * kFStage) >> 4);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
              const uint64_t b0 = db0 + (uint64_t)(((kk >> 1) * kPieces * kFTileC) >> 4) +
                                  (uint64_t)((kk & 1) * 2);
              const uint64_t b1 = b0 + (uint64_t)(kFTileC >> 4);
              const uint64_t b2 = b0 + (uint64_t)(2 * kFTileC >> 4);
              const uint32_t sub = (uint32_t)((kk & 1) * 8);
              const uint32_t a0 = tmem + slot_col(ch, 0, kk >> 1) + sub;
              const uint32_t a1 = tmem + slot_col(ch, 1, kk >> 1) + sub;
              const uint32_t a2 = tmem + slot_col(ch, 2, kk >> 1) + sub;
              const uint32_t dt = tmem + kFColD2;
              const uint32_t acc = (first_group && ch == c0 && kk == 0) ? 0u : 1u;
              mma_bf16_ts(dt, a2, b0, idesc2, acc);
              mma_bf16_ts(dt, a1, b1, idesc2, 1);
              mma_bf16_ts(dt, a1, b0, idesc2, 1);
              mma_bf16_ts(dt, a0, b2, idesc2, 1);
              mma_bf16_ts(dt, a0, b1, idesc2, 1);
              mma_bf16_ts(dt, a0, b0, idesc2, 1);
            }
            mma_commit(&empty[g % kFStages]);
          }
          if (stop) break;
          if (last_group) {
            mma_commit(acc_full);
            ++nt;
          }
        }
        if (stop) break;
        for (int ch = 0; ch < nch; ++ch) ++pu[ch];  // waited on or not, every chunk completed
        mma_commit(p_done);
      }
    }
    mma_commit(drain);
    mbar_wait(drain, 0);
  } else if (warp >= 2) {
    // ---------------- epilogue warps: split D1 into pieces, then write T
    pdl_wait();
    const int q = warp & 3;            // TMEM lane quarter
    const int half = (warp - 2) >> 2;  // column half
    const uint32_t lane_off = (uint32_t)(q * 32) << 16;
    uint32_t grp = 0, nt = 0;
    bool stop = false;
    auto warp_wait = [&](uint64_t* bar, uint32_t parity) -> bool {
      if (__all_sync(0xffffffffu, mbar_wait_sleep(bar, parity))) return true;
      if (lane == 0) atomicCAS(L.err, 0, kErrTimeoutDone);
      *abort_v = 1;
      stop = true;
      return false;
    };
    auto arrive = [&](uint64_t* bar) {
      tc_fence_before();
      __syncwarp();
      if (lane == 0)
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
    };
    for (int u = blockIdx.x; u < L.nunits && !stop; u += gridDim.x) {
      const UnitF w = decode_unitf(L, u);
      const TcPassDesc* D = w.d;
      int xlo, xhi;
      x2_union(w, xlo, xhi);
      for (int g2 = xlo; g2 < xhi && !stop; g2 += kFRowsW, ++grp) {
        const int nch = (min(kFRowsW, xhi - g2) + 63) / 64;
        // the slots are free once the previous group's MMA2 have completed
        if (grp > 0 && !warp_wait(p_done, (grp - 1) & 1)) break;
        if (!warp_wait(d1_full, grp & 1)) break;
        tc_fence_after();
        for (int ch = 0; ch < nch; ++ch) {
          uint32_t r[2][16];
          const uint32_t src = tmem + lane_off + kFColD1 + (uint32_t)(ch * 64 + half * 32);
          tmem_ld16_nw(src, r[0]);
          tmem_ld16_nw(src + 16, r[1]);
          tmem_wait_ld();
          tmem_fence16(r[0]);
          tmem_fence16(r[1]);
          uint32_t pk[3][16];
#pragma unroll
          for (int j = 0; j < 16; ++j)
            split3_pair(__uint_as_float(r[j / 8][(2 * j) % 16]),
                        __uint_as_float(r[j / 8][(2 * j + 1) % 16]), pk[0][j], pk[1][j], pk[2][j]);
#pragma unroll
          for (int p = 0; p < 3; ++p) tmem_st16(tmem + lane_off + slot_col(ch, p, half), pk[p]);
          tmem_wait_st();
          arrive(&p_full[ch]);
        }
        arrive(d1_free);  // every D1 column of this group has been read
      }
      if (stop) break;
      // ---- T, one j2 tile at a time
      const int n1 = D->n1, n2 = D->n2, mode = D->mode;
      const int m = w.a * kBM + q * 32 + lane;  // j1
      const bool mrow = m < n1;
      const int64_t slab = (int64_t)w.s * n2 * n1;
      float* lp = (mode == kAxpy && D->lo[w.c]) ? D->lo[w.c] + slab : nullptr;
      double* ind = (IND && mode == kAxpy) ? indicator_slot(D, w.c) : nullptr;
      const float* bsrc = D->base[w.c] ? D->base[w.c] + slab : nullptr;
      const bool plain = mode == kAxpy && !lp && !ind;
      const uint32_t ta = tmem + lane_off + kFColD2 + (uint32_t)(half * 64);
      for (int b = w.b0; b < w.b0 + w.nb && !stop; ++b, ++nt) {
        const int n0 = b * kBM + half * 64;  // first j2 of this warp
        // plain update: the warp's 64 base values are loaded before D2 is ready
        float bv[64];
#pragma unroll
        for (int j = 0; j < 64; ++j) {
          const int col = n0 + j;
          bv[j] = (plain && bsrc && mrow && col < n2) ? __ldg(bsrc + (int64_t)col * n1 + m) : 0.f;
        }
        if (!warp_wait(acc_full, nt & 1)) break;
        tc_fence_after();
        if (__any_sync(0xffffffffu, *abort_v)) {
          stop = true;
          break;
        }
        if (plain) {
          float* of = D->outf[w.c] + slab;
          const float alpha = D->alpha;
#pragma unroll
          for (int bt = 0; bt < 4; bt += 2) {
            uint32_t r[2][16];
            tmem_ld16_nw(ta + (uint32_t)(bt * 16), r[0]);
            tmem_ld16_nw(ta + (uint32_t)((bt + 1) * 16), r[1]);
            tmem_wait_ld();
            tmem_fence16(r[0]);
            tmem_fence16(r[1]);
#pragma unroll
            for (int jj = 0; jj < 32; ++jj) {
              const int col = n0 + bt * 16 + jj;
              if (mrow && col < n2)
                of[(int64_t)col * n1 + m] =
                    __fmaf_rn(alpha, __uint_as_float(r[jj / 16][jj % 16]), bv[bt * 16 + jj]);
            }
          }
        } else if (mode == kAxpy) {
          axpy_epilogue<4>(ta, D->outf[w.c] + slab, bsrc, lp, D->alpha, n1, n2, n0, m, mrow, ind,
                           D->ind_n1, D->ind_n2);
        } else {  // kPieces3: three BF16 pieces of T, natural layout
          // the warp's 64 columns are read into registers and D2 released
          // before the stores, so the next tile's MMA2 overlaps them
          uint32_t r[4][16];
#pragma unroll
          for (int bt = 0; bt < 4; ++bt) tmem_ld16_nw(ta + (uint32_t)(bt * 16), r[bt]);
          tmem_wait_ld();
#pragma unroll
          for (int bt = 0; bt < 4; ++bt) tmem_fence16(r[bt]);
          arrive(acc_empty);
          // Lanes pair up (rows m, m + 1; n1 is even): of two columns the even
          // lane takes the first and the odd lane the second, each with both
          // rows, so every store writes two BF16 of one piece (4 bytes)
          uint32_t* op = reinterpret_cast<uint32_t*>(D->outp[w.c]);
          const int64_t plane2 = (int64_t)D->slabs * n2 * n1 / 2;
          const bool odd = lane & 1;
          const int mp = m - (odd ? 1 : 0);
#pragma unroll
          for (int jj = 0; jj < 64; jj += 2) {
            const float x0 = __uint_as_float(r[jj / 16][jj % 16]);
            const float x1 = __uint_as_float(r[jj / 16][jj % 16 + 1]);
            const float got = __shfl_xor_sync(0xffffffffu, odd ? x0 : x1, 1);
            const int col = n0 + jj + (odd ? 1 : 0);
            if (mp < n1 && col < n2) {
              uint32_t w0, w1, w2;
              split3_pair(odd ? got : x0, odd ? x1 : got, w0, w1, w2);
              const int64_t o2 = (slab + (int64_t)col * n1 + mp) >> 1;
              op[o2] = w0;
              op[plane2 + o2] = w1;
              op[2 * plane2 + o2] = w2;
            }
          }
          continue;  // D2 already released
        }
        arrive(acc_empty);  // D2 of this tile has been read
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, 512);
  }
}

// ---------------------------------------------------------------- pointwise
// Per-solve arguments of the pointwise kernels of the tensor-core path; one
// launch covers one solve or a whole batch.
//
// The stencil kernel sees every grid as three axes: x = i1 (contiguous), y
// (the x2 direction of a 3D grid, absent in 2D) and z, the slowest axis (x3
// in 3D, x2 in 2D).  A warp owns a run of 128 x-points (four per lane, so
// loads are float4 and stores of four BF16 values 8 bytes) on one y row and
// marches `zlen` consecutive z planes, keeping the z neighbours in registers.
struct PwDesc {
  CUtensorMap tu, tv;  // 3D grids: u and v as [nz][ny][nx] FP32, box {kRingBoxX, kRingBoxY, 1}
  PointwiseArgsT<float> a;
  const float* u;
  const float* v;
  const float* u2;
  const float* v2;
  __nv_bfloat16* wu;   // pieces [3][N] of the u output
  __nv_bfloat16* wv;
  double* ind;         // indicator ring [ind_k][4] and step counter (null: off)
  int64_t* ind_ctr;
  int ind_k;
  float tau;
  int nx, ny, nz;      // stencil axes (ny = 1 in 2D)
  int xsegs, zlen, zsegs;  // 2D: warp x segments; 3D: block x tiles.  z runs
  int ytiles;          // 3D: block y tiles
  int64_t sy, sz;      // element strides of y and z
};

// Kernel parameter of a pointwise launch: one solve carries its descriptor
// in the parameter; a grouped launch reads them from device memory.
struct PwLaunch {
  PwDesc one;          // used when desc is null
  const PwDesc* desc;  // [nsolves] in device memory, or null
  const int* bstart;   // [nsolves + 1] prefix sums of this kernel's blocks (desc non-null)
  int nsolves;
  int* err;            // device error word (bounded waits)
};

constexpr int kPwThreads = 256;
constexpr int kPwWarps = kPwThreads / 32;
constexpr int kSegX = 128;                          // x-points per warp
constexpr int kFlatVec = 2;                         // float4 per thread per array
constexpr int kFlatPerBlock = kPwThreads * 4 * kFlatVec;

// The block's descriptor: the launch parameter for one solve, else staged
// once in shared memory.  lb = the block's index within its solve.  Waits
// for the previous kernel of the step before returning (the descriptor is
// static; the data it points to is not).
// home = the descriptor where it lives (launch parameter or device memory),
// from where tensor maps must be read.
__device__ __forceinline__ const PwDesc* block_desc(const PwLaunch& L, PwDesc* sd, int& lb,
                                                    const PwDesc** home = nullptr) {
  pdl_trigger();
  if (L.desc == nullptr) {
    lb = blockIdx.x;
    if (home) *home = &L.one;
    pdl_wait();
    return &L.one;
  }
  const int s = find_segment(L.bstart, L.nsolves, blockIdx.x);
  if (home) *home = L.desc + s;
  static_assert(sizeof(PwDesc) % 4 == 0, "PwDesc is copied in 32-bit words");
  const uint32_t* src = reinterpret_cast<const uint32_t*>(L.desc + s);
  uint32_t* dst = reinterpret_cast<uint32_t*>(sd);
  for (int w = threadIdx.x; w < (int)(sizeof(PwDesc) / 4); w += blockDim.x) dst[w] = __ldg(src + w);
  lb = blockIdx.x - __ldg(L.bstart + s);
  __syncthreads();
  pdl_wait();
  return sd;
}

// Indicators of Sec. 4: the first kernel of a step opens the step's slot in
// the solve's indicator ring (the counter and slot are written by one thread
// after the previous step has completed; the last product of the step, which
// runs after this kernel has completed, accumulates into it).
__device__ __forceinline__ void indicator_open_step(const PwDesc* dp, int lb) {
  if (lb != 0 || threadIdx.x != 0 || dp->ind == nullptr) return;
  const int64_t s = *dp->ind_ctr + 1;
  *dp->ind_ctr = s;
  double* slot = dp->ind + 4 * (s % dp->ind_k);
  slot[0] = slot[1] = slot[2] = slot[3] = 0.0;
}

// One direction of the stencil of Eq. 6 at an interior point, and at any
// point (the Neumann rows at i = 0 and i = n - 1 take one neighbour).
__device__ __forceinline__ float tri_in(float xm, float xc, float xp, float lo, float up) {
  return lo * (xm - xc) + up * (xp - xc);
}
__device__ __forceinline__ float tri_dir(float xm, float xc, float xp, int i, int n, float lo,
                                         float up, float b0, float bn) {
  if (i == 0) return b0 * (xp - xc);
  if (i == n - 1) return bn * (xm - xc);
  return tri_in(xm, xc, xp, lo, up);
}
// The x direction at point j of a group of four starting at a multiple of
// 4, on a row whose length n is a multiple of 4: only j = 0 can be the
// row's first point and only j = 3 its last (j is a constant once the
// loop over the group is unrolled).
__device__ __forceinline__ float tri_x4(int j, float xm, float xc, float xp, int i, int n,
                                        float lo, float up, float b0, float bn) {
  if (j == 0 && i == 0) return b0 * (xp - xc);
  if (j == 3 && i == n - 1) return bn * (xm - xc);
  return tri_in(xm, xc, xp, lo, up);
}

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ float el(const float4& q, int j) {
  return j == 0 ? q.x : (j == 1 ? q.y : (j == 2 ? q.z : q.w));
}

// Split four values into BF16 pieces and store piece k of all four at
// out + k * N + idx (idx a multiple of 4: 8-byte stores).
// The pieces are those of split3, two values per conversion instruction.
__device__ __forceinline__ void store_pieces4(__nv_bfloat16* out, int64_t N, int64_t idx,
                                              const float (&w)[4]) {
  float r[4] = {w[0], w[1], w[2], w[3]};
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const __nv_bfloat162 lo = __floats2bfloat162_rn(r[0], r[1]);
    const __nv_bfloat162 hi = __floats2bfloat162_rn(r[2], r[3]);
    uint2 q;
    q.x = *reinterpret_cast<const uint32_t*>(&lo);
    q.y = *reinterpret_cast<const uint32_t*>(&hi);
    *reinterpret_cast<uint2*>(out + k * N + idx) = q;
    if (k < 2) {
      const float2 a = __bfloat1622float2(lo), b = __bfloat1622float2(hi);
      r[0] -= a.x;
      r[1] -= a.y;
      r[2] -= b.x;
      r[3] -= b.y;
    }
  }
}

// The same in the operand format F: for TF32, two FP32 words per value
// (piece k of the four values at out + k * N + idx, 16-byte stores).
template <int F>
__device__ __forceinline__ void store_pieces_fmt(__nv_bfloat16* out, int64_t N, int64_t idx,
                                                 const float (&w)[4]) {
  if constexpr (F == kFmtTF32) {
    float* o = reinterpret_cast<float*>(out);
    float hi[4], lo[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) split2_tf32(w[j], hi[j], lo[j]);
    *reinterpret_cast<float4*>(o + idx) = make_float4(hi[0], hi[1], hi[2], hi[3]);
    *reinterpret_cast<float4*>(o + N + idx) = make_float4(lo[0], lo[1], lo[2], lo[3]);
  } else {
    store_pieces4(out, N, idx, w);
  }
}

// The tridiagonal coefficients of one component on one axis.
struct Coef {
  float lo, up, b0, bn;
};
__device__ __forceinline__ Coef coef(const TridiagT<float>& A) { return Coef{A.lo, A.up, A.b0, A.bn}; }

// W^c = K^c U^c + G^c(U, V) as BF16 pieces [3][N] in the natural layout
// (Eq. 11, first stage: the stencil of Eq. 6 plus the reaction), 2D grids
// (x = x1, z = x2).  Each iteration of a warp covers ZB consecutive z planes
// and issues all their loads (the planes and the x values beyond the warp's
// run) before any arithmetic, so that a warp keeps several planes of loads
// in flight; the planes z - 1 and z + ZB carry over.
template <int ZB, int F = kFmtBF16, bool DF = false>
__global__ void __launch_bounds__(kPwThreads, 2) rhs_pieces_kernel(const __grid_constant__ PwLaunch L) {
  __shared__ PwDesc sd;
  int lb;
  const PwDesc* dp = block_desc(L, &sd, lb);
  indicator_open_step(dp, lb);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nx = dp->nx, nz = dp->nz, xsegs = dp->xsegs;
  int64_t unit = (int64_t)lb * kPwWarps + warp;
  if (unit >= (int64_t)xsegs * dp->zsegs) return;  // whole warps only
  const int xs = (int)(unit % xsegs);
  const int z0 = (int)(unit / xsegs) * dp->zlen;
  const int z1 = min(z0 + dp->zlen, nz);
  const int x0 = xs * kSegX + 4 * lane;
  const bool act = x0 < nx;
  const int64_t sz = dp->sz, N = dp->a.N;
  const float* __restrict__ u = dp->u;
  const float* __restrict__ v = dp->v;
  __nv_bfloat16* wu = dp->wu;
  __nv_bfloat16* wv = dp->wv;
  // axis coefficients: x = mu 1, z = mu 2
  const Coef cxu = coef(dp->a.A[0][0]), cxv = coef(dp->a.A[1][0]);
  const Coef czu = coef(dp->a.A[0][1]), czv = coef(dp->a.A[1][1]);
  const ReactionT<float> rx = dp->a.rx;
  const int64_t col = x0;
  const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
  // run ends: lane 0 needs x0 - 1, lane 31 needs x0 + 4 (others come by shuffle)
  const int64_t eoff = lane == 0 ? -1 : 4;
  const bool eok = act && ((lane == 0 && x0 > 0) || (lane == 31 && x0 + 4 < nx));
  float4 pu[ZB + 2], pv[ZB + 2];  // planes z - 1 .. z + ZB
  pu[0] = (act && z0 > 0) ? ld4(u + (z0 - 1) * sz + col) : zero4;
  pv[0] = (act && z0 > 0) ? ld4(v + (z0 - 1) * sz + col) : zero4;
  pu[1] = act ? ld4(u + z0 * sz + col) : zero4;
  pv[1] = act ? ld4(v + z0 * sz + col) : zero4;
  for (int z = z0; z < z1; z += ZB) {  // trip counts uniform over the warp
    float eu[ZB], ev[ZB];
#pragma unroll
    for (int j = 2; j < ZB + 2; ++j) {
      const int zz = z + j - 1;
      const bool ok = act && zz < nz;
      pu[j] = ok ? ld4(u + zz * sz + col) : zero4;
      pv[j] = ok ? ld4(v + zz * sz + col) : zero4;
    }
#pragma unroll
    for (int q = 0; q < ZB; ++q) {
      const int64_t idx = (int64_t)(z + q) * sz + col;
      const bool ok = act && z + q < z1;
      eu[q] = (ok && eok) ? u[idx + eoff] : 0.f;
      ev[q] = (ok && eok) ? v[idx + eoff] : 0.f;
    }
#pragma unroll
    for (int q = 0; q < ZB; ++q) {
      const int zq = z + q;
      if (zq >= z1) break;  // uniform
      const float4 uc = pu[q + 1], vc = pv[q + 1];
      float ul = __shfl_up_sync(0xffffffffu, uc.w, 1), vl = __shfl_up_sync(0xffffffffu, vc.w, 1);
      float ur = __shfl_down_sync(0xffffffffu, uc.x, 1), vr = __shfl_down_sync(0xffffffffu, vc.x, 1);
      if (lane == 0) {
        ul = eu[q];
        vl = ev[q];
      }
      if (lane == 31) {
        ur = eu[q];
        vr = ev[q];
      }
      float ou[4], ov[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int xi = x0 + j;
        const float cu = el(uc, j), cv = el(vc, j);
        const float lu = j == 0 ? ul : el(uc, j - 1), lv = j == 0 ? vl : el(vc, j - 1);
        const float ru = j == 3 ? ur : el(uc, j + 1), rv = j == 3 ? vr : el(vc, j + 1);
        if constexpr (DF) {  // accurate mode: stencil and reaction in double-float, one rounding
          const CoefDF dxu = coef_df(dp->a.A[0][0], dp->a.Alo[0][0]);
          const CoefDF dxv = coef_df(dp->a.A[1][0], dp->a.Alo[1][0]);
          const CoefDF dzu = coef_df(dp->a.A[0][1], dp->a.Alo[0][1]);
          const CoefDF dzv = coef_df(dp->a.A[1][1], dp->a.Alo[1][1]);
          dfloat gu, gv;
          react_dfd(rx, cu, cv, gu, gv);
          ou[j] = df_round(dtri_x4(j, lu, cu, ru, xi, nx, dxu.lo, dxu.up, dxu.b0, dxu.bn) +
                           dtri_dir(el(pu[q], j), cu, el(pu[q + 2], j), zq, nz, dzu.lo, dzu.up,
                                    dzu.b0, dzu.bn) + gu);
          ov[j] = df_round(dtri_x4(j, lv, cv, rv, xi, nx, dxv.lo, dxv.up, dxv.b0, dxv.bn) +
                           dtri_dir(el(pv[q], j), cv, el(pv[q + 2], j), zq, nz, dzv.lo, dzv.up,
                                    dzv.b0, dzv.bn) + gv);
        } else {
          float ku = tri_x4(j, lu, cu, ru, xi, nx, cxu.lo, cxu.up, cxu.b0, cxu.bn);
          float kv = tri_x4(j, lv, cv, rv, xi, nx, cxv.lo, cxv.up, cxv.b0, cxv.bn);
          ku += tri_dir(el(pu[q], j), cu, el(pu[q + 2], j), zq, nz, czu.lo, czu.up, czu.b0, czu.bn);
          kv += tri_dir(el(pv[q], j), cv, el(pv[q + 2], j), zq, nz, czv.lo, czv.up, czv.b0, czv.bn);
          float gu, gv;
          react<float>(rx, cu, cv, gu, gv);
          ou[j] = ku + gu;
          ov[j] = kv + gv;
        }
      }
      if (act) {
        const int64_t idx = (int64_t)zq * sz + col;
        store_pieces_fmt<F>(wu, N, idx, ou);
        store_pieces_fmt<F>(wv, N, idx, ov);
      }
    }
    pu[0] = pu[ZB];
    pv[0] = pv[ZB];
    pu[1] = pu[ZB + 1];
    pv[1] = pv[ZB + 1];
  }
}
// The same for 3D grids (x = x1, y = x2, z = x3).  A block owns a
// kRingX x kRingY tile of the (x, y) plane and marches a run of z planes.
// Each plane of u and v arrives with its x and y halo by one TMA copy per
// field (out-of-range points read as zero and are never used: the boundary
// rows of Eq. 6 take no outer neighbour) into a ring of kRingSlots
// shared-memory slots.  The copy of plane z + 3 is issued before plane z is
// computed, so every block keeps about two planes of loads in flight and
// every value is read from HBM once per tile.  Warp w computes tile rows w
// and w + 8; the arithmetic is that of the 2D kernel plus the y term.
constexpr int kRingX = 128, kRingY = 16;
constexpr int kRingBoxX = kRingX + 8;   // x0 - 4 .. x0 + 131: 16-byte aligned start
constexpr int kRingBoxY = kRingY + 2;   // y0 - 1 .. y0 + 16
constexpr int kRingPlane = kRingBoxX * kRingBoxY;        // floats per field and plane copy
constexpr int kRingField = (kRingPlane + 31) / 32 * 32;  // its slot part: 128-byte multiple
constexpr int kRingTx = 2 * kRingPlane * 4;              // bytes per plane (u and v)
constexpr int kRingSlots = 5;
constexpr int kRingSmem = kRingSlots * 2 * kRingField * 4 + 128 + kRingSlots * 8;
static_assert(kRingField * 4 % 128 == 0, "copy destinations keep 128-byte alignment");

template <int F = kFmtBF16, bool DF = false>
__global__ void __launch_bounds__(kPwThreads, 2) rhs3_ring_kernel(const __grid_constant__ PwLaunch L) {
  extern __shared__ uint8_t smem_raw[];
  float* ring = (float*)(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
  uint64_t* full = (uint64_t*)(ring + kRingSlots * 2 * kRingField);
  __shared__ PwDesc sd;
  __shared__ int abort_s;
  int lb;
  const PwDesc* src = nullptr;
  const PwDesc* dp = block_desc(L, &sd, lb, &src);
  indicator_open_step(dp, lb);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nx = dp->nx, ny = dp->ny, nz = dp->nz;
  int b = lb;
  const int x0 = (b % dp->xsegs) * kRingX;
  b /= dp->xsegs;
  const int y0 = (b % dp->ytiles) * kRingY;
  const int z0 = (b / dp->ytiles) * dp->zlen;
  if (z0 >= nz) return;  // whole block
  const int z1 = min(z0 + dp->zlen, nz);
  const int plo = max(z0 - 1, 0), phi = min(z1, nz - 1);  // planes read: plo .. phi
  const int np = phi - plo + 1;
  const CUtensorMap* mu = &src->tu;
  const CUtensorMap* mv = &src->tv;
  auto issue = [&](int q) {  // plane plo + q into slot q % kRingSlots
    const int sl = q % kRingSlots;
    float* dst = ring + sl * 2 * kRingField;
    mbar_arrive_expect_tx(&full[sl], kRingTx);
    tma_load_3d(dst, mu, &full[sl], x0 - 4, y0 - 1, plo + q);
    tma_load_3d(dst + kRingField, mv, &full[sl], x0 - 4, y0 - 1, plo + q);
  };
  int issued = 0, ready = 0;  // planes requested / known landed (thread 0)
  if (threadIdx.x == 0) {
    abort_s = 0;
    for (int sl = 0; sl < kRingSlots; ++sl) mbar_init(&full[sl], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)mu) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)mv) : "memory");
    for (; issued < np && issued < kRingSlots; ++issued) issue(issued);
  }
  const Coef cxu = coef(dp->a.A[0][0]), cxv = coef(dp->a.A[1][0]);
  const Coef cyu = coef(dp->a.A[0][1]), cyv = coef(dp->a.A[1][1]);
  const Coef czu = coef(dp->a.A[0][2]), czv = coef(dp->a.A[1][2]);
  const ReactionT<float> rx = dp->a.rx;
  const int64_t sy = dp->sy, sz = dp->sz, N = dp->a.N;
  __nv_bfloat16* wu = dp->wu;
  __nv_bfloat16* wv = dp->wv;
  const int xl = x0 + 4 * lane;
  const bool act = xl < nx;
  for (int z = z0; z < z1; ++z) {
    if (threadIdx.x == 0) {
      // planes z - 1 .. z + 1 must have landed
      const int need = min(z + 1, phi) - plo + 1;
      for (; ready < need; ++ready) {
        if (!mbar_wait(&full[ready % kRingSlots], (uint32_t)(ready / kRingSlots) & 1u)) {
          atomicCAS(L.err, 0, kErrTimeoutFull);
          abort_s = 1;
          break;
        }
      }
    }
    __syncthreads();  // data visible; every warp is done with plane z - 2
    if (abort_s) break;
    if (threadIdx.x == 0) {
      const int qfree = z - 2 - plo;  // plane z - 2's slot takes plane z + 3
      if (qfree >= 0 && qfree + kRingSlots < np && issued == qfree + kRingSlots) issue(issued++);
    }
    const float* pc = ring + ((z - plo) % kRingSlots) * 2 * kRingField;
    const float* pm = z > 0 ? ring + ((z - 1 - plo) % kRingSlots) * 2 * kRingField : nullptr;
    const float* pp = z + 1 < nz ? ring + ((z + 1 - plo) % kRingSlots) * 2 * kRingField : nullptr;
#pragma unroll 1
    for (int rr = 0; rr < 2; ++rr) {
      const int r = warp + 8 * rr;
      const int y = y0 + r;
      if (y >= ny) break;  // uniform over the warp
      const bool yzin = y > 0 && y + 1 < ny && z > 0 && z + 1 < nz;  // uniform over the warp
      const int o = (r + 1) * kRingBoxX + 4 + 4 * lane;
      const float4 uc = *reinterpret_cast<const float4*>(pc + o);
      const float4 vc = *reinterpret_cast<const float4*>(pc + kRingField + o);
      const float4 uym = *reinterpret_cast<const float4*>(pc + o - kRingBoxX);
      const float4 vym = *reinterpret_cast<const float4*>(pc + kRingField + o - kRingBoxX);
      const float4 uyp = *reinterpret_cast<const float4*>(pc + o + kRingBoxX);
      const float4 vyp = *reinterpret_cast<const float4*>(pc + kRingField + o + kRingBoxX);
      const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
      const float4 uzm = pm ? *reinterpret_cast<const float4*>(pm + o) : zero4;
      const float4 vzm = pm ? *reinterpret_cast<const float4*>(pm + kRingField + o) : zero4;
      const float4 uzp = pp ? *reinterpret_cast<const float4*>(pp + o) : zero4;
      const float4 vzp = pp ? *reinterpret_cast<const float4*>(pp + kRingField + o) : zero4;
      float ul = __shfl_up_sync(0xffffffffu, uc.w, 1), vl = __shfl_up_sync(0xffffffffu, vc.w, 1);
      float ur = __shfl_down_sync(0xffffffffu, uc.x, 1), vr = __shfl_down_sync(0xffffffffu, vc.x, 1);
      if (lane == 0) {
        ul = pc[o - 1];
        vl = pc[kRingField + o - 1];
      }
      if (lane == 31) {
        ur = pc[o + 4];
        vr = pc[kRingField + o + 4];
      }
      float ou[4], ov[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int xi = xl + j;
        const float cu = el(uc, j), cv = el(vc, j);
        const float lu = j == 0 ? ul : el(uc, j - 1), lv = j == 0 ? vl : el(vc, j - 1);
        const float ru = j == 3 ? ur : el(uc, j + 1), rv = j == 3 ? vr : el(vc, j + 1);
        if constexpr (DF) {  // accurate mode: stencil and reaction in double-float, one rounding
          const CoefDF dxu = coef_df(dp->a.A[0][0], dp->a.Alo[0][0]);
          const CoefDF dxv = coef_df(dp->a.A[1][0], dp->a.Alo[1][0]);
          const CoefDF dyu = coef_df(dp->a.A[0][1], dp->a.Alo[0][1]);
          const CoefDF dyv = coef_df(dp->a.A[1][1], dp->a.Alo[1][1]);
          const CoefDF dzu = coef_df(dp->a.A[0][2], dp->a.Alo[0][2]);
          const CoefDF dzv = coef_df(dp->a.A[1][2], dp->a.Alo[1][2]);
          dfloat gu, gv;
          react_dfd(rx, cu, cv, gu, gv);
          const dfloat ku = dtri_x4(j, lu, cu, ru, xi, nx, dxu.lo, dxu.up, dxu.b0, dxu.bn) +
                            dtri_dir(el(uym, j), cu, el(uyp, j), y, ny, dyu.lo, dyu.up, dyu.b0, dyu.bn) +
                            dtri_dir(el(uzm, j), cu, el(uzp, j), z, nz, dzu.lo, dzu.up, dzu.b0, dzu.bn);
          const dfloat kv = dtri_x4(j, lv, cv, rv, xi, nx, dxv.lo, dxv.up, dxv.b0, dxv.bn) +
                            dtri_dir(el(vym, j), cv, el(vyp, j), y, ny, dyv.lo, dyv.up, dyv.b0, dyv.bn) +
                            dtri_dir(el(vzm, j), cv, el(vzp, j), z, nz, dzv.lo, dzv.up, dzv.b0, dzv.bn);
          ou[j] = df_round(ku + gu);
          ov[j] = df_round(kv + gv);
        } else {
          float ku = tri_x4(j, lu, cu, ru, xi, nx, cxu.lo, cxu.up, cxu.b0, cxu.bn);
          float kv = tri_x4(j, lv, cv, rv, xi, nx, cxv.lo, cxv.up, cxv.b0, cxv.bn);
          if (yzin) {
            ku += tri_in(el(uym, j), cu, el(uyp, j), cyu.lo, cyu.up);
            kv += tri_in(el(vym, j), cv, el(vyp, j), cyv.lo, cyv.up);
            ku += tri_in(el(uzm, j), cu, el(uzp, j), czu.lo, czu.up);
            kv += tri_in(el(vzm, j), cv, el(vzp, j), czv.lo, czv.up);
          } else {
            ku += tri_dir(el(uym, j), cu, el(uyp, j), y, ny, cyu.lo, cyu.up, cyu.b0, cyu.bn);
            kv += tri_dir(el(vym, j), cv, el(vyp, j), y, ny, cyv.lo, cyv.up, cyv.b0, cyv.bn);
            ku += tri_dir(el(uzm, j), cu, el(uzp, j), z, nz, czu.lo, czu.up, czu.b0, czu.bn);
            kv += tri_dir(el(vzm, j), cv, el(vzp, j), z, nz, czv.lo, czv.up, czv.b0, czv.bn);
          }
          float gu, gv;
          react<float>(rx, cu, cv, gu, gv);
          ou[j] = ku + gu;
          ov[j] = kv + gv;
        }
      }
      if (act) {
        const int64_t idx = (int64_t)z * sz + (int64_t)y * sy + xl;
        store_pieces_fmt<F>(wu, N, idx, ou);
        store_pieces_fmt<F>(wv, N, idx, ov);
      }
    }
  }
  if (threadIdx.x == 0 && abort_s) {
    // copies still in flight land before the block's shared memory is released
    for (int q = ready; q < issued; ++q) mbar_wait(&full[q % kRingSlots], (uint32_t)(q / kRingSlots) & 1u);
  }
}

constexpr int kZB2 = 4;  // planes per iteration of the 2D stencil kernel

// Elementwise kernels: thread t of a block handles float4 groups
// base + k * kPwThreads + t, k < kFlatVec; loads are issued before any store.
#define FLAT_PROLOGUE                                                            \
  __shared__ PwDesc sdesc;                                                       \
  int lb;                                                                        \
  const PwDesc& sd = *block_desc(L, &sdesc, lb);                                 \
  const int64_t N = sd.a.N, N4 = N / 4;                                          \
  const int64_t g0 = (int64_t)lb * (kFlatPerBlock / 4) + threadIdx.x;

// D^c = G^c(U2, V2) - G^c(U, V) written as BF16 pieces [3][N] (Eq. 11,
// second stage).
template <int F = kFmtBF16>
__global__ void __launch_bounds__(kPwThreads) rdiff_pieces_kernel(const __grid_constant__ PwLaunch L) {
  FLAT_PROLOGUE
  const ReactionT<float> rx = sd.a.rx;
  float4 a0[kFlatVec], a1[kFlatVec], a2[kFlatVec], a3[kFlatVec];
#pragma unroll
  for (int k = 0; k < kFlatVec; ++k) {
    const int64_t g = g0 + k * kPwThreads;
    if (g < N4) {
      a0[k] = ld4(sd.u + 4 * g);
      a1[k] = ld4(sd.v + 4 * g);
      a2[k] = ld4(sd.u2 + 4 * g);
      a3[k] = ld4(sd.v2 + 4 * g);
    }
  }
#pragma unroll
  for (int k = 0; k < kFlatVec; ++k) {
    const int64_t g = g0 + k * kPwThreads;
    if (g >= N4) break;
    float du[4], dv[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      // the increment form (react_diff) in both modes: its rounding is
      // relative to the difference itself
      react_diff<float>(rx, el(a0[k], j), el(a1[k], j), el(a2[k], j), el(a3[k], j), du[j], dv[j]);
    }
    store_pieces_fmt<F>(sd.wu, N, 4 * g, du);
    store_pieces_fmt<F>(sd.wv, N, 4 * g, dv);
  }
}

// Lawson2b (Eq. 7) first pointwise stage, also used for the second:
// W^c = U^c + factor tau G^c(U, V) as BF16 pieces [3][N].
template <int F = kFmtBF16>
__global__ void __launch_bounds__(kPwThreads) lawson_pre_pieces_kernel(const __grid_constant__ PwLaunch L,
                                                                       float factor) {
  FLAT_PROLOGUE
  const ReactionT<float> rx = sd.a.rx;
  const float sc = factor * sd.tau;
  float4 a0[kFlatVec], a1[kFlatVec];
#pragma unroll
  for (int k = 0; k < kFlatVec; ++k) {
    const int64_t g = g0 + k * kPwThreads;
    if (g < N4) {
      a0[k] = ld4(sd.u + 4 * g);
      a1[k] = ld4(sd.v + 4 * g);
    }
  }
#pragma unroll
  for (int k = 0; k < kFlatVec; ++k) {
    const int64_t g = g0 + k * kPwThreads;
    if (g >= N4) break;
    float wu[4], wv[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float uu = el(a0[k], j), vv = el(a1[k], j);
      float gu, gv;
      react<float>(rx, uu, vv, gu, gv);
      wu[j] = uu + sc * gu;
      wv[j] = vv + sc * gv;
    }
    store_pieces_fmt<F>(sd.wu, N, 4 * g, wu);
    store_pieces_fmt<F>(sd.wv, N, 4 * g, wv);
  }
}

// Lawson2b last stage: u += factor tau G(u2, v2) in FP32, in place.
__global__ void __launch_bounds__(kPwThreads) lawson_post_kernel(const __grid_constant__ PwLaunch L, float factor) {
  FLAT_PROLOGUE
  const ReactionT<float> rx = sd.a.rx;
  const float sc = factor * sd.tau;
  float* u = const_cast<float*>(sd.u);
  float* v = const_cast<float*>(sd.v);
  float4 a0[kFlatVec], a1[kFlatVec], a2[kFlatVec], a3[kFlatVec];
#pragma unroll
  for (int k = 0; k < kFlatVec; ++k) {
    const int64_t g = g0 + k * kPwThreads;
    if (g < N4) {
      a0[k] = ld4(sd.u2 + 4 * g);
      a1[k] = ld4(sd.v2 + 4 * g);
      a2[k] = ld4(u + 4 * g);
      a3[k] = ld4(v + 4 * g);
    }
  }
#pragma unroll
  for (int k = 0; k < kFlatVec; ++k) {
    const int64_t g = g0 + k * kPwThreads;
    if (g >= N4) break;
    float ou[4], ov[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      float gu, gv;
      react<float>(rx, el(a0[k], j), el(a1[k], j), gu, gv);
      ou[j] = el(a2[k], j) + sc * gu;
      ov[j] = el(a3[k], j) + sc * gv;
    }
    *reinterpret_cast<float4*>(u + 4 * g) = make_float4(ou[0], ou[1], ou[2], ou[3]);
    *reinterpret_cast<float4*>(v + 4 * g) = make_float4(ov[0], ov[1], ov[2], ov[3]);
  }
}
#undef FLAT_PROLOGUE

// Phi (FP64, row-major n x n) -> three BF16 pieces [3][n][n].
__global__ void split_matrix_kernel(const double* __restrict__ src, __nv_bfloat16* __restrict__ dst,
                                    int64_t count) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double x = src[i];
    const __nv_bfloat16 b0 = __double2bfloat16(x);
    const double r1 = x - (double)__bfloat162float(b0);
    const __nv_bfloat16 b1 = __double2bfloat16(r1);
    const double r2 = r1 - (double)__bfloat162float(b1);
    dst[i] = b0;
    dst[count + i] = b1;
    dst[2 * count + i] = __double2bfloat16(r2);
  }
}

// Phi (FP64, row-major n x n) -> two TF32 pieces [2][n][n] (FP32 words):
// hi = tf32(x), lo = tf32(x - hi) with the difference taken in FP64.
__global__ void split_matrix_tf32_kernel(const double* __restrict__ src, float* __restrict__ dst,
                                         int64_t count) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double x = src[i];
    const float hi = tf32_rna((float)x);
    dst[i] = hi;
    dst[count + i] = tf32_rna((float)(x - (double)hi));
  }
}

// Column support of each 128-row group of an FP64 n x n matrix Phi
// (row-major).  Row i keeps the narrowest column range [lo_i, hi_i) whose
// left-out entries weigh at most drop * sum_j |Phi_ij|, half on each side:
//   lo_i = max { l : sum_{j < l} |Phi_ij| <= t_i },
//   hi_i = min { h : sum_{j >= h} |Phi_ij| <= t_i },   t_i = drop / 2 * sum_j |Phi_ij|.
// A product restricted to the range then differs from the full one by at most
// drop * max|x| * sum_j |Phi_ij| per row.  With drop < 1 the range is never
// empty (the two left-out sums cannot cover the row); an all-zero row keeps
// its diagonal entry.  band[g] = the union over the group's rows, widened to
// multiples of 64 (the end clipped to n).  One block of kBandWarps warps per
// group, one warp per row at a time.
constexpr int kBandRows = 128, kBandWarps = 8;
// Mass of a row of Phi a tile may leave out: 2^-40 of the row's absolute sum,
// far below the 2^-24 relative rounding of the split products themselves.
constexpr double kBandDrop = 9.094947017729282e-13;
__device__ __forceinline__ double warp_incl_scan(double x, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  return x;
}
__global__ void __launch_bounds__(32 * kBandWarps) band_support_kernel(
    const double* __restrict__ A, int n, double drop, int2* __restrict__ band) {
  __shared__ int s_lo, s_hi;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    s_lo = n;
    s_hi = 0;
  }
  __syncthreads();
  const int r_end = min(n, (int)(blockIdx.x + 1) * kBandRows);
  for (int i = blockIdx.x * kBandRows + warp; i < r_end; i += kBandWarps) {
    const double* row = A + (int64_t)i * n;
    double tot = 0.0;
    for (int j = lane; j < n; j += 32) tot += fabs(row[j]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
    int lo = i, hi = i + 1;
    if (tot > 0.0) {
      const double t = 0.5 * drop * tot;
      lo = n - 1;  // left prefix sums: the last l whose prefix before it is <= t
      double run = 0.0;
      for (int c0 = 0; c0 < n; c0 += 32) {
        const int j = c0 + lane;
        const double a = j < n ? fabs(row[j]) : 0.0;
        const double incl = run + warp_incl_scan(a, lane);
        const unsigned over = __ballot_sync(0xffffffffu, j < n && incl - a > t);
        if (over) {
          lo = c0 + __ffs(over) - 2;  // the element before the first prefix above t
          break;
        }
        run = __shfl_sync(0xffffffffu, incl, 31);
      }
      hi = 1;  // right suffix sums: one past the last h whose suffix from it exceeds t
      run = 0.0;
      for (int c0 = 0; c0 < n; c0 += 32) {
        const int j = n - 1 - c0 - lane;
        const double a = j >= 0 ? fabs(row[j]) : 0.0;
        const double incl = run + warp_incl_scan(a, lane);
        const unsigned over = __ballot_sync(0xffffffffu, j >= 0 && incl > t);
        if (over) {
          hi = n - c0 - __ffs(over) + 1;
          break;
        }
        run = __shfl_sync(0xffffffffu, incl, 31);
      }
    }
    if (lane == 0) {
      atomicMin(&s_lo, lo);
      atomicMax(&s_hi, hi);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) band[blockIdx.x] = make_int2(s_lo & ~63, min(n, (s_hi + 63) & ~63));
}

// ---------------------------------------------------------------- host side
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

cudaError_t get_encoder() {
  if (g_encode) return cudaSuccess;
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                   cudaEnableDefault, &q);
  if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
  g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
  return cudaSuccess;
}

// [3][rows][K] BF16 pieces, box {SW/2, box_rows, 3}, SW-byte swizzle: one
// copy brings a K chunk of all three pieces of a tile, laid out in shared
// memory as [piece][row][SW bytes].  (The copy engine's cost is largely per
// instruction, so one large box moves data much faster than three small ones.)
// TF32 pieces: [2][rows][K] FP32 words, box {SW/4, box_rows, 2}.
cudaError_t encode_pieces(CUtensorMap* map, const void* base, int64_t K, int64_t rows,
                          int box_rows, int sw, int fmt = kFmtBF16) {
  const int np = fmt == kFmtTF32 ? 2 : kPieces, esz = fmt == kFmtTF32 ? 4 : 2;
  cuuint64_t dims[3] = {(cuuint64_t)K, (cuuint64_t)rows, (cuuint64_t)np};
  cuuint64_t strides[2] = {(cuuint64_t)K * esz, (cuuint64_t)(K * rows) * esz};
  cuuint32_t box[3] = {(cuuint32_t)(sw / esz), (cuuint32_t)box_rows, (cuuint32_t)np};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = g_encode(map, fmt == kFmtTF32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16,
                        3, const_cast<void*>(base), dims,
                        strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        sw == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// [3][K][M] BF16 pieces read MN-major (M contiguous): box {64, bk, 3} with
// 128-byte swizzle, two boxes per 128-row tile.
cudaError_t encode_pieces_mn(CUtensorMap* map, const void* base, int64_t M, int64_t K, int bk) {
  cuuint64_t dims[3] = {(cuuint64_t)M, (cuuint64_t)K, (cuuint64_t)kPieces};
  cuuint64_t strides[2] = {(cuuint64_t)M * 2, (cuuint64_t)(M * K) * 2};
  cuuint32_t box[3] = {64, (cuuint32_t)bk, (cuuint32_t)kPieces};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims,
                        strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// Kernel variants (swizzle width, tile width, CTA pair).  Pair variants run
// tc_pair_kernel: 256-row tiles over two SMs.
struct Variant {
  int sw, bn, cta2;
};
constexpr Variant kVariants[] = {{64, 128, 0}, {128, 128, 0}, {64, 64, 0}, {64, 128, 1}, {128, 128, 1}};
constexpr int kNumVariants = 5;
constexpr int tile_rows(int variant) { return kVariants[variant].cta2 ? 2 * kBM : kBM; }

template <int SW, int BN>
cudaError_t set_smem_attr() {
  const int sm = TcCfg<SW, BN>::SMEM;
  cudaError_t e = cudaFuncSetAttribute(tc_mode_kernel<SW, BN, false, false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(tc_mode_kernel<SW, BN, true, false>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(tc_mode_kernel<SW, BN, false, true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(tc_mode_kernel<SW, BN, false, false, kFmtBF16, true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  return e;
}
template <int SW>
cudaError_t set_smem_attr_pair() {
  cudaError_t e = cudaFuncSetAttribute(tc_pair_kernel<SW>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, Tc2Cfg<SW>::SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(tc_pair_kernel<SW, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             Tc2Cfg<SW>::SMEM);
  return e;
}

// Programmatic dependent launch for the kernels of a step (ADR_PDL=0 turns
// it off: every kernel then waits for the previous one to finish).
static bool pdl_enabled() {
  static const int on = [] {
    const char* e = getenv("ADR_PDL");
    return e ? atoi(e) : 1;
  }();
  return on != 0;
}

template <typename... KArgs, typename... Args>
cudaError_t launch_k(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                     Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl_enabled() ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

template <bool PAIR, bool IND = false>
cudaError_t launch_tc_t(int v, dim3 grid, cudaStream_t s, const TcLaunch& L) {
  switch (v) {
    case 0:
      return launch_k(tc_mode_kernel<64, 128, PAIR, false, kFmtBF16, IND>, grid, dim3(kThreads),
                      TcCfg<64, 128>::SMEM, s, L);
    case 1:
      return launch_k(tc_mode_kernel<128, 128, PAIR, false, kFmtBF16, IND>, grid, dim3(kThreads),
                      TcCfg<128, 128>::SMEM, s, L);
    case 2:
      return launch_k(tc_mode_kernel<64, 64, PAIR, false, kFmtBF16, IND>, grid, dim3(kThreads),
                      TcCfg<64, 64>::SMEM, s, L);
    default:
      return cudaErrorInvalidValue;
  }
}

// The kStage1X pass: clusters of two CTAs (u and v of one tile).
template <int SW, int BN>
cudaError_t launch_xchg_t(int clusters, cudaStream_t s, const TcLaunch& L) {
  const int pairs = L.nunits / 2;
  const int nc = pairs < clusters ? pairs : clusters;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(2 * nc));
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = TcCfg<SW, BN>::SMEM;
  cfg.stream = s;
  cudaLaunchAttribute at[2];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 2;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl_enabled() ? 2 : 1;
  return cudaLaunchKernelEx(&cfg, tc_mode_kernel<SW, BN, false, true>, L);
}
cudaError_t launch_xchg(int v, int clusters, cudaStream_t s, const TcLaunch& L) {
  if (L.nunits <= 0) return cudaSuccess;
  switch (v) {
    case 0:
      return launch_xchg_t<64, 128>(clusters, s, L);
    case 1:
      return launch_xchg_t<128, 128>(clusters, s, L);
    case 2:
      return launch_xchg_t<64, 64>(clusters, s, L);
    default:
      return cudaErrorInvalidValue;
  }
}
// Clusters of the XCHG kernel that fit on the GPU at once.
int xchg_clusters(int v) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(2);
  cfg.blockDim = dim3(kThreads);
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 2;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int n = 0;
  cudaError_t e = cudaErrorInvalidValue;
  if (v == 0) {
    cfg.dynamicSmemBytes = TcCfg<64, 128>::SMEM;
    e = cudaOccupancyMaxActiveClusters(&n, tc_mode_kernel<64, 128, false, true>, &cfg);
  } else if (v == 1) {
    cfg.dynamicSmemBytes = TcCfg<128, 128>::SMEM;
    e = cudaOccupancyMaxActiveClusters(&n, tc_mode_kernel<128, 128, false, true>, &cfg);
  } else if (v == 2) {
    cfg.dynamicSmemBytes = TcCfg<64, 64>::SMEM;
    e = cudaOccupancyMaxActiveClusters(&n, tc_mode_kernel<64, 64, false, true>, &cfg);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

// pair: the launch's units are (u, v) pairs (the fused stage-1 epilogue).
// A pair-variant launch: clusters of two CTAs, at most `clusters` of them
// (the number that fit on the GPU at once).
template <int SW, bool IND = false>
cudaError_t launch_pair(int clusters, cudaStream_t s, const TcLaunch& L) {
  const int nc = L.nunits < clusters ? L.nunits : clusters;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(2 * nc));
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = Tc2Cfg<SW>::SMEM;
  cfg.stream = s;
  cudaLaunchAttribute at[2];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 2;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl_enabled() ? 2 : 1;
  return cudaLaunchKernelEx(&cfg, tc_pair_kernel<SW, IND>, L);
}

// Clusters of the pair kernel that can be resident at once.
int pair_clusters(int variant) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(2);
  cfg.blockDim = dim3(kThreads);
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 2;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int n = 0;
  cudaError_t e;
  if (kVariants[variant].sw == 64) {
    cfg.dynamicSmemBytes = Tc2Cfg<64>::SMEM;
    e = cudaOccupancyMaxActiveClusters(&n, tc_pair_kernel<64>, &cfg);
  } else {
    cfg.dynamicSmemBytes = Tc2Cfg<128>::SMEM;
    e = cudaOccupancyMaxActiveClusters(&n, tc_pair_kernel<128>, &cfg);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

// pair: the launch's units are (u, v) pairs (the fused stage-1 epilogue).
// slots: resident CTAs (one-CTA variants) or clusters (pair variants).
// ind: the pass accumulates the step's indicators.
cudaError_t launch_tc(int v, int slots, cudaStream_t s, const TcLaunch& L, bool pair, bool ind) {
  if (L.nunits <= 0) return cudaSuccess;
  if (kVariants[v].cta2) {
    if (ind)
      return kVariants[v].sw == 64 ? launch_pair<64, true>(slots, s, L)
                                   : launch_pair<128, true>(slots, s, L);
    return kVariants[v].sw == 64 ? launch_pair<64>(slots, s, L) : launch_pair<128>(slots, s, L);
  }
  dim3 grid((unsigned)(L.nunits < slots ? L.nunits : slots));
  if (ind) return launch_tc_t<false, true>(v, grid, s, L);
  return pair ? launch_tc_t<true>(v, grid, s, L) : launch_tc_t<false>(v, grid, s, L);
}

// The fused two-mode kernel: one CTA per SM at most (all of TMEM each).
cudaError_t launch_fused(int slots, cudaStream_t s, const TcLaunch& L, bool ind) {
  if (L.nunits <= 0) return cudaSuccess;
  const dim3 grid((unsigned)(L.nunits < slots ? L.nunits : slots));
  if (ind) return launch_k(tc_fused_kernel<true>, grid, dim3(kThreads), kFSmem, s, L);
  return launch_k(tc_fused_kernel<false>, grid, dim3(kThreads), kFSmem, s, L);
}

int grid_for(int64_t total) {
  int64_t b = (total + 255) / 256;
  if (b < 1) b = 1;
  if (b > 152 * 16) b = 152 * 16;
  return (int)b;
}

// One tensor-core pass of the step sequence.
enum { kOutPieces = 0, kOutStage = 1, kOutState = 2 };   // outputs: pieces, U2/V2, u/v
enum { kBaseNone = 0, kBaseState = 1, kBaseStage = 2 };  // FP32 base: none, u/v, U2/V2
enum { kAlphaOne = 0, kAlphaTau = 1, kAlphaTauD = 2 };   // 1, tau, 2^(d-1) tau
struct TcPass {
  int b;      // piece buffer read (output pieces go to 1 - b)
  int mu;     // direction
  int ell;    // matrix: 0 = e^(tau A), 1 = phi_1, 2 = phi_2
  int mode;   // TcMode
  int pair;
  int out, base, alpha;
  int fused;  // 1: modes 1 and 2 in one launch (tc_fused_kernel); mu = 0
  int amn;    // 1: reads the fused pass's natural-layout pieces as an MN-major A (mu = 2)
};

// One launch of the step sequence.
enum { kOpRhs = 0, kOpTc = 1, kOpRdiff = 2, kOpLawsonPre = 3, kOpLawsonPost = 4 };
struct TcOp {
  int kind;
  int pass;       // kOpTc: index into the passes
  float factor;   // Lawson stages: multiple of tau
};

}  // namespace

constexpr int kIndSlots = 4096;  // steps of indicator history a plan keeps

// Host-side state of the tensor-core path of one plan (owned through TcOperands).
struct TcState {
  int d;
  int64_t n[3];
  int64_t N;
  __nv_bfloat16* phi[2][3][3];   // [c][mu][ell] -> [3][n][n]; ell 0 = e^(tau A)
  __nv_bfloat16* buf[2][2];      // [b][c] -> [3][N]
  CUtensorMap amap[2][2][3];     // [b][c][mu]: buffer b viewed as [3][N/n_mu][n_mu]
  CUtensorMap bmap[2][3][3];     // [c][mu][ell]
  // column supports of the 128-row groups of each Phi (device, inside the
  // cached piece buffer; host copies for the work accounting); kband null
  // when the supports are off (every tile contracts over all of K)
  const int2* kband[2][3][3];
  std::vector<int2> hband[2][3][3];
  int ksupport;
  // fused two-mode passes (2D, BF16 pieces): Phi of directions 1 and 2 with
  // 128-row boxes, and each piece buffer as W with kFRowsW-row boxes
  int fused12;
  CUtensorMap fa[2][3], fc[2][3];  // [c][ell]
  CUtensorMap fw[2][2];            // [b][c]
  CUtensorMap amn_map[2][2];       // [b][c] 3D: buffer b as [piece][x3][x2 x1], 64 x BK boxes
  int variant;
  int fmt;       // operand format: kFmtBF16 (three BF16 pieces) or kFmtTF32 (two TF32 pieces)
  int fuse;      // 1: fuse the stage-1 combination into the last stage-1 product
  int num_sms;
  std::vector<void*> shared;  // operand pieces held in the process-wide cache
  int slots;     // resident CTAs (or CTA pairs) of the mode-product kernel
  int xslots;    // resident clusters of the exchanging (kStage1X) kernel
  int* err;
  std::vector<void*> allocs;
  // step sequence: tensor-core passes and the launches around them
  int scheme;
  std::vector<TcPass> passes;
  std::vector<TcOp> ops;
  // descriptors of this plan as a group of one, bound to (bound_u, bound_v);
  // they travel in the kernel parameters of every launch
  std::vector<TcPassDesc> h_desc;  // [passes]
  PwDesc h_pw;
  int units[8];
  int rhs_blocks, rdiff_blocks;
  void* bound_u;
  void* bound_v;
  // compensated state: low-order words per component [N], valid for the
  // state pair (comp_u, comp_v); null when the plan carries a plain state.
  // comp: 0 plain; 2 compensated (hi + lo state, double-float reactions)
  int comp;
  float* lo[2];
  void* comp_u;
  void* comp_v;
  // indicators of Sec. 4 per step (null when off): ring [kIndSlots][4] of
  // sums (w u, w v, |dU|^2, |dV|^2) and the step counter
  double* ind;
  int64_t* ind_ctr;
};

static int units_of(const TcState* S, const TcPass& ps, int bn) {
  if (ps.fused) {  // one unit per j1 tile and (when n2 > 256) j2 tile
    const int64_t n1 = S->n[0], n2 = S->n[1], slabs = S->N / (n1 * n2);
    return (int)(2 * slabs * ((n1 + kBM - 1) / kBM) * (n2 <= kFRowsW ? 1 : (n2 + kBM - 1) / kBM));
  }
  const int64_t nmu = S->n[ps.mu];
  const int64_t M = S->N / nmu;
  const int bm = tile_rows(S->variant);
  const int tm = (int)((M + bm - 1) / bm), tn = (int)((nmu + bn - 1) / bn);
  return (ps.pair ? 1 : 2) * tm * tn;
}

static TcPassDesc make_desc(const TcState* S, const adr_plan_s* P, const TcPass& ps, float* u,
                            float* v) {
  TcPassDesc D;
  memset(&D, 0, sizeof(D));
  const int bn = kVariants[S->variant].bn;
  const int64_t nmu = S->n[ps.mu];
  D.M = (int)(S->N / nmu);
  D.N = (int)nmu;
  D.K = (int)nmu;
  D.tiles_m = (D.M + tile_rows(S->variant) - 1) / tile_rows(S->variant);
  D.tiles_n = (D.N + bn - 1) / bn;
  D.pair = ps.pair;
  D.mode = ps.mode;
  D.amn = ps.amn;
  D.rx = P->pwf.rx;
  float* stage[2] = {(float*)P->u2, (float*)P->v2};
  float* state[2] = {u, v};
  const double tau = P->prob.tau;
  for (int c = 0; c < 2; ++c) {
    D.amap[c] = ps.amn ? S->amn_map[ps.b][c] : S->amap[ps.b][c][ps.mu];
    D.bmap[c] = S->bmap[c][ps.mu][ps.ell];
    D.kband[c] = S->ksupport ? S->kband[c][ps.mu][ps.ell] : nullptr;
    D.outp[c] = S->buf[1 - ps.b][c];
    D.outf[c] = ps.out == kOutStage ? stage[c] : (ps.out == kOutState ? state[c] : nullptr);
    D.base[c] = ps.base == kBaseStage ? stage[c] : (ps.base == kBaseState ? state[c] : nullptr);
    // the stage updates U2 = U + tau T and U+ = U2 + 2^(d-1) tau S of a
    // compensated state carry the low-order words (stage 1 leaves U2's in
    // place of U's, stage 2 replaces them by U+'s)
    D.lo[c] = (S->comp && ps.mode == kAxpy && !ps.pair) ? S->lo[c] : nullptr;
  }
  // the last product of an ETD2RKds step writes the new state: it adds the
  // step's indicator sums
  if (S->ind && S->scheme == ADR_ETD2RKDS && ps.mode == kAxpy && ps.out == kOutState && !ps.pair) {
    D.ind = S->ind;
    D.ind_ctr = S->ind_ctr;
    D.ind_k = kIndSlots;
    D.ind_n1 = (int)S->n[0];
    D.ind_n2 = S->d == 3 ? (int)S->n[1] : 0;
  }
  D.alpha = ps.alpha == kAlphaTau ? (float)tau
                                  : (ps.alpha == kAlphaTauD ? (float)ldexp(tau, S->d - 1) : 1.0f);
  if (ps.fused) {  // modes 1 and 2: Phi_a = direction 1, Phi_b = direction 2, W = buffer b
    D.n1 = (int)S->n[0];
    D.n2 = (int)S->n[1];
    D.slabs = (int)(S->N / (S->n[0] * S->n[1]));
    D.M = D.n1;
    D.N = D.n2;
    D.K = D.n1;
    D.tiles_m = (D.n1 + kBM - 1) / kBM;
    D.tiles_n = (D.n2 + kBM - 1) / kBM;
    D.bunit = D.n2 <= kFRowsW ? D.tiles_n : 1;  // the tiles of x2 share one intermediate
    for (int c = 0; c < 2; ++c) {
      D.amap[c] = S->fa[c][ps.ell];
      D.bmap[c] = S->fw[ps.b][c];
      D.cmap[c] = S->fc[c][ps.ell];
      D.kband[c] = S->ksupport ? S->kband[c][0][ps.ell] : nullptr;
      D.kband2[c] = S->ksupport ? S->kband[c][1][ps.ell] : nullptr;
    }
  }
  return D;
}

// Stencil geometry of a solve (see PwDesc).  share = the solve's fraction
// of the points of its launch (1 for a single solve), so that a batch's
// blocks together fill the GPU about as one large solve does.
// 3D: one block per kRingX x kRingY tile and z run; the runs are cut so that
// the blocks fill about two waves of two blocks per SM, and hold at least
// four planes (each run reads two planes beyond its own).
// 2D: one warp per 128 x-points and z run; the runs are long enough to
// reuse the z neighbours and short enough to leave several warps per SM.
struct PwGeom {
  int nx, ny, nz, xsegs, ytiles, zlen, zsegs;
  int64_t sy, sz;
};
static PwGeom pw_geom(const TcState* S, int num_sms, double share) {
  PwGeom g;
  const bool d3 = S->d == 3;
  g.nx = (int)S->n[0];
  g.sy = S->n[0];
  if (d3) {
    g.ny = (int)S->n[1];
    g.nz = (int)S->n[2];
    g.sz = S->n[0] * S->n[1];
    g.xsegs = (g.nx + kRingX - 1) / kRingX;
    g.ytiles = (g.ny + kRingY - 1) / kRingY;
    const int64_t cols = (int64_t)g.xsegs * g.ytiles;
    const int64_t want = std::max<int64_t>(1, (int64_t)(num_sms * 2 * 2 * share + 0.5));
    int64_t segs = (want + cols - 1) / cols;
    if (segs > g.nz) segs = g.nz;
    int64_t zl = (g.nz + segs - 1) / segs;
    if (zl < 4) zl = 4;
    g.zlen = (int)zl;
    g.zsegs = (g.nz + g.zlen - 1) / g.zlen;
    return g;
  }
  g.ny = 1;
  g.nz = (int)S->n[1];
  g.sz = S->n[0];
  g.ytiles = 1;
  g.xsegs = (g.nx + kSegX - 1) / kSegX;
  // z runs: a multiple of the planes per iteration, as long as leaves about
  // four waves of 16 warps per SM (whole waves balance the SMs; each warp
  // keeps several planes of loads in flight), at most 64 planes
  const int zb = kZB2;
  const int64_t cols = g.xsegs;
  const int64_t want = std::max<int64_t>(1, (int64_t)(num_sms * 16 * 4 * share + 0.5));
  int64_t zl = (cols * g.nz + want - 1) / want;
  zl = ((zl + zb - 1) / zb) * zb;
  if (zl < zb) zl = zb;
  if (zl > 64) zl = 64;
  g.zlen = (int)zl;
  g.zsegs = (g.nz + g.zlen - 1) / g.zlen;
  return g;
}

// 3D state field [nz][ny][nx] FP32 for the stencil's plane copies: box
// {kRingBoxX, kRingBoxY, 1}, zero fill outside the grid.
static cudaError_t encode_field(CUtensorMap* map, const float* base, const PwGeom& g) {
  cuuint64_t dims[3] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz};
  cuuint64_t strides[2] = {(cuuint64_t)g.sy * 4, (cuuint64_t)g.sz * 4};
  cuuint32_t box[3] = {(cuuint32_t)kRingBoxX, (cuuint32_t)kRingBoxY, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(base), dims,
                        strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

static cudaError_t make_pw(const TcState* S, const adr_plan_s* P, float* u, float* v, PwDesc* out,
                           double share = 1.0) {
  PwDesc& W = *out;
  memset(&W, 0, sizeof(W));
  W.a = P->pwf;
  W.u = u;
  W.v = v;
  W.u2 = (const float*)P->u2;
  W.v2 = (const float*)P->v2;
  W.wu = S->buf[0][0];
  W.wv = S->buf[0][1];
  W.tau = (float)P->prob.tau;
  W.ind = S->ind;
  W.ind_ctr = S->ind_ctr;
  W.ind_k = kIndSlots;
  const PwGeom g = pw_geom(S, S->num_sms, share);
  W.nx = g.nx;
  W.ny = g.ny;
  W.nz = g.nz;
  W.xsegs = g.xsegs;
  W.ytiles = g.ytiles;
  W.zlen = g.zlen;
  W.zsegs = g.zsegs;
  W.sy = g.sy;
  W.sz = g.sz;
  if (S->d == 3) {
    cudaError_t e = encode_field(&W.tu, u, g);
    if (e == cudaSuccess) e = encode_field(&W.tv, v, g);
    return e;
  }
  return cudaSuccess;
}

static int rhs_blocks_of(const TcState* S, double share = 1.0) {
  const PwGeom g = pw_geom(S, S->num_sms, share);
  if (S->d == 3) return g.xsegs * g.ytiles * g.zsegs;
  const int64_t warps = (int64_t)g.xsegs * g.zsegs;
  return (int)((warps + kPwWarps - 1) / kPwWarps);
}
static int rdiff_blocks_of(const TcState* S) {
  return (int)((S->N + kFlatPerBlock - 1) / kFlatPerBlock);
}

void tc_init(TcOperands* t) { memset(t, 0, sizeof(*t)); }

void tc_free(TcOperands* t) {
  TcState* S = (TcState*)t->work[0];
  if (S) {
    for (void* p : S->allocs) cudaFree(p);
    for (void* p : S->shared) shared_release(p);
    delete S;
  }
  t->work[0] = nullptr;
}

cudaError_t tc_prepare(TcOperands* t, int prec, int scheme, int d, const int64_t n[3],
                       double* const master[2][3][4], cudaStream_t s, int variant_req, int comp) {
  if (prec != ADR_BF16X3 && prec != ADR_TF32X3) return cudaErrorNotSupported;
  for (int m = 0; m < d; ++m)
    if (n[m] % 8 != 0) return cudaErrorNotSupported;  // TMA row strides: 16-byte multiples
  cudaError_t e = get_encoder();
  if (e != cudaSuccess) return e;
  static bool attr_set = false;
  if (!attr_set) {
    if ((e = set_smem_attr<64, 128>()) != cudaSuccess) return e;
    if ((e = set_smem_attr<128, 128>()) != cudaSuccess) return e;
    if ((e = set_smem_attr<64, 64>()) != cudaSuccess) return e;
    if ((e = set_smem_attr_pair<64>()) != cudaSuccess) return e;
    if ((e = set_smem_attr_pair<128>()) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(tc_fused_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  kFSmem)) != cudaSuccess)
      return e;
    if ((e = cudaFuncSetAttribute(tc_fused_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  kFSmem)) != cudaSuccess)
      return e;
    if ((e = cudaFuncSetAttribute(tc_mode_kernel<128, 128, false, false, kFmtTF32>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  TcCfg<128, 128, kFmtTF32>::SMEM)) != cudaSuccess)
      return e;
    if ((e = cudaFuncSetAttribute(tc_mode_kernel<128, 128, false, false, kFmtTF32, true>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  TcCfg<128, 128, kFmtTF32>::SMEM)) != cudaSuccess)
      return e;
    if ((e = cudaFuncSetAttribute(rhs3_ring_kernel<kFmtBF16, true>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, kRingSmem)) != cudaSuccess)
      return e;
    if ((e = cudaFuncSetAttribute(rhs3_ring_kernel<kFmtTF32, true>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, kRingSmem)) != cudaSuccess)
      return e;
    if ((e = cudaFuncSetAttribute(rhs3_ring_kernel<kFmtBF16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  kRingSmem)) != cudaSuccess)
      return e;
    if ((e = cudaFuncSetAttribute(rhs3_ring_kernel<kFmtTF32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  kRingSmem)) != cudaSuccess)
      return e;
    attr_set = true;
  }
  TcState* S = new TcState();
  t->work[0] = S;
  t->prec = prec;
  // Tiles contract over the column support of their rows of Phi (ADR_KSUPPORT=0: all of K)
  S->ksupport = 1;
  if (const char* ev = getenv("ADR_KSUPPORT")) S->ksupport = atoi(ev) != 0;
  S->d = d;
  S->fmt = prec == ADR_TF32X3 ? kFmtTF32 : kFmtBF16;
  // Default kernel: on grids of about a million points and more, the
  // CTA-pair kernel (256 x 128 tiles over two SMs, 128-byte swizzle, three
  // 72 KB stages: the tensor pipe stays fed, and each SM streams half of B);
  // on smaller grids one CTA per 128 x 128 tile with 64-byte swizzle and four
  // 48 KB stages, whose smaller tiles waste less.  A batch mixing the two runs
  // one grouped launch sequence per kernel.  ADR_TC_VARIANT overrides.
  {
    int64_t npts = 1;
    for (int m = 0; m < d; ++m) npts *= n[m];
    S->variant = npts >= 1000000 ? 4 : 0;
  }
  if (variant_req >= 0 && variant_req < kNumVariants) S->variant = variant_req;
  if (const char* ev = getenv("ADR_TC_VARIANT")) {
    const int v = atoi(ev);
    if (v >= 0 && v < kNumVariants) S->variant = v;
  }
  // the fused stage-1 epilogue is kept behind ADR_TC_FUSE=1 until it beats
  // the separate reaction-difference kernel on large grids
  // Stage-1 reaction difference: 0 = separate kernel, 1 = pair units (u and
  // v of a tile in one CTA), 2 = clusters of two CTAs exchanging U2 and V2.
  S->fuse = 0;
  if (const char* ev = getenv("ADR_TC_FUSE")) {
    const int f = atoi(ev);
    S->fuse = f >= 0 && f <= 2 ? f : 0;
  }
  if (kVariants[S->variant].cta2) S->fuse = 0;  // the CTA-pair kernel has neither epilogue
  // BF16 pieces: the first two directions of each Tucker operator as one
  // fused launch (2D: the whole operator; 3D: then the x3 product on the
  // fused pass's natural-layout output read MN-major).  ADR_TC_FUSED=0: one
  // launch per direction.
  S->fused12 = (d == 2 || d == 3) && prec == ADR_BF16X3;
  if (const char* ev = getenv("ADR_TC_FUSED")) S->fused12 = S->fused12 && atoi(ev) != 0;
  if (S->fused12) S->fuse = 0;
  S->comp = scheme == ADR_ETD2RKDS ? comp : 0;
  if (S->comp) S->fuse = 0;  // the fused stage-1 epilogues keep a plain state
  if (S->fmt == kFmtTF32) {  // TF32 pieces: the one-CTA kernel, 128-byte swizzle, plain epilogues
    S->variant = 1;
    S->fuse = 0;
  }
  int dev = 0;
  cudaGetDevice(&dev);
  S->num_sms = 148;
  cudaDeviceGetAttribute(&S->num_sms, cudaDevAttrMultiProcessorCount, dev);
  S->slots = S->num_sms;
  if (kVariants[S->variant].cta2) {
    S->slots = pair_clusters(S->variant);
    if (S->slots <= 0) {  // no room for clusters of two: the one-CTA kernel
      S->variant = 0;
      S->slots = S->num_sms;
    }
  }
  S->xslots = 0;
  if (S->fuse == 2) {
    S->xslots = xchg_clusters(S->variant);
    if (S->xslots <= 0) S->fuse = 0;  // clusters unavailable: separate kernel
  }
  const int sw = kVariants[S->variant].sw, bn = kVariants[S->variant].bn;
  S->N = 1;
  for (int m = 0; m < 3; ++m) S->n[m] = m < d ? n[m] : 1;
  for (int m = 0; m < d; ++m) S->N *= n[m];
  auto alloc = [&](void** p, size_t bytes) -> cudaError_t {
    cudaError_t r = cudaMalloc(p, bytes);
    if (r == cudaSuccess) S->allocs.push_back(*p);
    return r;
  };
  e = alloc((void**)&S->err, sizeof(int));
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(S->err, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  for (int c = 0; c < 2; ++c)
    for (int m = 0; m < d; ++m)
      for (int l = 0; l < 3; ++l) {
        if ((scheme == ADR_LAWSON2B) != (l == 0)) continue;  // only the matrices the scheme uses
        const int64_t nn = n[m] * n[m];
        const size_t pb = S->fmt == kFmtTF32 ? 2 * 4 : (size_t)kPieces * 2;  // piece bytes per value
        const int nbands = (int)((n[m] + kBandRows - 1) / kBandRows);
        // the pieces of a cached FP64 matrix, followed by the column supports
        // of its row groups, are cached with it (keyed by that matrix and the
        // piece format); pb * nn is a multiple of 8 bytes
        const double* src = master[c][m][1 + l];
        const std::vector<uint64_t> key = {1, (uint64_t)(uintptr_t)src, (uint64_t)S->fmt,
                                           (uint64_t)nn};
        void* buf = nullptr;
        bool hit = false;
        e = shared_acquire(key, 1, pb * nn + sizeof(int2) * nbands, [&](void* const* b) {
          if (S->fmt == kFmtTF32)
            split_matrix_tf32_kernel<<<grid_for(nn), 256, 0, s>>>(src, (float*)b[0], nn);
          else
            split_matrix_kernel<<<grid_for(nn), 256, 0, s>>>(src, (__nv_bfloat16*)b[0], nn);
          band_support_kernel<<<nbands, 32 * kBandWarps, 0, s>>>(
              src, (int)n[m], kBandDrop, (int2*)((uint8_t*)b[0] + pb * nn));
          return cudaGetLastError();
        }, s, &buf, &hit);
        if (e != cudaSuccess) return e;
        S->shared.push_back(buf);
        S->phi[c][m][l] = (__nv_bfloat16*)buf;
        S->kband[c][m][l] = (const int2*)((uint8_t*)buf + pb * nn);
        S->hband[c][m][l].resize(nbands);
        e = encode_pieces(&S->bmap[c][m][l], S->phi[c][m][l], n[m], n[m],
                          kVariants[S->variant].cta2 ? bn / 2 : bn, sw, S->fmt);
        if (e != cudaSuccess) return e;
      }
  S->lo[0] = S->lo[1] = nullptr;
  S->comp_u = S->comp_v = nullptr;
  S->ind = nullptr;
  S->ind_ctr = nullptr;
  if (S->comp)
    for (int c = 0; c < 2; ++c) {
      e = alloc((void**)&S->lo[c], sizeof(float) * S->N);
      if (e != cudaSuccess) return e;
      e = cudaMemsetAsync(S->lo[c], 0, sizeof(float) * S->N, s);
      if (e != cudaSuccess) return e;
    }
  for (int b = 0; b < 2; ++b)
    for (int c = 0; c < 2; ++c) {
      e = alloc((void**)&S->buf[b][c], (S->fmt == kFmtTF32 ? 8 : (size_t)kPieces * 2) * S->N);
      if (e != cudaSuccess) return e;
      for (int m = 0; m < d; ++m) {
        e = encode_pieces(&S->amap[b][c][m], S->buf[b][c], n[m], S->N / n[m], kBM, sw, S->fmt);
        if (e != cudaSuccess) return e;
      }
    }
  if (S->fused12) {
    for (int c = 0; c < 2; ++c) {
      for (int l = 0; l < 3; ++l) {
        if (!S->phi[c][0][l]) continue;
        e = encode_pieces(&S->fa[c][l], S->phi[c][0][l], n[0], n[0], kBM, 64, S->fmt);
        if (e == cudaSuccess)
          e = encode_pieces(&S->fc[c][l], S->phi[c][1][l], n[1], n[1], kBM, 64, S->fmt);
        if (e != cudaSuccess) return e;
      }
      for (int b = 0; b < 2; ++b) {
        e = encode_pieces(&S->fw[b][c], S->buf[b][c], n[0], S->N / n[0], kFRowsW, 64, S->fmt);
        if (e == cudaSuccess && d == 3)
          e = encode_pieces_mn(&S->amn_map[b][c], S->buf[b][c], S->N / n[2], n[2], sw / 2);
        if (e != cudaSuccess) return e;
      }
    }
  }
  // step sequence (piece buffers alternate; pointwise stages write buffer 0)
  S->scheme = scheme;
  auto add_tucker = [&](int ell, int last_out, int last_base, int last_alpha, int stage1_fuse) {
    int b = 0;
    if (S->fused12) {  // reads buffer 0; 2D: writes the operator's result
      if (d == 3) {    // modes 1 and 2 to pieces in buffer 1, then mode 3 from them
        TcPass f{0, 0, ell, kPieces3, 0, kOutPieces, kBaseNone, kAlphaOne, 1, 0};
        S->passes.push_back(f);
        S->ops.push_back({kOpTc, (int)S->passes.size() - 1, 0.f});
        TcPass m3{1, 2, ell, kAxpy, 0, last_out, last_base, last_alpha, 0, 1};
        S->passes.push_back(m3);
      } else {
        TcPass f{0, 0, ell, kAxpy, 0, last_out, last_base, last_alpha, 1, 0};
        S->passes.push_back(f);
      }
      S->ops.push_back({kOpTc, (int)S->passes.size() - 1, 0.f});
      return 1;
    }
    for (int mu = 0; mu < d; ++mu) {
      TcPass ps{b, mu, ell, kPieces3, 0, kOutPieces, kBaseNone, kAlphaOne};
      if (mu == d - 1) {
        ps.mode = stage1_fuse == 1 ? kStage1 : (stage1_fuse == 2 ? kStage1X : kAxpy);
        ps.pair = stage1_fuse == 1;
        ps.out = last_out;
        ps.base = last_base;
        ps.alpha = last_alpha;
      }
      S->passes.push_back(ps);
      S->ops.push_back({kOpTc, (int)S->passes.size() - 1, 0.f});
      b ^= 1;
    }
    return b;
  };
  if (scheme == ADR_LAWSON2B) {
    // U2 = (U + tau G) x e^(tau A);  U+ = (U + tau/2 G) x e^(tau A) + tau/2 G(U2, V2)
    S->ops.push_back({kOpLawsonPre, -1, 1.0f});
    add_tucker(0, kOutStage, kBaseNone, kAlphaOne, 0);
    S->ops.push_back({kOpLawsonPre, -1, 0.5f});
    add_tucker(0, kOutState, kBaseNone, kAlphaOne, 0);
    S->ops.push_back({kOpLawsonPost, -1, 0.5f});
  } else {
    // ETD2RKds: stencil, phi_1 Tucker to U2 (+ reaction difference), phi_2
    // Tucker back to the state
    S->ops.push_back({kOpRhs, -1, 0.f});
    const int b1 = add_tucker(1, kOutStage, kBaseState, kAlphaTau, S->fuse);
    if (!S->fuse) S->ops.push_back({kOpRdiff, -1, 0.f});
    // stage 2 reads the reaction difference from buffer 0 (separate kernel)
    // or from the buffer the fused epilogue wrote
    const int b2 = S->fuse ? b1 : 0;
    if (S->fused12) {
      if (d == 3) {
        TcPass f{b2, 0, 2, kPieces3, 0, kOutPieces, kBaseNone, kAlphaOne, 1, 0};
        S->passes.push_back(f);
        S->ops.push_back({kOpTc, (int)S->passes.size() - 1, 0.f});
        TcPass m3{1 - b2, 2, 2, kAxpy, 0, kOutState, kBaseStage, kAlphaTauD, 0, 1};
        S->passes.push_back(m3);
      } else {
        TcPass f{b2, 0, 2, kAxpy, 0, kOutState, kBaseStage, kAlphaTauD, 1, 0};
        S->passes.push_back(f);
      }
      S->ops.push_back({kOpTc, (int)S->passes.size() - 1, 0.f});
    }
    for (int mu = 0, b = b2; mu < d && !S->fused12; ++mu, b ^= 1) {
      TcPass ps{b, mu, 2, kPieces3, 0, kOutPieces, kBaseNone, kAlphaOne};
      if (mu == d - 1) {
        ps.mode = kAxpy;
        ps.out = kOutState;
        ps.base = kBaseStage;
        ps.alpha = kAlphaTauD;
      }
      S->passes.push_back(ps);
      S->ops.push_back({kOpTc, (int)S->passes.size() - 1, 0.f});
    }
  }
  const int np = (int)S->passes.size();
  for (int p = 0; p < np; ++p) S->units[p] = units_of(S, S->passes[p], bn);
  S->rhs_blocks = rhs_blocks_of(S);
  S->rdiff_blocks = rdiff_blocks_of(S);
  // host copies of the supports, ordered on the plan's stream (a copy on the
  // legacy stream would wait for every other stream's queued work)
  for (int c = 0; c < 2; ++c)
    for (int m = 0; m < d; ++m)
      for (int l = 0; l < 3; ++l)
        if (!S->hband[c][m][l].empty()) {
          e = cudaMemcpyAsync(S->hband[c][m][l].data(), S->kband[c][m][l],
                              sizeof(int2) * S->hband[c][m][l].size(), cudaMemcpyDeviceToHost, s);
          if (e != cudaSuccess) return e;
        }
  e = cudaStreamSynchronize(s);  // the split matrices and the supports' copies are complete
  if (e != cudaSuccess) return e;
  S->bound_u = S->bound_v = nullptr;
  t->ready = 1;
  return cudaSuccess;
}

// Point this plan's descriptors at the state buffers (u, v).  The
// descriptors are host copies passed by value in every launch, so binding
// neither copies to the device nor synchronises.  A no-op when already bound.
// Start of a stepping call on (u, v).  The low-order words of a
// compensated state restart at zero (enqueued on s) when the call steps
// another pair than the one they belong to.
static cudaError_t comp_own(TcState* S, void* u, void* v, cudaStream_t s) {
  if (!S->comp || (S->comp_u == u && S->comp_v == v)) return cudaSuccess;
  for (int c = 0; c < 2; ++c) {
    cudaError_t e = cudaMemsetAsync(S->lo[c], 0, sizeof(float) * S->N, s);
    if (e != cudaSuccess) return e;
  }
  S->comp_u = u;
  S->comp_v = v;
  return cudaSuccess;
}

cudaError_t tc_reset_state(TcOperands* t, cudaStream_t s) {
  TcState* S = (TcState*)t->work[0];
  if (!S || !t->ready || !S->comp) return cudaSuccess;
  S->comp_u = S->comp_v = nullptr;  // the words belong to no pair until the next call
  for (int c = 0; c < 2; ++c) {
    cudaError_t e = cudaMemsetAsync(S->lo[c], 0, sizeof(float) * S->N, s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t tc_begin_call(TcOperands* t, void* u, void* v, cudaStream_t s) {
  TcState* S = (TcState*)t->work[0];
  if (!S || !t->ready) return cudaSuccess;
  return comp_own(S, u, v, s);
}

cudaError_t tc_bind(TcOperands* t, adr_plan_s* P, void* u, void* v) {
  TcState* S = (TcState*)t->work[0];
  if (!S || !t->ready) return cudaErrorNotSupported;
  if (S->bound_u == u && S->bound_v == v) return cudaSuccess;
  const int np = (int)S->passes.size();
  S->h_desc.resize(np);
  for (int p = 0; p < np; ++p) S->h_desc[p] = make_desc(S, P, S->passes[p], (float*)u, (float*)v);
  cudaError_t e = make_pw(S, P, (float*)u, (float*)v, &S->h_pw);
  if (e != cudaSuccess) return e;
  S->bound_u = u;
  S->bound_v = v;
  return cudaSuccess;
}

// Launch the kernels of one step for a group of solves (one solve or a
// batch), following the plan's operation list.
struct GroupStep {
  int d, variant, num_sms, nsolves;  // num_sms: resident CTAs or CTA pairs of the TC kernel
  int fmt;                           // operand format of the pieces
  int np, nops;
  TcOp ops[16];
  const TcPassDesc* desc;   // [np][nsolves]
  const TcPassDesc* hdesc;  // one solve: host copies [np], passed in the launch; else null
  const int* ustart;        // [np][nsolves + 1]
  int units[16];
  int pair[16];             // per pass: units are (u, v) pairs
  int xchg[16];             // per pass: kStage1X (clusters of two)
  int fused[16];            // per pass: modes 1 and 2 in one launch
  int fslots;               // resident CTAs of the fused kernel (one per SM)
  int ind[16];              // per pass: accumulates the step's indicators
  int df;                   // reactions in double-float (ADR_STATE_COMPENSATED)
  int xslots;               // resident clusters of the exchanging kernel
  PwLaunch rhs, flat;       // stencil blocks; flat pointwise blocks
  int rhs_blocks, flat_blocks;
  int* err;
  double flops[16], bytes[16];  // algorithmic work per pass (timing statistics)
  double pw_n;                  // total points (pointwise statistics)
};

static cudaError_t group_step(adr_plan_s* ctl, const GroupStep& G) {
  const double N = G.pw_n;
  cudaStream_t st = ctl->stream;
  for (int o = 0; o < G.nops; ++o) {
    const TcOp& op = G.ops[o];
    cudaError_t e = cudaSuccess;
    switch (op.kind) {
      case kOpRhs:
        e = timed_kernel(ctl, KC_RHS, N * 2.0 * (6.0 * G.d + 10.0), N * (8.0 + 12.0), [&] {
          PwLaunch R = G.rhs;
          R.err = G.err;
          const dim3 gr(G.rhs_blocks), bl(kPwThreads);
          if (G.fmt == kFmtTF32) {
            if (G.d == 3)
              return G.df ? launch_k(rhs3_ring_kernel<kFmtTF32, true>, gr, bl, kRingSmem, st, R)
                          : launch_k(rhs3_ring_kernel<kFmtTF32>, gr, bl, kRingSmem, st, R);
            return G.df ? launch_k(rhs_pieces_kernel<kZB2, kFmtTF32, true>, gr, bl, 0, st, R)
                        : launch_k(rhs_pieces_kernel<kZB2, kFmtTF32>, gr, bl, 0, st, R);
          }
          if (G.d == 3)
            return G.df ? launch_k(rhs3_ring_kernel<kFmtBF16, true>, gr, bl, kRingSmem, st, R)
                        : launch_k(rhs3_ring_kernel<>, gr, bl, kRingSmem, st, R);
          return G.df ? launch_k(rhs_pieces_kernel<kZB2, kFmtBF16, true>, gr, bl, 0, st, R)
                      : launch_k(rhs_pieces_kernel<kZB2>, gr, bl, 0, st, R);
        });
        break;
      case kOpRdiff:
        e = timed_kernel(ctl, KC_RDIFF, N * 2.0 * 12.0, N * (16.0 + 12.0), [&] {
          const dim3 gr(G.flat_blocks), bl(kPwThreads);
          if (G.fmt == kFmtTF32)
            return launch_k(rdiff_pieces_kernel<kFmtTF32>, gr, bl, 0, st, G.flat);
          return launch_k(rdiff_pieces_kernel<>, gr, bl, 0, st, G.flat);
        });
        break;
      case kOpLawsonPre:
        e = timed_kernel(ctl, KC_LAWSON_PW, N * 2.0 * 12.0, N * (8.0 + 12.0), [&] {
          if (G.fmt == kFmtTF32)
            return launch_k(lawson_pre_pieces_kernel<kFmtTF32>, dim3(G.flat_blocks), dim3(kPwThreads),
                            0, st, G.flat, op.factor);
          return launch_k(lawson_pre_pieces_kernel<>, dim3(G.flat_blocks), dim3(kPwThreads), 0, st,
                          G.flat, op.factor);
        });
        break;
      case kOpLawsonPost:
        e = timed_kernel(ctl, KC_LAWSON_PW, N * 2.0 * 12.0, N * 16.0, [&] {
          return launch_k(lawson_post_kernel, dim3(G.flat_blocks), dim3(kPwThreads), 0, st, G.flat,
                          op.factor);
        });
        break;
      case kOpTc: {
        const int p = op.pass;
        TcLaunch L;
        memset(&L, 0, sizeof(L));
        if (G.hdesc) {
          L.one = G.hdesc[p];
          L.desc = nullptr;
          L.ustart = nullptr;
        } else {
          L.desc = G.desc + (size_t)p * G.nsolves;
          L.ustart = G.ustart + (size_t)p * (G.nsolves + 1);
        }
        L.nsolves = G.nsolves;
        L.nunits = G.units[p];
        L.err = G.err;
        e = timed_kernel(ctl, KC_MODE_TC, G.flops[p], G.bytes[p],
                         [&] {
                           if (G.xchg[p]) return launch_xchg(G.variant, G.xslots, st, L);
                           if (G.fused[p]) return launch_fused(G.fslots, st, L, G.ind[p] != 0);
                           if (G.fmt == kFmtTF32) {
                             dim3 grid((unsigned)(L.nunits < G.num_sms ? L.nunits : G.num_sms));
                             if (G.ind[p])
                               return launch_k(tc_mode_kernel<128, 128, false, false, kFmtTF32, true>,
                                               grid, dim3(kThreads), TcCfg<128, 128, kFmtTF32>::SMEM,
                                               st, L);
                             return launch_k(tc_mode_kernel<128, 128, false, false, kFmtTF32>, grid,
                                             dim3(kThreads), TcCfg<128, 128, kFmtTF32>::SMEM, st, L);
                           }
                           return launch_tc(G.variant, G.num_sms, st, L, G.pair[p] != 0, G.ind[p] != 0);
                         });
      } break;
      default:
        e = cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

static void pass_work(const TcState* S, const TcPass& ps, double& flops, double& bytes) {
  const double N = (double)S->N, nmu = (double)S->n[ps.mu];
  const double pb = S->fmt == kFmtTF32 ? 8.0 : 6.0;  // piece bytes per value
  flops = 2.0 * 2.0 * nmu * N;
  if (ps.fused) flops = 2.0 * 2.0 * (double)(S->n[0] + S->n[1]) * N;  // two products
  bytes = 2.0 * (pb * N + pb * nmu * nmu);
  if (ps.mode == kPieces3) bytes += 2.0 * pb * N;
  if (ps.mode == kAxpy) bytes += 2.0 * (S->comp ? 16.0 : 8.0) * N;  // base, out (+ lo in, out)
  if (ps.mode == kStage1 || ps.mode == kStage1X) bytes += 2.0 * (8.0 + pb) * N;
}

static void fill_ops(GroupStep& G, const TcState* S) {
  G.np = (int)S->passes.size();
  G.nops = (int)S->ops.size();
  for (int o = 0; o < G.nops; ++o) G.ops[o] = S->ops[o];
  for (int p = 0; p < G.np; ++p) {
    G.pair[p] = S->passes[p].pair;
    G.xchg[p] = S->passes[p].mode == kStage1X;
    G.fused[p] = S->passes[p].fused;
  }
  G.xslots = S->xslots;
  G.fslots = S->num_sms;
  G.fmt = S->fmt;
  G.df = S->comp == 2;
}

cudaError_t tc_step(TcOperands* t, adr_plan_s* P, void* u, void* v) {
  TcState* S = (TcState*)t->work[0];
  if (!S || !t->ready || S->bound_u != u || S->bound_v != v) return cudaErrorNotSupported;
  GroupStep G;
  memset(&G, 0, sizeof(G));
  G.d = S->d;
  G.variant = S->variant;
  G.num_sms = S->slots;
  G.nsolves = 1;
  fill_ops(G, S);
  G.desc = nullptr;
  G.hdesc = S->h_desc.data();
  G.ustart = nullptr;
  for (int p = 0; p < G.np; ++p) {
    G.units[p] = S->units[p];
    G.ind[p] = S->h_desc[p].ind != nullptr;
    pass_work(S, S->passes[p], G.flops[p], G.bytes[p]);
  }
  memset(&G.rhs, 0, sizeof(G.rhs));
  G.rhs.one = S->h_pw;  // one solve: the descriptor travels in the launch
  G.flat = G.rhs;
  G.rhs_blocks = S->rhs_blocks;
  G.flat_blocks = S->rdiff_blocks;
  G.err = S->err;
  G.pw_n = (double)S->N;
  return group_step(P, G);
}

// Duration of the tensor-core mode-product launches as they run inside a
// step: the passes of `reps` steps are captured back to back in one graph
// (programmatic dependent launch between consecutive passes, no event node
// between them), the graph is replayed once to warm up and once between two
// events.  *ms = the replay's time / (reps x passes per step).  (u, v) are
// scratch state buffers (the AXPY passes write them).
// Host mirror of k_blocks: the K-blocks a tile starting at row n0 runs.
static void host_k_blocks(const std::vector<int2>& band, int64_t K, int64_t n0, int bk,
                          int64_t& kb0, int64_t& kb1) {
  const int64_t nk = (K + bk - 1) / bk;
  kb0 = 0;
  kb1 = nk;
  if (band.empty()) return;
  const int2 r = band[n0 >> 7];
  if (r.x < r.y) {
    kb0 = r.x / bk;
    kb1 = std::min<int64_t>(nk, (r.y + bk - 1) / bk);
  }
}

void tc_mode_macs(const TcOperands* t, double* dense, double* computed) {
  *dense = *computed = 0.0;
  const TcState* S = (const TcState*)t->work[0];
  if (!S) return;
  const int bn = kVariants[S->variant].bn;
  const int bk = kVariants[S->variant].sw / (S->fmt == kFmtTF32 ? 4 : 2);
  static const std::vector<int2> none;
  for (const TcPass& ps : S->passes) {
    if (ps.fused) {  // both products of tc_fused_kernel, as its loops run them
      const int64_t n1 = S->n[0], n2 = S->n[1], slabs = S->N / (n1 * n2);
      const int64_t tn = (n2 + kBM - 1) / kBM, bunit = n2 <= kFRowsW ? tn : 1;
      for (int c = 0; c < 2; ++c) {
        *dense += (double)slabs * ((double)n1 * n1 * n2 + (double)n2 * n2 * n1);
        const std::vector<int2>& ba = S->ksupport ? S->hband[c][0][ps.ell] : none;
        const std::vector<int2>& bb = S->ksupport ? S->hband[c][1][ps.ell] : none;
        auto range = [&](int64_t b, int64_t& lo, int64_t& hi) {
          lo = 0;
          hi = n2;
          if (!bb.empty() && bb[b].x < bb[b].y) {
            lo = bb[b].x;
            hi = bb[b].y;
          }
        };
        for (int64_t a = 0; a * kBM < n1; ++a) {
          int64_t kb0, kb1;
          host_k_blocks(ba, n1, a * kBM, kFBK, kb0, kb1);
          const double rows = (double)std::min<int64_t>(kBM, n1 - a * kBM);
          const double kin = (double)(std::min(kb1 * kFBK, n1) - kb0 * kFBK);
          for (int64_t b0 = 0; b0 < tn; b0 += bunit) {
            int64_t lo, hi;
            range(b0, lo, hi);
            for (int64_t b = b0 + 1; b < b0 + bunit; ++b) {
              int64_t l, h;
              range(b, l, h);
              lo = std::min(lo, l);
              hi = std::max(hi, h);
            }
            for (int64_t g2 = lo; g2 < hi; g2 += kFRowsW) {
              const int64_t nch = (std::min<int64_t>(kFRowsW, hi - g2) + 63) / 64;
              *computed += (double)slabs * rows * (double)(64 * nch) * kin;  // MMA1
              for (int64_t b = b0; b < b0 + bunit; ++b) {                   // MMA2 per tile
                int64_t l, h;
                range(b, l, h);
                const int64_t c0 = std::max<int64_t>(0, (l - g2) / 64);
                const int64_t c1 = std::min<int64_t>(nch, (h - g2 + 63) / 64);
                const double cols = (double)std::min<int64_t>(kBM, n2 - b * kBM);
                if (c1 > c0) *computed += (double)slabs * rows * cols * (double)(64 * (c1 - c0));
              }
            }
          }
        }
      }
      continue;
    }
    const int64_t K = S->n[ps.mu], M = S->N / K;
    for (int c = 0; c < 2; ++c) {
      *dense += (double)M * (double)K * (double)K;
      const std::vector<int2>& band = S->ksupport ? S->hband[c][ps.mu][ps.ell] : none;
      for (int64_t n0 = 0; n0 < K; n0 += bn) {
        int64_t kb0, kb1;
        host_k_blocks(band, K, n0, bk, kb0, kb1);
        const int64_t rows = std::min<int64_t>(bn, K - n0);
        *computed += (double)M * (double)rows * (double)(std::min(kb1 * bk, K) - kb0 * bk);
      }
    }
  }
}

cudaError_t tc_time_passes(TcOperands* t, adr_plan_s* P, void* u, void* v, int reps, float* ms,
                           int* passes) {
  TcState* S = (TcState*)t->work[0];
  if (!S || !t->ready) return cudaErrorNotSupported;
  cudaError_t e = tc_bind(t, P, u, v);
  if (e != cudaSuccess) return e;
  GroupStep G;
  memset(&G, 0, sizeof(G));
  G.d = S->d;
  G.variant = S->variant;
  G.num_sms = S->slots;
  G.nsolves = 1;
  fill_ops(G, S);
  int k = 0;  // keep only the mode-product launches
  for (int o = 0; o < G.nops; ++o)
    if (G.ops[o].kind == kOpTc) G.ops[k++] = G.ops[o];
  G.nops = k;
  *passes = k;
  G.hdesc = S->h_desc.data();
  for (int p = 0; p < G.np; ++p) {
    G.units[p] = S->units[p];
    G.ind[p] = S->h_desc[p].ind != nullptr;
    pass_work(S, S->passes[p], G.flops[p], G.bytes[p]);
  }
  G.err = S->err;
  G.pw_n = (double)S->N;
  const bool timing = P->timing;
  const int64_t l0 = P->launches;
  cudaStream_t saved = P->stream;
  P->timing = false;
  P->stream = P->cap_stream;
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ge = nullptr;
  e = cudaStreamBeginCapture(P->cap_stream, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaError_t e1 = cudaSuccess;
    for (int r = 0; r < reps && e1 == cudaSuccess; ++r) e1 = group_step(P, G);
    cudaError_t e2 = cudaStreamEndCapture(P->cap_stream, &g);
    e = e1 != cudaSuccess ? e1 : e2;
  }
  P->stream = saved;
  P->timing = timing;
  P->launches = l0;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&ge, g, 0);
  if (g) cudaGraphDestroy(g);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = cudaGraphLaunch(ge, P->stream);
  if (e == cudaSuccess) e = cudaEventRecord(e0, P->stream);
  if (e == cudaSuccess) e = cudaGraphLaunch(ge, P->stream);
  if (e == cudaSuccess) e = cudaEventRecord(e1, P->stream);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float t_ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t_ms, e0, e1);
  if (e == cudaSuccess) *ms = t_ms / (float)(reps * (k > 0 ? k : 1));
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (ge) cudaGraphExecDestroy(ge);
  return e;
}

cudaError_t tc_set_indicators(TcOperands* t, int enable, cudaStream_t s) {
  TcState* S = (TcState*)t->work[0];
  if (!S || !t->ready) return cudaErrorNotSupported;
  if (enable && !S->ind) {
    cudaError_t e = cudaMalloc((void**)&S->ind, sizeof(double) * 4 * kIndSlots);
    if (e != cudaSuccess) return e;
    S->allocs.push_back(S->ind);
    e = cudaMalloc((void**)&S->ind_ctr, sizeof(int64_t));
    if (e != cudaSuccess) return e;
    S->allocs.push_back(S->ind_ctr);
  }
  if (enable) {  // counter -1: the first step opens slot 0
    cudaError_t e = cudaMemsetAsync(S->ind_ctr, 0xff, sizeof(int64_t), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(S->ind, 0, sizeof(double) * 4 * kIndSlots, s);
    if (e != cudaSuccess) return e;
  } else {
    S->ind = nullptr;  // the buffers stay allocated (freed with the plan)
    S->ind_ctr = nullptr;
  }
  S->bound_u = S->bound_v = nullptr;  // descriptors are rebuilt at the next bind
  return cudaSuccess;
}

cudaError_t tc_indicator_log(TcOperands* t, cudaStream_t s, double* out, int64_t max_steps,
                             int64_t* count) {
  TcState* S = (TcState*)t->work[0];
  *count = 0;
  if (!S || !S->ind) return cudaErrorNotSupported;
  int64_t ctr = -1;
  cudaError_t e = cudaMemcpyAsync(&ctr, S->ind_ctr, sizeof(ctr), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return e;
  const int64_t have = std::min<int64_t>(ctr + 1, kIndSlots);
  const int64_t n = std::min<int64_t>(have, max_steps);
  std::vector<double> ring(4 * kIndSlots);
  e = cudaMemcpy(ring.data(), S->ind, sizeof(double) * ring.size(), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return e;
  double wsum = 1.0;
  for (int m = 0; m < S->d; ++m) wsum *= (double)(S->n[m] - 1);
  for (int64_t k = 0; k < n; ++k) {  // the last n steps, oldest first
    const int64_t step = ctr - (n - 1) + k;
    const double* q = ring.data() + 4 * (step % kIndSlots);
    out[4 * k + 0] = q[0] / wsum;
    out[4 * k + 1] = q[1] / wsum;
    out[4 * k + 2] = sqrt(q[2]);
    out[4 * k + 3] = sqrt(q[3]);
  }
  *count = n;
  return cudaSuccess;
}

int* tc_error_word(TcOperands* t) {
  TcState* S = (TcState*)t->work[0];
  return S ? S->err : nullptr;
}


}  // namespace adr

// ================================================================ batches
// Many independent solves advanced together.  When every plan is a BF16x3
// plan with the same dimension and kernel variant, one step of the whole
// batch is one grouped launch per kernel: the stencil kernel and the
// reaction-difference kernel cover every solve's blocks, and each
// tensor-core pass covers every solve's tiles in one persistent launch
// (per-solve descriptors and tensor maps in device memory).  Other batches
// step their plans one after another with each plan's own kernels.
using namespace adr;

struct adr_batch_s {
  std::vector<adr_plan> plans;
  adr_plan_s* ctl;   // stream, launch counters and timing events of the batch
  int grouped;
  // grouped descriptors
  int np, variant, num_sms, d, nsolves;
  const TcState* proto;   // plan whose operation list every solve shares
  TcPassDesc* d_desc;   // [np][nsolves]
  int* d_ustart;        // [np][nsolves + 1]
  PwDesc* d_pw;         // [nsolves]
  int* d_bstart;        // rhs [nsolves + 1], then rdiff [nsolves + 1]
  int* d_err;
  int units[8];
  int rhs_blocks, rdiff_blocks;
  double flops[8], bytes[8], pw_n;
  std::vector<void*> bound_u, bound_v;
  int ind_pass[8];      // per pass: some solve of the binding has indicators on
  // CUDA graph of kBatchChunk steps
  cudaStream_t cap;
  cudaGraphExec_t gexec;
  cudaGraphExec_t gexec_timed;   // timing mode: with event-record nodes
  int64_t g_launches;
  std::vector<void*> allocs;
  // a batch of plans that cannot all share one launch sequence is split into
  // parts, each a batch of mutually compatible plans (solve indices in idx)
  std::vector<adr_batch_s*> parts;
  std::vector<std::vector<int>> idx;
  cudaStream_t stream;   // the stream given at creation
  // batches over subsets of the solves, for the later phases of a call with
  // uneven horizons (created on first use, kept until the batch is freed)
  std::map<std::vector<int>, adr_batch_s*> subs;
};

static constexpr int64_t kBatchChunk = 16;

// Uploads of descriptor tables that never synchronise: the bytes are staged
// in a page-locked ring (one per process) and copied asynchronously on the
// caller's stream.  An event recorded after each copy guards its slice, and
// a slice is reused only once that event has completed.
class PinnedRing {
 public:
  cudaError_t upload(void* dst, const void* src, size_t n, cudaStream_t s) {
    std::lock_guard<std::mutex> lock(mu_);
    const size_t n16 = (n + 15) & ~(size_t)15;
    cudaError_t e = reserve(n16);
    if (e != cudaSuccess) return e;
    if (head_ + n16 > cap_) head_ = 0;
    // retire finished slices; wait for the unfinished ones this slice overlaps
    for (size_t i = 0; i < pend_.size();) {
      Slice& q = pend_[i];
      const bool overlap = q.lo < head_ + n16 && q.hi > head_;
      if (cudaEventQuery(q.ev) == cudaSuccess || (overlap && cudaEventSynchronize(q.ev) == cudaSuccess)) {
        events_.push_back(q.ev);
        pend_[i] = pend_.back();
        pend_.pop_back();
      } else {
        cudaGetLastError();
        if (overlap) return cudaErrorUnknown;
        ++i;
      }
    }
    memcpy(buf_ + head_, src, n);
    e = cudaMemcpyAsync(dst, buf_ + head_, n, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    cudaEvent_t ev;
    if (!events_.empty()) {
      ev = events_.back();
      events_.pop_back();
    } else if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) {
      return e;
    }
    if ((e = cudaEventRecord(ev, s)) != cudaSuccess) return e;
    pend_.push_back(Slice{head_, head_ + n16, ev});
    head_ += n16;
    return cudaSuccess;
  }

 private:
  struct Slice {
    size_t lo, hi;
    cudaEvent_t ev;
  };
  // Room for a slice of n bytes (grows rarely: waits for every pending copy).
  cudaError_t reserve(size_t n) {
    if (n <= cap_) return cudaSuccess;
    for (Slice& q : pend_) {
      cudaEventSynchronize(q.ev);
      events_.push_back(q.ev);
    }
    pend_.clear();
    size_t cap = cap_ ? 2 * cap_ : ((size_t)1 << 20);
    while (cap < n) cap *= 2;
    uint8_t* nb = nullptr;
    cudaError_t e = cudaHostAlloc((void**)&nb, cap, cudaHostAllocDefault);
    if (e != cudaSuccess) return e;
    if (buf_) cudaFreeHost(buf_);
    buf_ = nb;
    cap_ = cap;
    head_ = 0;
    return cudaSuccess;
  }
  std::mutex mu_;
  uint8_t* buf_ = nullptr;
  size_t cap_ = 0, head_ = 0;
  std::vector<Slice> pend_;
  std::vector<cudaEvent_t> events_;
};
PinnedRing g_upload_ring;

// The library's pool for batch descriptors on the current device (created
// once per device; freed memory stays in the pool).  Null on failure.
static cudaMemPool_t batch_pool() {
  static std::mutex mu;
  static cudaMemPool_t pools[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lock(mu);
  if (!pools[dev]) {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t p = nullptr;
    if (cudaMemPoolCreate(&p, &props) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    uint64_t keep = UINT64_MAX;
    cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
    pools[dev] = p;
  }
  return pools[dev];
}

// Frees nothing synchronously: graph and stream destruction are deferred by
// CUDA until their work completes, and the device arrays are returned to
// the stream-ordered pool after the batch's last launch on its stream.
static void batch_free(adr_batch B) {
  if (!B) return;
  for (adr_batch_s* q : B->parts) batch_free(q);
  for (auto& kv : B->subs) batch_free(kv.second);
  cudaStream_t st = B->ctl ? B->ctl->stream : nullptr;
  if (B->gexec) cudaGraphExecDestroy(B->gexec);
  if (B->gexec_timed) cudaGraphExecDestroy(B->gexec_timed);
  if (B->cap) cudaStreamDestroy(B->cap);
  for (void* q : B->allocs) cudaFreeAsync(q, st);
  if (B->ctl) {
    for (cudaEvent_t e : B->ctl->event_pool) cudaEventDestroy(e);
    delete B->ctl;
  }
  delete B;
}

// Plans a and b can share grouped launches: tensor-core plans running the
// same kernels and step sequence (sizes and coefficients may differ).
static bool same_sequence(const adr_plan_s* a, const adr_plan_s* b) {
  const TcState* A = (const TcState*)a->tc.work[0];
  const TcState* S = (const TcState*)b->tc.work[0];
  if (a->prec != b->prec || (a->prec != ADR_BF16X3 && a->prec != ADR_TF32X3) || !A || !S)
    return false;
  if (S->d != A->d || S->variant != A->variant || S->fmt != A->fmt || S->scheme != A->scheme ||
      (S->comp == 2) != (A->comp == 2) ||
      S->passes.size() != A->passes.size() || S->ops.size() != A->ops.size())
    return false;
  for (size_t p = 0; p < S->passes.size(); ++p)
    if (memcmp(&S->passes[p], &A->passes[p], sizeof(TcPass)) != 0) return false;
  for (size_t o = 0; o < S->ops.size(); ++o)
    if (memcmp(&S->ops[o], &A->ops[o], sizeof(TcOp)) != 0) return false;
  return true;
}

static adr_status batch_create_one(const adr_plan* plans, int count, void* stream, adr_batch* out);

static adr_status batch_create_any(const adr_plan* plans, int count, void* stream, adr_batch* out);

// A live batch holds a reference on each of its plans: destroying a plan or
// changing its kernel would leave the batch's descriptors pointing at freed
// memory, so both are refused while the count is non-zero.
extern "C" adr_status adr_batch_create(const adr_plan* plans, int count, void* stream,
                                       adr_batch* out) {
  const adr_status st = batch_create_any(plans, count, stream, out);
  if (st == ADR_OK)
    for (int i = 0; i < count; ++i) __atomic_add_fetch(&plans[i]->batch_refs, 1, __ATOMIC_ACQ_REL);
  return st;
}

static adr_status batch_create_any(const adr_plan* plans, int count, void* stream, adr_batch* out) {
  if (!plans || count < 1 || !out) {
    set_error("adr_batch_create: need count >= 1 plans and an output pointer");
    return ADR_EINVAL;
  }
  for (int i = 0; i < count; ++i)
    if (!plans[i]) {
      set_error("adr_batch_create: NULL plan");
      return ADR_EINVAL;
    }
  // classes of mutually compatible plans, in order of first appearance; plans
  // that group with nothing (not BF16X3) form one class stepped plan by plan
  std::vector<std::vector<int>> cls;
  int loose = -1;
  for (int i = 0; i < count; ++i) {
    int c = -1;
    if (same_sequence(plans[i], plans[i])) {
      for (size_t k = 0; k < cls.size() && c < 0; ++k)
        if ((int)k != loose && same_sequence(plans[cls[k][0]], plans[i])) c = (int)k;
    } else {
      c = loose;
    }
    if (c < 0) {
      cls.emplace_back();
      c = (int)cls.size() - 1;
      if (!same_sequence(plans[i], plans[i])) loose = c;
    }
    cls[c].push_back(i);
  }
  if (cls.size() == 1) return batch_create_one(plans, count, stream, out);
  adr_batch B = new adr_batch_s();
  B->plans.assign(plans, plans + count);
  B->nsolves = count;
  B->grouped = loose < 0 ? 1 : 0;
  B->stream = (cudaStream_t)stream;
  for (const std::vector<int>& c : cls) {
    std::vector<adr_plan> sub;
    for (int i : c) sub.push_back(plans[i]);
    adr_batch part = nullptr;
    adr_status st = batch_create_one(sub.data(), (int)sub.size(), stream, &part);
    if (st != ADR_OK) {
      batch_free(B);
      return st;
    }
    B->parts.push_back(part);
    B->idx.push_back(c);
  }
  *out = B;
  return ADR_OK;
}

static adr_status batch_create_one(const adr_plan* plans, int count, void* stream, adr_batch* out) {
  adr_batch B = new adr_batch_s();
  B->plans.assign(plans, plans + count);
  B->stream = (cudaStream_t)stream;
  B->ctl = new adr_plan_s();
  B->ctl->stream = (cudaStream_t)stream;
  B->ctl->prec = plans[0]->prec;
  B->ctl->use_graphs = 1;
  if (const char* ev = getenv("ADR_GRAPHS")) B->ctl->use_graphs = atoi(ev) != 0;
  B->nsolves = count;
  // grouped only if every plan runs the same tensor-core step sequence
  const TcState* S0 = (const TcState*)plans[0]->tc.work[0];
  bool grouped = true;
  for (int i = 0; i < count && grouped; ++i) grouped = same_sequence(plans[0], plans[i]);
  B->grouped = grouped ? 1 : 0;
  cudaError_t e = cudaSuccess;
  // stream-ordered device memory from the library's own pool (one per
  // device, keeping freed memory): creating a batch never synchronises, and
  // a server that creates and destroys batches all the time reuses memory.
  cudaMemPool_t pool = batch_pool();
  if (!pool) {
    set_error("adr_batch_create: no memory pool");
    batch_free(B);
    return ADR_ECUDA;
  }
  auto alloc = [&](void** q, size_t bytes) -> cudaError_t {
    cudaError_t r = cudaMallocFromPoolAsync(q, bytes < 16 ? 16 : bytes, pool, (cudaStream_t)stream);
    if (r == cudaSuccess) B->allocs.push_back(*q);
    return r;
  };
  if (B->grouped) {
    const int S_ = count;
    B->np = (int)S0->passes.size();
    B->proto = S0;
    B->variant = S0->variant;
    B->num_sms = S0->slots;
    B->d = S0->d;
    const int bn = kVariants[B->variant].bn;
    std::vector<int> us((size_t)B->np * (S_ + 1)), bs(2 * (size_t)(S_ + 1));
    B->pw_n = 0;
    for (int p = 0; p < B->np; ++p) {
      int acc = 0;
      B->flops[p] = B->bytes[p] = 0;
      for (int i = 0; i < S_; ++i) {
        const TcState* S = (const TcState*)plans[i]->tc.work[0];
        us[(size_t)p * (S_ + 1) + i] = acc;
        acc += units_of(S, S->passes[p], bn);
        double f, b;
        pass_work(S, S->passes[p], f, b);
        B->flops[p] += f;
        B->bytes[p] += b;
      }
      us[(size_t)p * (S_ + 1) + S_] = acc;
      B->units[p] = acc;
    }
    int ra = 0, rd = 0;
    for (int i = 0; i < S_; ++i) B->pw_n += (double)((const TcState*)plans[i]->tc.work[0])->N;
    for (int i = 0; i < S_; ++i) {
      const TcState* S = (const TcState*)plans[i]->tc.work[0];
      bs[i] = ra;
      bs[(S_ + 1) + i] = rd;
      ra += rhs_blocks_of(S, (double)S->N / B->pw_n);
      rd += rdiff_blocks_of(S);
    }
    bs[S_] = ra;
    bs[(S_ + 1) + S_] = rd;
    B->rhs_blocks = ra;
    B->rdiff_blocks = rd;
    if ((e = alloc((void**)&B->d_desc, sizeof(TcPassDesc) * B->np * S_)) == cudaSuccess &&
        (e = alloc((void**)&B->d_ustart, sizeof(int) * us.size())) == cudaSuccess &&
        (e = alloc((void**)&B->d_pw, sizeof(PwDesc) * S_)) == cudaSuccess &&
        (e = alloc((void**)&B->d_bstart, sizeof(int) * bs.size())) == cudaSuccess &&
        (e = alloc((void**)&B->d_err, sizeof(int))) == cudaSuccess)
      e = g_upload_ring.upload(B->d_ustart, us.data(), sizeof(int) * us.size(), (cudaStream_t)stream);
    if (e == cudaSuccess)
      e = g_upload_ring.upload(B->d_bstart, bs.data(), sizeof(int) * bs.size(), (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(B->d_err, 0, sizeof(int), (cudaStream_t)stream);
  }
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    set_error(std::string("adr_batch_create: ") + cudaGetErrorString(e));
    batch_free(B);
    return e == cudaErrorMemoryAllocation ? ADR_ENOMEM : ADR_ECUDA;
  }
  *out = B;
  return ADR_OK;
}

extern "C" adr_status adr_batch_destroy(adr_batch batch) {
  if (batch)
    for (adr_plan p : batch->plans) __atomic_sub_fetch(&p->batch_refs, 1, __ATOMIC_ACQ_REL);
  batch_free(batch);
  return ADR_OK;
}

static cudaError_t batch_bind(adr_batch B, void* const* u, void* const* v) {
  bool same = B->bound_u.size() == (size_t)B->nsolves;
  for (int i = 0; same && i < B->nsolves; ++i) same = B->bound_u[i] == u[i] && B->bound_v[i] == v[i];
  if (same) return cudaSuccess;
  const int S_ = B->nsolves;
  std::vector<TcPassDesc> hd((size_t)B->np * S_);
  std::vector<PwDesc> hp(S_);
  for (int i = 0; i < S_; ++i) {
    adr_plan_s* P = B->plans[i];
    const TcState* S = (const TcState*)P->tc.work[0];
    for (int p = 0; p < B->np; ++p)
      hd[(size_t)p * S_ + i] = make_desc(S, P, S->passes[p], (float*)u[i], (float*)v[i]);
    cudaError_t e = make_pw(S, P, (float*)u[i], (float*)v[i], &hp[i], (double)S->N / B->pw_n);
    if (e != cudaSuccess) return e;
  }
  for (int p = 0; p < B->np; ++p) {
    B->ind_pass[p] = 0;
    for (int i = 0; i < S_; ++i) B->ind_pass[p] |= hd[(size_t)p * S_ + i].ind != nullptr;
  }
  cudaError_t e = g_upload_ring.upload(B->d_desc, hd.data(), sizeof(TcPassDesc) * hd.size(),
                                       B->ctl->stream);
  if (e == cudaSuccess)
    e = g_upload_ring.upload(B->d_pw, hp.data(), sizeof(PwDesc) * hp.size(), B->ctl->stream);
  if (e != cudaSuccess) return e;
  B->bound_u.assign(u, u + S_);
  B->bound_v.assign(v, v + S_);
  if (B->gexec) {  // the graph's descriptors now describe new buffers; recapture
    cudaGraphExecDestroy(B->gexec);
    B->gexec = nullptr;
  }
  if (B->gexec_timed) {
    cudaGraphExecDestroy(B->gexec_timed);
    B->gexec_timed = nullptr;
  }
  return cudaSuccess;
}

static cudaError_t batch_step_direct(adr_batch B, int64_t nsteps) {
  GroupStep G;
  memset(&G, 0, sizeof(G));
  G.d = B->d;
  G.variant = B->variant;
  G.num_sms = B->num_sms;
  G.nsolves = B->nsolves;
  fill_ops(G, B->proto);
  G.desc = B->d_desc;
  G.ustart = B->d_ustart;
  for (int p = 0; p < B->np; ++p) {
    G.units[p] = B->units[p];
    G.flops[p] = B->flops[p];
    G.bytes[p] = B->bytes[p];
    G.ind[p] = B->ind_pass[p];
  }
  memset(&G.rhs, 0, sizeof(G.rhs));
  G.rhs.desc = B->d_pw;
  G.rhs.bstart = B->d_bstart;
  G.rhs.nsolves = B->nsolves;
  G.flat = G.rhs;
  G.flat.bstart = B->d_bstart + (B->nsolves + 1);
  G.rhs_blocks = B->rhs_blocks;
  G.flat_blocks = B->rdiff_blocks;
  G.err = B->d_err;
  G.pw_n = B->pw_n;
  for (int64_t s = 0; s < nsteps; ++s) {
    cudaError_t e = group_step(B->ctl, G);
    if (e != cudaSuccess) return e;
    B->ctl->steps++;
  }
  return cudaSuccess;
}

// Every solve of B advances by the same nsteps (arguments checked).
static adr_status batch_step_uniform(adr_batch batch, void* const* u, void* const* v,
                                     int64_t nsteps) {
  adr_batch B = batch;
  if (!B->parts.empty()) {  // one grouped launch sequence per part
    for (size_t k = 0; k < B->parts.size(); ++k) {
      std::vector<void*> pu, pv;
      for (int i : B->idx[k]) {
        pu.push_back(u[i]);
        pv.push_back(v[i]);
      }
      adr_status st = batch_step_uniform(B->parts[k], pu.data(), pv.data(), nsteps);
      if (st != ADR_OK) return st;
    }
    return ADR_OK;
  }
  if (!B->grouped) {
    for (int i = 0; i < B->nsolves; ++i) {
      adr_status st = plan_step_continue(B->plans[i], u[i], v[i], nsteps);
      if (st != ADR_OK) return st;
    }
    return ADR_OK;
  }
  if (nsteps == 0) return ADR_OK;
  cudaError_t e = batch_bind(B, u, v);
  if (e != cudaSuccess) {
    set_error(std::string("adr_batch_step: binding: ") + cudaGetErrorString(e));
    return ADR_ECUDA;
  }
  adr_plan_s* ctl = B->ctl;
  int64_t done = 0;
  if (ctl->use_graphs && nsteps >= kBatchChunk) {
    // timing mode replays a second graph with event-record nodes around
    // every kernel and harvests the times after each replay
    const bool timed = ctl->timing;
    cudaGraphExec_t& ge = timed ? B->gexec_timed : B->gexec;
    if (!ge) {
      const int64_t l0 = ctl->launches, s0 = ctl->steps;
      cudaStream_t saved = ctl->stream;
      ctl->stream = B->cap;
      if (timed) ctl->graph_timed.clear();
      ctl->capturing = true;
      cudaGraph_t g = nullptr;
      cudaError_t ce = cudaStreamBeginCapture(B->cap, cudaStreamCaptureModeThreadLocal);
      if (ce == cudaSuccess) {
        cudaError_t e1 = batch_step_direct(B, kBatchChunk);
        cudaError_t e2 = cudaStreamEndCapture(B->cap, &g);
        ce = e1 != cudaSuccess ? e1 : e2;
      }
      ctl->capturing = false;
      ctl->stream = saved;
      B->g_launches = ctl->launches - l0;
      ctl->launches = l0;
      ctl->steps = s0;
      if (ce == cudaSuccess && g) ce = cudaGraphInstantiate(&ge, g, 0);
      if (g) cudaGraphDestroy(g);
      if (ce != cudaSuccess) {
        cudaGetLastError();
        ge = nullptr;
        ctl->use_graphs = 0;
      }
    }
    if (ge) {
      for (; done + kBatchChunk <= nsteps; done += kBatchChunk) {
        e = cudaGraphLaunch(ge, ctl->stream);
        if (e != cudaSuccess) {
          set_error(std::string("adr_batch_step: cudaGraphLaunch: ") + cudaGetErrorString(e));
          return ADR_ECUDA;
        }
        ctl->launches += B->g_launches;
        ctl->steps += kBatchChunk;
        if (timed) {
          e = cudaStreamSynchronize(ctl->stream);
          if (e != cudaSuccess) {
            set_error(std::string("adr_batch_step: ") + cudaGetErrorString(e));
            return ADR_ECUDA;
          }
          harvest_timing(ctl, ctl->graph_timed);
        }
      }
    }
  }
  e = batch_step_direct(B, nsteps - done);
  if (e != cudaSuccess) {
    set_error(std::string("adr_batch_step: ") + cudaGetErrorString(e));
    return ADR_ECUDA;
  }
  return ADR_OK;
}

// Batch over the solves idx of B (cached; created on first use).
static adr_batch sub_batch(adr_batch B, const std::vector<int>& idx, adr_status* st) {
  auto it = B->subs.find(idx);
  if (it != B->subs.end()) return it->second;
  std::vector<adr_plan> sp;
  for (int i : idx) sp.push_back(B->plans[i]);
  adr_batch sub = nullptr;
  *st = batch_create_any(sp.data(), (int)sp.size(), B->stream, &sub);
  if (*st != ADR_OK) return nullptr;
  B->subs[idx] = sub;
  return sub;
}

extern "C" adr_status adr_batch_step(adr_batch batch, void* const* u, void* const* v,
                                     const int64_t* nsteps) {
  if (!batch || !u || !v || !nsteps) {
    set_error("adr_batch_step: bad argument");
    return ADR_EINVAL;
  }
  adr_batch B = batch;
  const int S_ = B->nsolves;
  for (int i = 0; i < S_; ++i) {
    if (nsteps[i] < 0) {
      set_error("adr_batch_step: nsteps[i] < 0");
      return ADR_EINVAL;
    }
    if (!u[i] || !v[i] || u[i] == v[i]) {
      set_error("adr_batch_step: state pointers must be distinct and non-NULL");
      return ADR_EINVAL;
    }
    const int prec = B->plans[i]->prec;
    if ((prec == ADR_BF16X3 || prec == ADR_TF32X3) && ((((uintptr_t)u[i]) | ((uintptr_t)v[i])) & 15)) {
      set_error("adr_batch_step: tensor-core state buffers must be 16-byte aligned");
      return ADR_EINVAL;
    }
  }
  // the start of a call for every solve that steps (compensated states)
  for (int i = 0; i < S_; ++i) {
    if (nsteps[i] == 0) continue;
    cudaError_t e = tc_begin_call(&B->plans[i]->tc, u[i], v[i], B->stream);
    if (e != cudaSuccess) {
      set_error(std::string("adr_batch_step: ") + cudaGetErrorString(e));
      return ADR_ECUDA;
    }
  }
  // phases: between consecutive distinct horizons, the solves still running
  // advance together; the first phase covers every solve that steps at all
  std::vector<int64_t> hs;
  for (int i = 0; i < S_; ++i)
    if (nsteps[i] > 0) hs.push_back(nsteps[i]);
  std::sort(hs.begin(), hs.end());
  hs.erase(std::unique(hs.begin(), hs.end()), hs.end());
  int64_t prev = 0;
  for (int64_t h : hs) {
    std::vector<int> idx;
    for (int i = 0; i < S_; ++i)
      if (nsteps[i] >= h) idx.push_back(i);
    adr_status st = ADR_OK;
    if ((int)idx.size() == S_) {
      st = batch_step_uniform(B, u, v, h - prev);
    } else {
      adr_batch sub = sub_batch(B, idx, &st);
      if (sub) {
        std::vector<void*> su, sv;
        for (int i : idx) {
          su.push_back(u[i]);
          sv.push_back(v[i]);
        }
        st = batch_step_uniform(sub, su.data(), sv.data(), h - prev);
      }
    }
    if (st != ADR_OK) return st;
    prev = h;
  }
  return ADR_OK;
}

extern "C" adr_status adr_batch_set_timing(adr_batch batch, int enable) {
  if (!batch) return ADR_EINVAL;
  if (!batch->parts.empty()) {
    for (adr_batch_s* q : batch->parts) {
      adr_status st = adr_batch_set_timing(q, enable);
      if (st != ADR_OK) return st;
    }
    return ADR_OK;
  }
  if (batch->gexec_timed) {  // its event nodes use events the plan hands out again
    cudaStreamSynchronize(batch->ctl->stream);
    cudaGraphExecDestroy(batch->gexec_timed);
    batch->gexec_timed = nullptr;
  }
  adr_status st = adr_plan_set_timing(batch->ctl, enable);
  if (st == ADR_OK && batch->d_err) {
    if (cudaMemset(batch->d_err, 0, sizeof(int)) != cudaSuccess) return ADR_ECUDA;
  }
  return st;
}

extern "C" adr_status adr_batch_stats(adr_batch batch, adr_stats* out) {
  if (!batch || !out) return ADR_EINVAL;
  if (!batch->parts.empty()) {  // sums over the parts (steps: those of one part)
    memset(out, 0, sizeof(*out));
    for (size_t k = 0; k < batch->parts.size(); ++k) {
      adr_stats q;
      adr_status st = adr_batch_stats(batch->parts[k], &q);
      if (st != ADR_OK) return st;
      if (k == 0) {
        *out = q;
        continue;
      }
      out->launches += q.launches;
      out->device_error = out->device_error ? out->device_error : q.device_error;
      for (int c = 0; c < 16; ++c) {
        out->count[c] += q.count[c];
        out->ms[c] += q.ms[c];
        out->flops[c] += q.flops[c];
        out->bytes[c] += q.bytes[c];
      }
    }
    return ADR_OK;
  }
  adr_status st = adr_plan_stats(batch->ctl, out);
  if (st == ADR_OK && batch->d_err) {
    int h = 0;
    if (cudaMemcpy(&h, batch->d_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
      return ADR_ECUDA;
    out->device_error = h;
  }
  return st;
}

extern "C" int adr_batch_is_grouped(adr_batch batch) { return batch ? batch->grouped : 0; }

// ---------------------------------------------------------------- self-test
// The bounded wait of the kernels above, exercised on its own: thread 0
// waits on an mbarrier that a thread of another warp arrives on (arrive != 0)
// or that nothing arrives on, gives up after limit_ns, and records the
// timeout code in the error word as a kernel of a step does.
__global__ void bounded_wait_selftest_kernel(int arrive, uint64_t limit_ns, int* err,
                                             unsigned long long* waited_ns) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (arrive && threadIdx.x == 32)
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&bar)) : "memory");
  if (threadIdx.x == 0) {
    const uint64_t t0 = globaltimer();
    const bool ok = mbar_wait(&bar, 0, limit_ns);
    *waited_ns = globaltimer() - t0;
    if (!ok) atomicCAS(err, 0, kErrTimeoutFull);
  }
}

extern "C" adr_status adr_selftest_bounded_wait(void* stream, int32_t arrive, int64_t limit_ns,
                                                int32_t* code, int64_t* waited_ns) {
  if (!code || !waited_ns || limit_ns < 1000000 || limit_ns > 2000000000) {
    set_error("adr_selftest_bounded_wait: need code, waited_ns and 1e6 <= limit_ns <= 2e9");
    return ADR_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  void* buf = nullptr;
  cudaError_t e = cudaMalloc(&buf, 16);
  if (e == cudaSuccess) e = cudaMemsetAsync(buf, 0, 16, st);
  if (e == cudaSuccess) {
    bounded_wait_selftest_kernel<<<1, 64, 0, st>>>(arrive, (uint64_t)limit_ns, (int*)buf,
                                                   (unsigned long long*)((char*)buf + 8));
    e = cudaGetLastError();
  }
  int32_t h[4] = {0, 0, 0, 0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, buf, 16, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (buf) cudaFree(buf);
  if (e != cudaSuccess) {
    set_error(std::string("adr_selftest_bounded_wait: ") + cudaGetErrorString(e));
    return ADR_ECUDA;
  }
  *code = h[0];
  int64_t w;
  memcpy(&w, &h[2], 8);
  *waited_ns = w;
  return ADR_OK;
}

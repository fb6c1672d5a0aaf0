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
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "adr_internal.h"
#include "pointwise.cuh"

namespace adr {

namespace {

constexpr int kBM = 128;       // rows per tile (TMEM lanes)
constexpr int kPieces = 3;
constexpr uint64_t kWaitNs = 2000000000ull;    // bounded waits: 2 s

// Tile configuration: SW = bytes of K per stage row (the swizzle width: 64
// or 128, i.e. 32 or 64 BF16 values), BN = output columns per tile.
template <int SW, int BN>
struct TcCfg {
  static constexpr int BK = SW / 2;                  // K elements per stage
  static constexpr int KSTEPS = SW / 32;             // K16 MMA steps per stage
  static constexpr int TILE_A = kBM * SW;            // bytes of one A piece tile
  static constexpr int TILE_B = BN * SW;             // bytes of one B piece tile
  static constexpr int STAGE = kPieces * (TILE_A + TILE_B);
  static constexpr int STAGES = (224 * 1024) / STAGE > 8 ? 8 : (224 * 1024) / STAGE;
  static constexpr int SMEM = STAGES * STAGE + 1024 + 256;
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
// Wait for the phase with the given parity; false after kWaitNs.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer();
  while (!mbar_try_wait(bar, parity)) {
    if (globaltimer() - t0 > kWaitNs) return false;
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
__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
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

// Instruction descriptor, kind::f16: D = F32 (bits 4-5 = 1), A = B = BF16
// (bits 7-9 = 1, 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bits
// 17-22, M >> 4 at bits 24-28.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void split3(float x, __nv_bfloat16& b0, __nv_bfloat16& b1,
                                       __nv_bfloat16& b2) {
  b0 = __float2bfloat16_rn(x);
  const float r1 = x - __bfloat162float(b0);
  b1 = __float2bfloat16_rn(r1);
  const float r2 = r1 - __bfloat162float(b1);
  b2 = __float2bfloat16_rn(r2);
}

struct TcMaps {
  CUtensorMap a[2];  // X pieces [3][M][K] per component
  CUtensorMap b[2];  // Phi pieces [3][N][K] per component
};

// Epilogue of one mode-product pass.
enum TcMode : int {
  kPieces3 = 0,   // out pieces [3][N][M] of acc
  kStage1 = 1,    // pair units only: U2 = U + alpha acc_u, V2 = V + alpha acc_v
                  // (FP32 out) and D = G(U2, V2) - G(U, V) as pieces
  kAxpy = 2       // out = base + alpha acc (FP32)
};

struct TcEpilogue {
  int mode;
  int M, N, K;
  int tiles_m, tiles_n, nunits;
  int pair;                      // 1: unit = (u, v) tile pair; 0: unit = one tile of one component
  __nv_bfloat16* outp[2];        // [3][N][M] per component (kPieces3, kStage1)
  float* outf[2];                // FP32 output per component (kStage1, kStage2)
  const float* base[2];          // FP32 base per component (kStage1, kStage2)
  float alpha;
  ReactionT<float> rx;
  int* err;
};

// The six piece pairs (i, j): A piece i times B piece j, smallest first.
__device__ __constant__ int kPairA[6] = {1, 0, 2, 0, 1, 0};
__device__ __constant__ int kPairB[6] = {1, 2, 0, 1, 0, 0};

// Components and tile index of unit u.
__device__ __forceinline__ void unit_comps(const TcEpilogue& e, int u, int& c_lo, int& c_hi,
                                           int& r) {
  if (e.pair) {
    c_lo = 0;
    c_hi = 2;
    r = u;
  } else {
    const int per = e.tiles_m * e.tiles_n;
    c_lo = u / per;
    c_hi = c_lo + 1;
    r = u - c_lo * per;
  }
}

constexpr int kEpiWarps = 8;                  // two warps per TMEM lane quarter
constexpr int kThreads = 64 + 32 * kEpiWarps;  // producer warp, MMA warp, epilogue

// Persistent kernel.  CTA b handles units b, b + gridDim.x, ...; unit ->
// (m-tile, n-tile) with the n-tile fastest so that CTAs running together
// share A tiles in L2.  For each unit the MMA warp accumulates the u tile and
// then the v tile into one of two TMEM slots (4 accumulators of BN columns),
// so the epilogue of one unit overlaps the MMAs of the next and sees both
// components of every point.  Epilogue warp w owns TMEM lane quarter w % 4
// and half (w - 2) / 4 of the columns; it prefetches its FP32 base values
// two 16-column chunks ahead, starting before the accumulator is ready.
template <int SW, int BN>
__global__ void __launch_bounds__(kThreads, 1)
    tc_mode_kernel(const __grid_constant__ TcMaps maps, TcEpilogue e) {
  using C = TcCfg<SW, BN>;
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

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nk = (e.K + C::BK - 1) / C::BK;

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
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    tmem_alloc(tmem_slot, 4 * BN);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  volatile int* abort_v = abort_flag;

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer
    for (int c = 0; c < 2; ++c) {
      asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&maps.a[c]) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&maps.b[c]) : "memory");
    }
    uint32_t g = 0;  // k-block counter of this CTA
    bool stop = false;
    for (int u = blockIdx.x; u < e.nunits && !stop; u += gridDim.x) {
      int c_lo, c_hi, r;
      unit_comps(e, u, c_lo, c_hi, r);
      const int m0 = (r / e.tiles_n) * kBM, n0 = (r % e.tiles_n) * BN;
      for (int comp = c_lo; comp < c_hi && !stop; ++comp) {
        const CUtensorMap* ma = &maps.a[comp];
        const CUtensorMap* mb = &maps.b[comp];
        for (int kb = 0; kb < nk; ++kb, ++g) {
          const int s = g % C::STAGES;
          const uint32_t it = g / C::STAGES;
          if (*abort_v || (it > 0 && !mbar_wait(&empty[s], (it - 1) & 1))) {
            atomicCAS(e.err, 0, kErrTimeoutEmpty);
            *abort_v = 1;
            stop = true;
            break;
          }
          uint8_t* st = smem + s * C::STAGE;
          mbar_arrive_expect_tx(&full[s], C::STAGE);
          for (int p = 0; p < kPieces; ++p)
            tma_load_3d(st + p * C::TILE_A, ma, &full[s], kb * C::BK, m0, p);
          for (int p = 0; p < kPieces; ++p)
            tma_load_3d(st + kPieces * C::TILE_A + p * C::TILE_B, mb, &full[s], kb * C::BK, n0,
                        p);
        }
      }
    }
    // drain: the last STAGES issued loads must have landed before exit
    const uint32_t first = g > (uint32_t)C::STAGES ? g - C::STAGES : 0;
    for (uint32_t q = first; q < g; ++q) mbar_wait(&full[q % C::STAGES], (q / C::STAGES) & 1);
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer
    const uint32_t idesc = idesc_bf16(kBM, BN);
    uint32_t g = 0;
    int i = 0;  // local unit counter
    bool stop = false;
    for (int u = blockIdx.x; u < e.nunits && !stop; u += gridDim.x, ++i) {
      const int slot = i & 1;
      const uint32_t use = i >> 1;
      if (use > 0 && !mbar_wait(&acc_empty[slot], (use - 1) & 1)) {
        atomicCAS(e.err, 0, kErrTimeoutDone);
        *abort_v = 1;
        break;
      }
      tc_fence_after();
      int c_lo, c_hi, r;
      unit_comps(e, u, c_lo, c_hi, r);
      for (int comp = c_lo; comp < c_hi && !stop; ++comp) {
        const uint32_t d = tmem + (uint32_t)((slot * 2 + comp - c_lo) * BN);
        for (int kb = 0; kb < nk; ++kb, ++g) {
          const int s = g % C::STAGES;
          if (!mbar_wait(&full[s], (g / C::STAGES) & 1)) {
            atomicCAS(e.err, 0, kErrTimeoutFull);
            *abort_v = 1;
            stop = true;
            break;
          }
          tc_fence_after();
          const uint32_t sa = smem_u32(smem + s * C::STAGE);
          const uint32_t sb = sa + kPieces * C::TILE_A;
#pragma unroll
          for (int kk = 0; kk < C::KSTEPS; ++kk) {
#pragma unroll
            for (int q = 0; q < 6; ++q) {
              const uint64_t ad = kmajor_desc<SW>(sa + kPairA[q] * C::TILE_A + kk * 32);
              const uint64_t bd = kmajor_desc<SW>(sb + kPairB[q] * C::TILE_B + kk * 32);
              mma_bf16(d, ad, bd, idesc, (kb | kk | q) != 0);
            }
          }
          mma_commit(&empty[s]);  // frees the stage once these MMAs have read it
        }
      }
      if (stop) break;
      mma_commit(&acc_full[slot]);  // both accumulators of this slot complete
    }
    // every MMA this thread issued has completed once `drain` fires
    mma_commit(drain);
    mbar_wait(drain, 0);
  } else if (warp >= 2) {
    // ---------------- epilogue
    const int q = warp & 3;                   // TMEM lane quarter
    const int half = (warp - 2) >> 2;         // column half
    constexpr int HC = BN / 2;                // columns per epilogue warp
    constexpr int NCH = HC / 16;              // 16-column chunks
    const bool fp32_in = e.mode != kPieces3;
    int i = 0;
    for (int u = blockIdx.x; u < e.nunits; u += gridDim.x, ++i) {
      const int slot = i & 1;
      int c_lo, c_hi, r;
      unit_comps(e, u, c_lo, c_hi, r);
      const int nc = c_hi - c_lo;
      const int m0 = (r / e.tiles_n) * kBM, n0 = (r % e.tiles_n) * BN + half * HC;
      const int m = m0 + q * 32 + lane;
      const bool mrow = m < e.M;
      const int64_t plane = (int64_t)e.N * e.M;
      auto chunk_cols = [&](int ch) { return min(16, e.N - (n0 + ch * 16)); };
      // base prefetch, two chunks deep: pb[buffer][component slot][column]
      float pb[2][2][16];
      auto prefetch = [&](int ch, int buf) {
        const int jm = chunk_cols(ch);
        const int64_t o0 = (int64_t)(n0 + ch * 16) * e.M + m;
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
          for (int j = 0; j < 16; ++j)
            pb[buf][c][j] = (mrow && c < nc && j < jm)
                                ? __ldg(e.base[c_lo + c] + o0 + (int64_t)j * e.M)
                                : 0.f;
      };
      if (fp32_in) {
        prefetch(0, 0);
        if (NCH > 1) prefetch(1, 1);
      }
      if (!mbar_wait(&acc_full[slot], (i >> 1) & 1)) {
        if (lane == 0) atomicCAS(e.err, 0, kErrTimeoutDone);
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
        const int64_t o0 = (int64_t)(n0 + ch * 16) * e.M + m;
        const int buf = ch & 1;
        if (mrow && jm > 0) {
          if (e.mode == kStage1) {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              if (j >= jm) break;
              const int64_t o = o0 + (int64_t)j * e.M;
              const float u0 = pb[buf][0][j], v0 = pb[buf][1][j];
              const float u2 = u0 + e.alpha * acc[0][j];
              const float v2 = v0 + e.alpha * acc[1][j];
              e.outf[0][o] = u2;
              e.outf[1][o] = v2;
              float g0u, g0v, g2u, g2v;
              react<float>(e.rx, u0, v0, g0u, g0v);
              react<float>(e.rx, u2, v2, g2u, g2v);
              __nv_bfloat16 b0, b1, b2;
              split3(g2u - g0u, b0, b1, b2);
              e.outp[0][o] = b0;
              e.outp[0][plane + o] = b1;
              e.outp[0][2 * plane + o] = b2;
              split3(g2v - g0v, b0, b1, b2);
              e.outp[1][o] = b0;
              e.outp[1][plane + o] = b1;
              e.outp[1][2 * plane + o] = b2;
            }
          } else {
            auto emit = [&](int c, const float(&a)[16], const float(&bsv)[16]) {
              if (e.mode == kPieces3) {
                __nv_bfloat16* op = e.outp[c_lo + c];
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                  if (j >= jm) break;
                  const int64_t o = o0 + (int64_t)j * e.M;
                  __nv_bfloat16 b0, b1, b2;
                  split3(a[j], b0, b1, b2);
                  op[o] = b0;
                  op[plane + o] = b1;
                  op[2 * plane + o] = b2;
                }
              } else {
                float* of = e.outf[c_lo + c];
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                  if (j >= jm) break;
                  of[o0 + (int64_t)j * e.M] = bsv[j] + e.alpha * a[j];
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
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, 4 * BN);
  }
}

// W^c = K^c U^c + G^c(U, V) as BF16 pieces [3][N] in the natural layout.
// One thread per (i1, i2) marches kZ consecutive x3 planes and keeps the x3
// neighbours in registers (2D grids have a single plane).
constexpr int kZ = 8;

__device__ __forceinline__ float zdir(float xm, float xc, float xp, int z, int n3,
                                      const TridiagT<float>& A) {
  if (z == 0) return A.b0 * (xp - xc);
  if (z == n3 - 1) return A.bn * (xm - xc);
  return A.lo * (xm - xc) + A.up * (xp - xc);
}

__global__ void __launch_bounds__(128) rhs_pieces_kernel(PointwiseArgsT<float> a,
                                                         const float* __restrict__ u,
                                                         const float* __restrict__ v,
                                                         __nv_bfloat16* __restrict__ wu,
                                                         __nv_bfloat16* __restrict__ wv) {
  const int n1 = (int)a.n[0], n2 = (int)a.n[1], n3 = a.d == 3 ? (int)a.n[2] : 1;
  const int i1 = blockIdx.x * blockDim.x + threadIdx.x;
  if (i1 >= n1) return;
  const int i2 = blockIdx.y;
  const int z0 = blockIdx.z * kZ;
  const int64_t P = (int64_t)n1 * n2;
  const int64_t col = (int64_t)i2 * n1 + i1;
  float uc = u[z0 * P + col], vc = v[z0 * P + col];
  float um = z0 > 0 ? u[(z0 - 1) * P + col] : 0.f;
  float vm = z0 > 0 ? v[(z0 - 1) * P + col] : 0.f;
#pragma unroll 2
  for (int k = 0; k < kZ; ++k) {
    const int z = z0 + k;
    if (z >= n3) break;
    const int64_t idx = z * P + col;
    const float up = z + 1 < n3 ? u[idx + P] : 0.f;
    const float vp = z + 1 < n3 ? v[idx + P] : 0.f;
    float ku = stencil_dir(u, idx, 1, i1, n1, a.A[0][0]) +
               stencil_dir(u, idx, (int64_t)n1, i2, n2, a.A[0][1]);
    float kv = stencil_dir(v, idx, 1, i1, n1, a.A[1][0]) +
               stencil_dir(v, idx, (int64_t)n1, i2, n2, a.A[1][1]);
    if (a.d == 3) {
      ku += zdir(um, uc, up, z, n3, a.A[0][2]);
      kv += zdir(vm, vc, vp, z, n3, a.A[1][2]);
    }
    float gu, gv;
    react<float>(a.rx, uc, vc, gu, gv);
    split3(ku + gu, wu[idx], wu[a.N + idx], wu[2 * a.N + idx]);
    split3(kv + gv, wv[idx], wv[a.N + idx], wv[2 * a.N + idx]);
    um = uc;
    uc = up;
    vm = vc;
    vc = vp;
  }
}

// D^c = G^c(U2, V2) - G^c(U, V) written as BF16 pieces [3][N].
__global__ void __launch_bounds__(256) rdiff_pieces_kernel(PointwiseArgsT<float> a, const float* __restrict__ u,
                                                           const float* __restrict__ v,
                                                           const float* __restrict__ u2,
                                                           const float* __restrict__ v2,
                                                           __nv_bfloat16* __restrict__ du,
                                                           __nv_bfloat16* __restrict__ dv) {
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < a.N;
       idx += (int64_t)gridDim.x * blockDim.x) {
    float g0u, g0v, g2u, g2v;
    react<float>(a.rx, u[idx], v[idx], g0u, g0v);
    react<float>(a.rx, u2[idx], v2[idx], g2u, g2v);
    split3(g2u - g0u, du[idx], du[a.N + idx], du[2 * a.N + idx]);
    split3(g2v - g0v, dv[idx], dv[a.N + idx], dv[2 * a.N + idx]);
  }
}

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

// [3][rows][K] BF16 pieces, box {SW/2, box_rows, 1}, SW-byte swizzle.
cudaError_t encode_pieces(CUtensorMap* map, const void* base, int64_t K, int64_t rows,
                          int box_rows, int sw) {
  cuuint64_t dims[3] = {(cuuint64_t)K, (cuuint64_t)rows, (cuuint64_t)kPieces};
  cuuint64_t strides[2] = {(cuuint64_t)K * 2, (cuuint64_t)(K * rows) * 2};
  cuuint32_t box[3] = {(cuuint32_t)(sw / 2), (cuuint32_t)box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims,
                        strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        sw == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// Kernel variants (swizzle width, tile width).
struct Variant {
  int sw, bn;
};
constexpr Variant kVariants[] = {{64, 128}, {128, 128}, {64, 64}};
constexpr int kNumVariants = 3;

template <int SW, int BN>
cudaError_t set_smem_attr() {
  return cudaFuncSetAttribute(tc_mode_kernel<SW, BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              TcCfg<SW, BN>::SMEM);
}

cudaError_t launch_variant(int v, dim3 grid, cudaStream_t s, const TcMaps& maps,
                           const TcEpilogue& ep) {
  switch (v) {
    case 0:
      tc_mode_kernel<64, 128><<<grid, kThreads, TcCfg<64, 128>::SMEM, s>>>(maps, ep);
      break;
    case 1:
      tc_mode_kernel<128, 128><<<grid, kThreads, TcCfg<128, 128>::SMEM, s>>>(maps, ep);
      break;
    case 2:
      tc_mode_kernel<64, 64><<<grid, kThreads, TcCfg<64, 64>::SMEM, s>>>(maps, ep);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

int grid_for(int64_t total) {
  int64_t b = (total + 255) / 256;
  if (b < 1) b = 1;
  if (b > 152 * 16) b = 152 * 16;
  return (int)b;
}

}  // namespace

// Host-side state of the tensor-core path (owned through TcOperands).
struct TcState {
  int d;
  int64_t n[3];
  int64_t N;
  __nv_bfloat16* phi[2][3][2];   // [c][mu][ell-1] -> [3][n][n]
  __nv_bfloat16* buf[2][2];      // [b][c] -> [3][N]
  CUtensorMap amap[2][2][3];     // [b][c][mu]: buffer b viewed as [3][N/n_mu][n_mu]
  CUtensorMap bmap[2][3][2];     // [c][mu][ell-1]
  int variant;
  int fuse;      // 1: fuse the stage-1 combination into the last stage-1 product
  int num_sms;
  int* err;
  std::vector<void*> allocs;
};

void tc_init(TcOperands* t) { memset(t, 0, sizeof(*t)); }

void tc_free(TcOperands* t) {
  TcState* S = (TcState*)t->work[0];
  if (S) {
    for (void* p : S->allocs) cudaFree(p);
    delete S;
  }
  t->work[0] = nullptr;
}

cudaError_t tc_prepare(TcOperands* t, int prec, int d, const int64_t n[3],
                       double* const master[2][3][4], cudaStream_t s) {
  if (prec != ADR_BF16X3) return cudaErrorNotSupported;
  for (int m = 0; m < d; ++m)
    if (n[m] % 8 != 0) return cudaErrorNotSupported;  // TMA row strides: 16-byte multiples
  cudaError_t e = get_encoder();
  if (e != cudaSuccess) return e;
  static bool attr_set = false;
  if (!attr_set) {
    if ((e = set_smem_attr<64, 128>()) != cudaSuccess) return e;
    if ((e = set_smem_attr<128, 128>()) != cudaSuccess) return e;
    if ((e = set_smem_attr<64, 64>()) != cudaSuccess) return e;
    attr_set = true;
  }
  TcState* S = new TcState();
  t->work[0] = S;
  t->prec = prec;
  S->d = d;
  S->variant = 0;
  if (const char* ev = getenv("ADR_TC_VARIANT")) {
    const int v = atoi(ev);
    if (v >= 0 && v < kNumVariants) S->variant = v;
  }
  // the fused stage-1 epilogue is kept behind ADR_TC_FUSE=1 until it beats
  // the separate reaction-difference kernel on large grids
  S->fuse = 0;
  if (const char* ev = getenv("ADR_TC_FUSE")) S->fuse = atoi(ev) != 0 ? 1 : 0;
  int dev = 0;
  cudaGetDevice(&dev);
  S->num_sms = 148;
  cudaDeviceGetAttribute(&S->num_sms, cudaDevAttrMultiProcessorCount, dev);
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
      for (int l = 0; l < 2; ++l) {
        const int64_t nn = n[m] * n[m];
        e = alloc((void**)&S->phi[c][m][l], (size_t)kPieces * nn * 2);
        if (e != cudaSuccess) return e;
        split_matrix_kernel<<<grid_for(nn), 256, 0, s>>>(master[c][m][2 + l], S->phi[c][m][l], nn);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        e = encode_pieces(&S->bmap[c][m][l], S->phi[c][m][l], n[m], n[m], bn, sw);
        if (e != cudaSuccess) return e;
      }
  for (int b = 0; b < 2; ++b)
    for (int c = 0; c < 2; ++c) {
      e = alloc((void**)&S->buf[b][c], (size_t)kPieces * S->N * 2);
      if (e != cudaSuccess) return e;
      for (int m = 0; m < d; ++m) {
        e = encode_pieces(&S->amap[b][c][m], S->buf[b][c], n[m], S->N / n[m], kBM, sw);
        if (e != cudaSuccess) return e;
      }
    }
  t->ready = 1;
  return cudaSuccess;
}

// One mu-mode product for both components: buffer b viewed along direction
// mu times phi_ell; the epilogue writes pieces to buffer 1 - b, the FP32
// AXPY, or the fused stage-1 combination.
static cudaError_t tc_mode(adr_plan_s* P, TcState* S, int b, int mu, int ell, int mode, int pair,
                           float* const outf[2], const float* const base[2], double alpha) {
  TcMaps maps;
  TcEpilogue ep{};
  const int64_t nmu = S->n[mu];
  ep.M = (int)(S->N / nmu);
  ep.N = (int)nmu;
  ep.K = (int)nmu;
  ep.err = S->err;
  ep.mode = mode;
  ep.pair = pair;
  ep.alpha = (float)alpha;
  ep.rx = P->pwf.rx;
  for (int c = 0; c < 2; ++c) {
    maps.a[c] = S->amap[b][c][mu];
    maps.b[c] = S->bmap[c][mu][ell - 1];
    ep.outp[c] = S->buf[1 - b][c];
    ep.outf[c] = outf ? outf[c] : nullptr;
    ep.base[c] = base ? base[c] : nullptr;
  }
  const int bn = kVariants[S->variant].bn;
  ep.tiles_m = (ep.M + kBM - 1) / kBM;
  ep.tiles_n = (ep.N + bn - 1) / bn;
  ep.nunits = (pair ? 1 : 2) * ep.tiles_m * ep.tiles_n;
  dim3 grid((unsigned)(ep.nunits < S->num_sms ? ep.nunits : S->num_sms));
  const double flops = 2.0 * 2.0 * (double)nmu * (double)S->N;
  // algorithmic bytes: A pieces in, Phi pieces, outputs (+ FP32 base)
  double bytes = 2.0 * (6.0 * S->N + 6.0 * nmu * nmu);
  if (mode == kPieces3) bytes += 2.0 * 6.0 * S->N;
  if (mode == kAxpy) bytes += 2.0 * 8.0 * S->N;
  if (mode == kStage1) bytes += 2.0 * (8.0 + 6.0) * S->N;
  return timed_kernel(P, KC_MODE_TC, flops, bytes,
                      [&] { return launch_variant(S->variant, grid, P->stream, maps, ep); });
}

cudaError_t tc_step(TcOperands* t, adr_plan_s* P, void* u, void* v) {
  TcState* S = (TcState*)t->work[0];
  if (!S || !t->ready) return cudaErrorNotSupported;
  const float* U = (const float*)u;
  const float* V = (const float*)v;
  float* U2 = (float*)P->u2;
  float* V2 = (float*)P->v2;
  const PointwiseArgsT<float>& pw = P->pwf;
  const double tau = P->prob.tau;
  const double N = (double)S->N;
  const int d = S->d;
  cudaError_t e = timed_kernel(P, KC_RHS, N * 2.0 * (6.0 * d + 10.0), N * (8.0 + 12.0), [&] {
    dim3 g((unsigned)((S->n[0] + 127) / 128), (unsigned)S->n[1],
           (unsigned)((S->n[2] + kZ - 1) / kZ));
    rhs_pieces_kernel<<<g, 128, 0, P->stream>>>(pw, U, V, S->buf[0][0], S->buf[0][1]);
    return cudaGetLastError();
  });
  if (e != cudaSuccess) return e;
  // stage 1: U2 = U + tau W x_mu phi_1, then D = G(U2, V2) - G(U, V)
  float* o2[2] = {U2, V2};
  const float* b1[2] = {U, V};
  int b = 0;
  for (int mu = 0; mu < d - 1; ++mu, b ^= 1) {
    e = tc_mode(P, S, b, mu, 1, kPieces3, 0, nullptr, nullptr, 1.0);
    if (e != cudaSuccess) return e;
  }
  {
    // fuse the reaction difference into the last product when there are
    // enough (u, v) tile pairs to fill the GPU, else a separate kernel
    const int64_t nlast = S->n[d - 1];
    const int bn = kVariants[S->variant].bn;
    const int64_t pairs = ((S->N / nlast + kBM - 1) / kBM) * ((nlast + bn - 1) / bn);
    if (S->fuse == 1 && pairs > 0) {
      e = tc_mode(P, S, b, d - 1, 1, kStage1, 1, o2, b1, tau);
      if (e != cudaSuccess) return e;
      b ^= 1;
    } else {
      e = tc_mode(P, S, b, d - 1, 1, kAxpy, 0, o2, b1, tau);
      if (e != cudaSuccess) return e;
      b = 0;
      e = timed_kernel(P, KC_RDIFF, N * 2.0 * 12.0, N * (16.0 + 12.0), [&] {
        rdiff_pieces_kernel<<<grid_for(S->N), 256, 0, P->stream>>>(pw, U, V, U2, V2, S->buf[0][0],
                                                                   S->buf[0][1]);
        return cudaGetLastError();
      });
      if (e != cudaSuccess) return e;
    }
  }
  // stage 2: U+ = U2 + 2^(d-1) tau D x_mu phi_2
  float* o1[2] = {(float*)u, (float*)v};
  const float* b2[2] = {U2, V2};
  for (int mu = 0; mu < d; ++mu, b ^= 1) {
    const bool last = mu == d - 1;
    e = tc_mode(P, S, b, mu, 2, last ? kAxpy : kPieces3, 0, last ? o1 : nullptr,
                last ? b2 : nullptr, ldexp(tau, d - 1));
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

int* tc_error_word(TcOperands* t) {
  TcState* S = (TcState*)t->work[0];
  return S ? S->err : nullptr;
}

}  // namespace adr

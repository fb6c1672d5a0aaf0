// Error reduction that allocates no device memory.
//
// adr_max_abs_diff allocates (cudaMalloc) and frees (cudaFree) a small result
// buffer on every call.  Some callers cannot do that where they check a
// result: a serving loop that has already committed the whole device-memory
// budget to admitted solves, a host application that owns the CUDA
// allocator and forbids other libraries from calling cudaMalloc/cudaFree,
// and code that must not insert cudaFree's implicit device synchronisation
// into a running pipeline.  adr_max_abs_diff_noalloc computes the same two
// maxima with scratch memory that is part of the library image: the
// file-scope array g_noalloc_scratch below.
//
// Scratch layout (doubles): [2 * kMaxBlocks] per-block partial maxima
// (|x - ref| then |ref| for block b at 2b, 2b + 1), then 2 result slots.
// Every slot a call reads was written earlier in the same call, so nothing
// needs clearing between calls; the array keeps the last call's values.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <mutex>
#include <string>

#include "adr_internal.h"

namespace adr {
namespace {

constexpr int kThreads = 256;
constexpr int kPerThread = 16;
constexpr int64_t kPerBlock = (int64_t)kThreads * kPerThread;   // 4096 elements per block
constexpr int kMaxBlocks = 16384;                                 // 256 KB of partials
constexpr int64_t kMaxCount = kPerBlock * kMaxBlocks;             // 67,108,864 elements
constexpr int kMaxDevices = 64;

// Held by every GPU that loads the library until the process exits.
static __device__ __align__(256) double g_noalloc_scratch[2 * kMaxBlocks + 2];

// Host copies of the array's device address, resolved once per device.
void* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

__device__ __forceinline__ double nanmax(double a, double b) {
  return (b > a || b != b) ? b : a;  // a NaN wins
}

__global__ void __launch_bounds__(kThreads) noalloc_partials_kernel(const void* __restrict__ x,
                                                                    int x_is_double,
                                                                    const double* __restrict__ ref,
                                                                    int64_t count,
                                                                    double* __restrict__ part) {
  __shared__ double sd[kThreads], sr[kThreads];
  const int64_t base = (int64_t)blockIdx.x * kPerBlock;
  double md = 0.0, mr = 0.0;
#pragma unroll 4
  for (int k = 0; k < kPerThread; ++k) {
    const int64_t e = base + (int64_t)k * kThreads + threadIdx.x;
    if (e < count) {
      const double xv = x_is_double ? ((const double*)x)[e] : (double)((const float*)x)[e];
      const double r = ref[e];
      md = nanmax(md, fabs(xv - r));
      mr = fmax(mr, fabs(r));
    }
  }
  sd[threadIdx.x] = md;
  sr[threadIdx.x] = mr;
  __syncthreads();
  for (int w = kThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      sd[threadIdx.x] = nanmax(sd[threadIdx.x], sd[threadIdx.x + w]);
      sr[threadIdx.x] = fmax(sr[threadIdx.x], sr[threadIdx.x + w]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = sd[0];
    part[2 * blockIdx.x + 1] = sr[0];
  }
}

__global__ void __launch_bounds__(kThreads) noalloc_final_kernel(const double* __restrict__ part,
                                                                 int nblocks,
                                                                 double* __restrict__ result) {
  __shared__ double sd[kThreads], sr[kThreads];
  double md = 0.0, mr = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += kThreads) {
    md = nanmax(md, part[2 * b]);
    mr = fmax(mr, part[2 * b + 1]);
  }
  sd[threadIdx.x] = md;
  sr[threadIdx.x] = mr;
  __syncthreads();
  for (int w = kThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      sd[threadIdx.x] = nanmax(sd[threadIdx.x], sd[threadIdx.x + w]);
      sr[threadIdx.x] = fmax(sr[threadIdx.x], sr[threadIdx.x + w]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    result[0] = sd[0];
    result[1] = sr[0];
  }
}

}  // namespace
}  // namespace adr

using namespace adr;

extern "C" adr_status adr_max_abs_diff_noalloc(void* stream, const void* x, int x_is_double,
                                               const double* ref, int64_t count, double out[2]) {
  if (!x || !ref || !out || count < 0) {
    set_error("adr_max_abs_diff_noalloc: NULL pointer or negative count");
    return ADR_EINVAL;
  }
  if (count > kMaxCount) {
    set_error("adr_max_abs_diff_noalloc: count " + std::to_string((long long)count) +
              " exceeds the static scratch limit of " + std::to_string((long long)kMaxCount) +
              " elements; use adr_max_abs_diff");
    return ADR_EINVAL;
  }
  int dev = 0;
  ADR_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("adr_max_abs_diff_noalloc: device index out of range");
    return ADR_EINVAL;
  }
  void* scratch = nullptr;
  {
    // Set-up, once per device, with that device current: the array's name
    // is only a host-side stand-in, so fetch its device address.
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p) {
        set_error(std::string("adr_max_abs_diff_noalloc: cudaGetSymbolAddress: ") +
                  cudaGetErrorString(e));
        return ADR_ECUDA;
      }
      g_scratch_addr[dev] = p;
    }
    scratch = g_scratch_addr[dev];
  }
  if (count == 0) {
    out[0] = 0.0;
    out[1] = 0.0;
    return ADR_OK;
  }
  cudaStream_t s = (cudaStream_t)stream;
  double* part = (double*)scratch;
  double* result = part + 2 * kMaxBlocks;
  const int nblocks = (int)((count + kPerBlock - 1) / kPerBlock);
  noalloc_partials_kernel<<<nblocks, kThreads, 0, s>>>(x, x_is_double, ref, count, part);
  ADR_CUDA_TRY(cudaGetLastError());
  noalloc_final_kernel<<<1, kThreads, 0, s>>>(part, nblocks, result);
  ADR_CUDA_TRY(cudaGetLastError());
  ADR_CUDA_TRY(cudaMemcpyAsync(out, result, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
  ADR_CUDA_TRY(cudaStreamSynchronize(s));
  return ADR_OK;
}

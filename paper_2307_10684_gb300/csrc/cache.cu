// Process-wide cache of device buffers derived from a plan's operators.
//
// The matrix functions e^(tau A_mu), phi_1(tau A_mu), phi_2(tau A_mu) depend
// only on the directional operator (n_mu, its FD coefficients, which carry
// L_mu, delta and alpha_mu) and on tau, and are computed once per step size
// (Sec. 4, opening text).  Plans whose operators coincide (solves of one
// model family with the same side and coefficients, both directions of a
// square grid, ...) share one copy: a set of buffers is keyed by the values
// that determine its contents, counted by the plans holding it, and freed
// when the last one lets go.  The split operand pieces of the tensor-core
// path are cached the same way, keyed by the FP64 matrix they come from and
// the piece format.
//
// A set is filled on the acquiring plan's stream and inserted only after
// that stream has completed, so no other plan sees a half-computed set;
// two plans that miss at the same time both compute, and the later one
// drops its copy for the one already inserted.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <map>
#include <mutex>
#include <vector>

#include "adr_internal.h"

namespace adr {
namespace {

struct Entry {
  std::vector<void*> bufs;
  int refs;
};

std::mutex g_mu;
std::map<std::vector<uint64_t>, Entry> g_sets;
std::map<void*, std::vector<uint64_t>> g_by_ptr;  // first buffer -> key
uint64_t g_private = 0;                           // keys of uncached sets

bool cache_enabled() {
  static const bool on = [] {
    const char* ev = getenv("ADR_MATRIX_CACHE");
    return !(ev && atoi(ev) == 0);
  }();
  return on;
}

}  // namespace

cudaError_t shared_acquire(std::vector<uint64_t> key, int nbuf, size_t bytes,
                           const std::function<cudaError_t(void* const*)>& fill, cudaStream_t s,
                           void** out, bool* hit) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  key.insert(key.begin(), {(uint64_t)dev, (uint64_t)nbuf, (uint64_t)bytes});
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!cache_enabled()) key.push_back(~g_private++);  // a key nothing else has
    auto it = g_sets.find(key);
    if (it != g_sets.end()) {
      it->second.refs++;
      for (int b = 0; b < nbuf; ++b) out[b] = it->second.bufs[b];
      *hit = true;
      return cudaSuccess;
    }
  }
  std::vector<void*> bufs(nbuf, nullptr);
  for (int b = 0; b < nbuf && e == cudaSuccess; ++b) e = cudaMalloc(&bufs[b], bytes < 16 ? 16 : bytes);
  if (e == cudaSuccess) e = fill(bufs.data());
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    for (void* q : bufs)
      if (q) cudaFree(q);
    return e;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  auto it = g_sets.find(key);
  if (it != g_sets.end()) {  // another plan inserted the same set meanwhile
    for (void* q : bufs) cudaFree(q);
    it->second.refs++;
    for (int b = 0; b < nbuf; ++b) out[b] = it->second.bufs[b];
    *hit = true;
    return cudaSuccess;
  }
  g_sets[key] = Entry{bufs, 1};
  g_by_ptr[bufs[0]] = key;
  for (int b = 0; b < nbuf; ++b) out[b] = bufs[b];
  *hit = false;
  return cudaSuccess;
}

void shared_release(void* first) {
  if (!first) return;
  std::lock_guard<std::mutex> lock(g_mu);
  auto kp = g_by_ptr.find(first);
  if (kp == g_by_ptr.end()) return;
  auto it = g_sets.find(kp->second);
  if (it == g_sets.end()) return;
  if (--it->second.refs > 0) return;
  for (void* q : it->second.bufs) cudaFree(q);
  g_sets.erase(it);
  g_by_ptr.erase(kp);
}

int64_t shared_sets_live() {
  std::lock_guard<std::mutex> lock(g_mu);
  return (int64_t)g_sets.size();
}

}  // namespace adr

// Tensor-core (tcgen05) path: placeholder until the kernels land.
#include <cuda_runtime.h>
#include <string.h>

#include "adr_internal.h"

namespace adr {

void tc_init(TcOperands* t) { memset(t, 0, sizeof(*t)); }
void tc_free(TcOperands* t) { (void)t; }
cudaError_t tc_prepare(TcOperands* t, int prec, int d, const int64_t n[3],
                       double* const master[2][3][4], cudaStream_t s) {
  (void)t; (void)prec; (void)d; (void)n; (void)master; (void)s;
  return cudaErrorNotSupported;
}
cudaError_t tc_step(TcOperands* t, adr_plan_s* P, void* u, void* v) {
  (void)t; (void)P; (void)u; (void)v;
  return cudaErrorNotSupported;
}

}  // namespace adr

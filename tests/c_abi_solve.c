/* A C program that uses the library only through include/adr.h: it solves
 * the 2D FitzHugh-Nagumo system with advection (the model of ADR_FHN) on a
 * 96 x 64 grid of [0,100]^2 with BF16x3 tensor-core products, from host
 * buffers, and writes the result.
 *
 *   c_abi_solve <nsteps> <in.f32> <out.f32>
 *
 * in.f32 holds u0 then v0 (float32, x_1 fastest), out.f32 receives uT then
 * vT.  Exit status 0 on success; on failure the status name and
 * adr_last_error() go to stderr. */
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "adr.h"

#define NX 96
#define NY 64

static int check(adr_status s, const char* what) {
  if (s == ADR_OK) return 0;
  fprintf(stderr, "%s: %s (%s)\n", what, adr_status_str(s), adr_last_error());
  return 1;
}

int main(int argc, char** argv) {
  if (argc != 4) {
    fprintf(stderr, "usage: %s <nsteps> <in.f32> <out.f32>\n", argv[0]);
    return 2;
  }
  const long nsteps = strtol(argv[1], NULL, 10);
  const size_t npts = (size_t)NX * NY;
  float* buf = (float*)malloc(4 * npts * sizeof(float));
  if (!buf) return 2;
  float *u0 = buf, *v0 = buf + npts, *uT = buf + 2 * npts, *vT = buf + 3 * npts;
  FILE* f = fopen(argv[2], "rb");
  if (!f || fread(u0, sizeof(float), 2 * npts, f) != 2 * npts) {
    fprintf(stderr, "cannot read %s\n", argv[2]);
    return 2;
  }
  fclose(f);

  adr_problem p;
  memset(&p, 0, sizeof(p));
  p.d = 2;
  p.model = ADR_FHN;
  p.precision = ADR_BF16X3;
  p.scheme = ADR_ETD2RKDS;
  p.n[0] = NX;
  p.n[1] = NY;
  p.n[2] = 1;
  p.hi[0] = p.hi[1] = 100.0;
  p.hi[2] = 1.0;
  p.diff[0] = 1.0;
  p.diff[1] = 20.0;
  p.adv[0][0] = p.adv[0][1] = p.adv[1][0] = p.adv[1][1] = 0.5;
  p.params[0] = 0.05; /* eps */
  p.params[1] = 2.0;  /* a1 */
  p.params[2] = -0.03; /* a0 */
  p.tau = 1e-2;

  size_t state_bytes = 0, cache_bytes = 0;
  if (check(adr_plan_bytes(&p, &state_bytes, &cache_bytes), "adr_plan_bytes")) return 1;
  if (state_bytes != 2 * npts * sizeof(float)) {
    fprintf(stderr, "unexpected state_bytes %zu\n", state_bytes);
    return 1;
  }
  adr_plan plan = NULL;
  if (check(adr_plan_create(&p, NULL, &plan), "adr_plan_create")) return 1;
  if (check(adr_solve(plan, u0, v0, uT, vT, nsteps), "adr_solve")) return 1;
  adr_stats st;
  if (check(adr_plan_stats(plan, &st), "adr_plan_stats")) return 1;
  if (st.device_error != 0) {
    fprintf(stderr, "device error %d\n", st.device_error);
    return 1;
  }
  if (check(adr_plan_destroy(plan), "adr_plan_destroy")) return 1;

  f = fopen(argv[3], "wb");
  if (!f || fwrite(uT, sizeof(float), 2 * npts, f) != 2 * npts) {
    fprintf(stderr, "cannot write %s\n", argv[3]);
    return 2;
  }
  fclose(f);
  free(buf);
  printf("steps %lld launches %lld\n", (long long)st.steps, (long long)st.launches);
  return 0;
}

/*
 * A plain C99 program that drives the solver through include/wcns.h alone
 * (no Python, no CUDA headers): the boundary used the way a C or Fortran
 * code would use it.  Test infrastructure, built and run by
 * tests/test_abi.py (host checks, no GPU) and tests/test_gpu_edge.py
 * (a real run).
 *
 *   abi_consumer --checks
 *       argument checks and messages that need no GPU; exit status 0 when
 *       every call answers as the header states.
 *   abi_consumer IN OUT NSTEPS CFL
 *       IN holds a 1D state of 5 x n doubles ([5][n], Sec. 2 order, n =
 *       file size / 40) on [0,1] with transmissive ends and the water-air
 *       fluids of the Sec. 6 shock tube; advances it NSTEPS SSPRK3 steps at
 *       CFL through wcns_advance_steps_host (host buffer) and writes the
 *       result to OUT; prints the end time and the statistics.
 */
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "wcns.h"

static int expect(const char *what, int got, int want) {
  if (got != want) {
    fprintf(stderr, "%s: status %d (%s), expected %d\n", what, got, wcns_strerror(got), want);
    return 1;
  }
  return 0;
}

static int checks(void) {
  int bad = 0;
  wcns_grid g;
  wcns_bcs b;
  wcns_handle *h = (wcns_handle *)&g; /* must be reset to NULL on error */
  wcns_options o;
  memset(&g, 0, sizeof g);
  memset(&b, 0, sizeof b);
  g.ndim = 1;
  g.n[0] = 0;
  g.lo[0] = 0.0;
  g.hi[0] = 1.0;
  bad += expect("empty grid", wcns_create(&g, &b, 1.4, 4.4, 6e8, &h), WCNS_E_INVALID_ARG);
  bad += h != NULL;
  g.n[0] = 16;
  bad += expect("gamma_g > gamma_l", wcns_create(&g, &b, 4.4, 1.4, 6e8, &h), WCNS_E_INVALID_ARG);
  b.kind[0][1] = WCNS_BC_PERIODIC;
  bad += expect("one periodic face", wcns_create(&g, &b, 1.4, 4.4, 6e8, &h), WCNS_E_INVALID_ARG);
  bad += expect("null handle", wcns_rk3_step(NULL, NULL, 1e-6), WCNS_E_INVALID_ARG);
  wcns_default_options(&o);
  bad += o.precision != WCNS_FP64 || o.scheme != WCNS_SCHEME_PP_WCNS_IS || o.eps_ar != 1e-10;
  bad += strcmp(wcns_strerror(WCNS_E_INVALID_ARG), "invalid argument") != 0;
  return bad ? 1 : 0;
}

int main(int argc, char **argv) {
  if (argc == 2 && strcmp(argv[1], "--checks") == 0) return checks();
  if (argc != 5) {
    fprintf(stderr, "usage: %s --checks | IN OUT NSTEPS CFL\n", argv[0]);
    return 2;
  }
  FILE *f = fopen(argv[1], "rb");
  if (!f) return 2;
  fseek(f, 0, SEEK_END);
  const long bytes = ftell(f);
  fseek(f, 0, SEEK_SET);
  const int n = (int)(bytes / (5 * (long)sizeof(double)));
  double *W = (double *)malloc((size_t)bytes);
  if (n < 1 || !W || fread(W, 1, (size_t)bytes, f) != (size_t)bytes) return 2;
  fclose(f);

  wcns_grid g;
  wcns_bcs b;
  memset(&g, 0, sizeof g);
  memset(&b, 0, sizeof b);
  g.ndim = 1;
  g.n[0] = n;
  g.lo[0] = 0.0;
  g.hi[0] = 1.0;
  b.kind[0][0] = b.kind[0][1] = WCNS_BC_TRANSMISSIVE;
  wcns_handle *h = NULL;
  int st = wcns_create(&g, &b, 1.4, 4.4, 6e8, &h);
  if (st) {
    fprintf(stderr, "wcns_create: %s\n", wcns_strerror(st));
    return 1;
  }
  double t = 0.0;
  st = wcns_advance_steps_host(h, W, atoi(argv[3]), atof(argv[4]), 0.0, &t);
  wcns_stats s;
  if (!st) st = wcns_get_stats(h, &s);
  wcns_destroy(h);
  if (st) {
    fprintf(stderr, "wcns_advance_steps_host: %s\n", wcns_strerror(st));
    return 1;
  }
  f = fopen(argv[2], "wb");
  if (!f || fwrite(W, 1, (size_t)bytes, f) != (size_t)bytes) return 2;
  fclose(f);
  free(W);
  printf("t %.17g flux_limited %lld nonfinite %lld inadmissible %lld\n", t, s.flux_limited, s.nonfinite,
         s.inadmissible);
  return 0;
}

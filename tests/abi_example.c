/* A C program on the C ABI of include/lbm.h alone (no Python, no torch):
 * a doubly periodic 64 x 48 grid with a smooth density and temperature bump
 * in a uniform flow, FP64, 200 steps; the conservation totals of lbm_audit
 * must not change (periodic sides conserve rho, j and e exactly up to
 * rounding), the watchdog must stay quiet. Prints "abi example ok" and
 * returns 0 on success. Built and linked by tests/test_abi.py (CPU) and run
 * by tests/test_gpu_runtime.py (GPU). */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include "lbm.h"

#define NX 64
#define NY 48

static int check(int rc, lbm_ctx* ctx, const char* what) {
  if (rc != LBM_OK) {
    fprintf(stderr, "%s failed (%d): %s\n", what, rc, lbm_last_error(ctx));
    return 1;
  }
  return 0;
}

int main(void) {
  lbm_config cfg = {0};
  cfg.nx = NX;
  cfg.ny = NY;
  cfg.dx = cfg.dy = 0.01;
  cfg.dt = 1e-5;
  for (int k = 0; k < 16; ++k) cfg.s[k] = 1e4;
  cfg.precision = LBM_FP64;
  for (int side = 0; side < 4; ++side) cfg.bc[side].kind = LBM_BC_PERIODIC;
  cfg.audit_every = 0;

  lbm_ctx* ctx = NULL;
  if (check(lbm_create(&cfg, NULL, &ctx), NULL, "lbm_create")) return 1;

  double *rho = malloc(sizeof(double) * NX * NY), *u = malloc(sizeof(double) * NX * NY);
  double *v = malloc(sizeof(double) * NX * NY), *T = malloc(sizeof(double) * NX * NY);
  const double pi = 3.14159265358979323846;
  for (int y = 0; y < NY; ++y)
    for (int x = 0; x < NX; ++x) {
      const double bump = sin(2 * pi * x / NX) * cos(2 * pi * y / NY);
      rho[y * NX + x] = 1.0 + 0.1 * bump;
      u[y * NX + x] = 0.2;
      v[y * NX + x] = -0.1;
      T[y * NX + x] = 1.0 - 0.05 * bump;
    }
  int failed = check(lbm_set_init(ctx, rho, u, v, T, 0), ctx, "lbm_set_init");
  double before[4] = {0}, after[4] = {0};
  if (!failed) failed = check(lbm_audit(ctx, before), ctx, "lbm_audit");
  if (!failed) failed = check(lbm_step(ctx, 200), ctx, "lbm_step");
  if (!failed) failed = check(lbm_audit(ctx, after), ctx, "lbm_audit");
  if (!failed) failed = check(lbm_moments(ctx, rho, u, v, T, 0), ctx, "lbm_moments");
  long long bad = 0, negT = 0;
  if (!failed) failed = check(lbm_status(ctx, &bad, &negT), ctx, "lbm_status");
  if (!failed) {
    for (int q = 0; q < 4; ++q) {
      const double scale = fabs(before[0]) > 1.0 ? fabs(before[0]) : 1.0;
      if (fabs(after[q] - before[q]) > 1e-12 * scale) {
        fprintf(stderr, "total %d changed: %.17g -> %.17g\n", q, before[q], after[q]);
        failed = 1;
      }
    }
    if (bad != -1 || !(rho[0] > 0.0) || !(T[0] > 0.0)) {
      fprintf(stderr, "watchdog %lld or state unphysical\n", bad);
      failed = 1;
    }
  }
  lbm_destroy(ctx);
  free(rho);
  free(u);
  free(v);
  free(T);
  if (!failed) printf("abi example ok: mass %.15g, steps 200\n", after[0]);
  return failed;
}

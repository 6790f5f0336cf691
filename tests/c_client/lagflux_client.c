/* A plain C client of liblagflux: includes only include/lagflux.h and links
 * the shared library, so it checks that the boundary is usable from C with
 * no Python or C++ in between.
 *
 *   lagflux_client abi   -- no GPU needed: rejected configurations and NULL
 *                           arguments return LF_ERR_ARG with a message
 *   lagflux_client run   -- GPU: a periodic 2D shear layer from host
 *                           buffers, 50 Heun steps, conservation of the
 *                           four sums to 1e-12 (FP64), dt and time sane
 * Exit status 0 on success; the failing check is printed otherwise. */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "lagflux.h"

static int fail(const char* what) {
  fprintf(stderr, "FAIL: %s (%s)\n", what, lf_last_error(NULL));
  return 1;
}

static lf_config base_config(void) {
  lf_config c;
  memset(&c, 0, sizeof c);
  c.dim = 2;
  c.nx = 96;
  c.ny = 64;
  c.limiter = LF_LIMITER_VANLEER;
  c.bc = LF_BC_PERIODIC;
  c.precision = LF_FP64;
  c.riemann = LF_RIEMANN_MAXC;
  c.time_order = LF_TIME_HEUN;
  c.xmin = 0.0;
  c.xmax = 1.0;
  c.ymin = 0.0;
  c.ymax = 1.0;
  c.gamma = 1.4;
  c.cfl = 0.45;
  c.beta = 1.5;
  c.nz = 1;
  return c;
}

static int check_abi(void) {
  lf_ctx* ctx = NULL;
  lf_config c = base_config();
  c.dim = 4;
  if (lf_init(&c, NULL, &ctx) != LF_ERR_ARG || ctx != NULL) return fail("dim 4 accepted");
  if (strstr(lf_last_error(NULL), "invalid configuration") == NULL) return fail("no message for dim 4");
  c = base_config();
  c.cfl = 1.5;
  if (lf_init(&c, NULL, &ctx) != LF_ERR_ARG) return fail("cfl 1.5 accepted");
  c = base_config();
  c.nspecies = LF_MAX_SPECIES + 1;
  if (lf_init(&c, NULL, &ctx) != LF_ERR_ARG) return fail("too many species accepted");
  c = base_config();
  if (lf_init(&c, NULL, NULL) != LF_ERR_ARG) return fail("NULL out accepted");
  if (lf_step(NULL, NULL) != LF_ERR_ARG) return fail("lf_step(NULL)");
  if (lf_set_conservative(NULL, NULL, 0) != LF_ERR_ARG) return fail("lf_set_conservative(NULL)");
  if (lf_set_tile_rows(NULL, 8) != LF_ERR_ARG) return fail("lf_set_tile_rows(NULL)");
  if (lf_autotune(NULL, 1, NULL) != LF_ERR_ARG) return fail("lf_autotune(NULL)");
  c = base_config();
  c.tile_rows = -1;
  if (lf_init(&c, NULL, &ctx) != LF_ERR_ARG) return fail("negative tile_rows accepted");
  if (strcmp(lf_status_string(LF_ERR_NONPHYSICAL), "LF_ERR_NONPHYSICAL") != 0) return fail("status string");
  lf_destroy(NULL);
  return 0;
}

static int check_run(void) {
  lf_config c = base_config();
  const int nx = c.nx, ny = c.ny;
  const size_t n = (size_t)nx * ny;
  double* q = malloc(4 * n * sizeof(double));
  double* U = malloc(4 * n * sizeof(double));
  if (!q || !U) return fail("host allocation");
  /* shear layer: rho 2 / u +0.5 inside |y - 0.5| < 0.25, rho 1 / u -0.5 outside,
     p 2.5, v a small sine perturbation */
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      const double x = (i + 0.5) / nx, y = (j + 0.5) / ny;
      const int inside = fabs(y - 0.5) < 0.25;
      const size_t k = (size_t)j * nx + i;
      q[k] = inside ? 2.0 : 1.0;
      q[n + k] = inside ? 0.5 : -0.5;
      q[2 * n + k] = 0.01 * sin(2.0 * M_PI * 3.0 * x);
      q[3 * n + k] = 2.5;
    }
  lf_ctx* ctx = NULL;
  if (lf_init(&c, NULL, &ctx) != LF_OK) return fail("lf_init");
  if (lf_set_primitives(ctx, q, 0) != LF_OK) return fail("lf_set_primitives");
  double s0[4], s1[4];
  if (lf_conservation_sums(ctx, s0) != LF_OK) return fail("sums");
  int32_t done = 0;
  double t = 0.0;
  int32_t rows = 0;
  if (lf_autotune(ctx, 2, &rows) != LF_OK || rows < 4 || rows > 128) return fail("lf_autotune");
  int32_t now = 0;
  if (lf_get_tile_rows(ctx, &now) != LF_OK || now != rows) return fail("lf_get_tile_rows");
  if (lf_run(ctx, 0.0, 50, &done, &t) != LF_OK || done != 50 || !(t > 0.0)) return fail("lf_run");
  if (lf_conservation_sums(ctx, s1) != LF_OK) return fail("sums after");
  for (int l = 0; l < 4; ++l)
    if (fabs(s1[l] - s0[l]) > 1e-12 * fmax(1.0, fabs(s0[l]))) return fail("conservation");
  if (lf_get_conservative(ctx, U, 0) != LF_OK) return fail("lf_get_conservative");
  for (size_t k = 0; k < n; ++k)
    if (!(U[k] > 0.0)) return fail("density positive");
  lf_destroy(ctx);
  free(q);
  free(U);
  printf("ok: 50 steps to t = %.6g (%d-row tiles), sums conserved\n", t, (int)rows);
  return 0;
}

int main(int argc, char** argv) {
  if (argc < 2) return fail("usage: lagflux_client abi|run");
  if (strcmp(argv[1], "abi") == 0) return check_abi();
  if (strcmp(argv[1], "run") == 0) return check_run();
  return fail("unknown mode");
}

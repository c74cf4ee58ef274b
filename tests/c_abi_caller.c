/* A plain C caller of the library's C ABI (no Python, no torch): builds a
 * 2 x 2 x 2 Kuhn box with absorbing sides by hand, uploads it, asks adg_plan for the
 * element time steps and clusters, reads the reference operators and checks
 * the error statuses of calls out of order.  Uses only host entry points, so
 * it runs without a GPU.  Prints one line "ok <n_tets> <n_clusters> <dt_min>"
 * and exits 0, or prints the failed check and exits 1. */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "adg.h"

#define CHECK(cond)                                                  \
  do {                                                               \
    if (!(cond)) {                                                   \
      printf("failed: %s (line %d)\n", #cond, __LINE__);             \
      return 1;                                                      \
    }                                                                \
  } while (0)

enum { n = 2 };

static int64_t vid(int i, int j, int k) { return ((int64_t)k * (n + 1) + j) * (n + 1) + i; }

/* the six Kuhn tets of the unit cube: paths from corner 000 to 111 along the
 * axes in every order (positively oriented after the swap below) */
static const int kPerm[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};

int main(void) {
  const int64_t nv = (n + 1) * (n + 1) * (n + 1), nt = 6 * n * n * n;
  double* xyz = malloc(sizeof(double) * 3 * nv);
  int64_t* tets = malloc(sizeof(int64_t) * 4 * nt);
  int32_t* tag = malloc(sizeof(int32_t) * 4 * nt);
  for (int k = 0; k <= n; ++k)
    for (int j = 0; j <= n; ++j)
      for (int i = 0; i <= n; ++i) {
        double* x = xyz + 3 * vid(i, j, k);
        x[0] = (double)i / n;
        x[1] = (double)j / n;
        x[2] = (double)k / n;
      }
  int64_t t = 0;
  for (int k = 0; k < n; ++k)
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < n; ++i)
        for (int p = 0; p < 6; ++p, ++t) {
          int c[3] = {i, j, k};
          tets[4 * t] = vid(c[0], c[1], c[2]);
          for (int s = 0; s < 3; ++s) {
            c[kPerm[p][s]]++;
            tets[4 * t + 1 + s] = vid(c[0], c[1], c[2]);
          }
          /* orientation: odd permutations of the axes give negative volume */
          const double* a = xyz + 3 * tets[4 * t];
          double e[3][3];
          for (int s = 0; s < 3; ++s)
            for (int d = 0; d < 3; ++d) e[s][d] = xyz[3 * tets[4 * t + 1 + s] + d] - a[d];
          double det = e[0][0] * (e[1][1] * e[2][2] - e[1][2] * e[2][1]) -
                       e[0][1] * (e[1][0] * e[2][2] - e[1][2] * e[2][0]) +
                       e[0][2] * (e[1][0] * e[2][1] - e[1][1] * e[2][0]);
          if (det < 0) {
            int64_t tmp = tets[4 * t + 1];
            tets[4 * t + 1] = tets[4 * t + 2];
            tets[4 * t + 2] = tmp;
          }
        }
  /* a face is on the box boundary when its three vertices lie on one side
   * (coordinate 0 or 1 in one axis): absorbing there, interior elsewhere */
  for (int64_t e = 0; e < nt; ++e)
    for (int f = 0; f < 4; ++f) {
      int boundary = 0;
      for (int d = 0; d < 3; ++d)
        for (int side = 0; side <= 1; ++side) {
          int all = 1;
          for (int v = 0; v < 4; ++v)
            if (v != f && xyz[3 * tets[4 * e + v] + d] != (double)side) all = 0;
          boundary |= all;
        }
      tag[4 * e + f] = boundary ? ADG_TAG_ABSORB : ADG_TAG_INTERIOR;
    }
  double* rho = malloc(sizeof(double) * nt);
  double* lam = malloc(sizeof(double) * nt);
  double* mu = malloc(sizeof(double) * nt);
  for (int64_t e = 0; e < nt; ++e) {
    rho[e] = 1.0;
    lam[e] = 2.0;
    mu[e] = 1.0;
  }

  adg_config cfg;
  adg_default_config(&cfg);
  CHECK(cfg.degree == 5 && cfg.precision == ADG_FP64 && cfg.max_clusters == 1 && cfg.ensemble == 1);
  cfg.degree = 3;
  cfg.cfl = 0.5;
  adg_ctx* ctx = NULL;
  CHECK(adg_create(&cfg, &ctx) == ADG_OK && ctx != NULL);

  double dtmin = -1.0;
  CHECK(adg_plan(ctx, NULL, NULL, &dtmin, NULL) == ADG_E_STATE && dtmin == -1.0);
  CHECK(strlen(adg_last_error(ctx)) > 0);
  CHECK(adg_upload_mesh(ctx, nv, xyz, nt, tets, tag, NULL) == ADG_OK);
  CHECK(adg_upload_material(ctx, rho, lam, mu) == ADG_OK);
  CHECK(adg_query(ctx, &(adg_info){0}) == ADG_E_STATE); /* not initialised */

  double* dt = malloc(sizeof(double) * nt);
  int32_t* cl = malloc(sizeof(int32_t) * nt);
  int ncl = 0;
  CHECK(adg_plan(ctx, dt, cl, &dtmin, &ncl) == ADG_OK);
  /* uniform Kuhn tets: one size, one cluster; h = 6V / sum(A) of the tet with
   * edges 1/n along the axes, V = 1/(6 n^3), dt = cfl/(2N+1) h / c_p, c_p = 2 */
  const double a = 1.0 / n;
  CHECK(ncl == 1);
  for (int64_t e = 0; e < nt; ++e) CHECK(cl[e] == 0 && fabs(dt[e] - dtmin) <= 1e-15 * dtmin);
  /* every Kuhn tet of the cube has faces a^2/2, a^2/2, a^2 sqrt(2)/2, a^2 sqrt(2)/2 */
  const double sumA = 0.5 * a * a * (2.0 + 2.0 * sqrt(2.0));
  const double h = 6.0 * (a * a * a / 6.0) / sumA;
  CHECK(fabs(dtmin - 0.5 / 7.0 * h / 2.0) <= 1e-14 * dtmin);
  const double dt_planned = dtmin;

  /* reference operators of degree 3: B = 20, B1 = 10, Bf = 10 */
  double* kt = malloc(sizeof(double) * 3 * 20 * 20);
  CHECK(adg_reference_operators(3, kt, NULL, NULL, NULL) == ADG_OK);
  /* kt[a][m][l] = int phi_m dphi_l/dxi_a: the column of the constant phi_0 vanishes */
  for (int ax = 0; ax < 3; ++ax)
    for (int m = 0; m < 20; ++m) CHECK(fabs(kt[ax * 400 + m * 20 + 0]) < 1e-13);
  /* and phi_1.. are not constant: some derivative is nonzero */
  double big = 0;
  for (int q = 0; q < 1200; ++q) big = fmax(big, fabs(kt[q]));
  CHECK(big > 0.1);
  CHECK(adg_reference_operators(9, kt, NULL, NULL, NULL) == ADG_E_INVALID);

  /* a bad material is reported, nothing written */
  mu[3] = -1.0;
  CHECK(adg_upload_material(ctx, rho, lam, mu) == ADG_OK);
  dtmin = -1.0;
  CHECK(adg_plan(ctx, NULL, NULL, &dtmin, NULL) == ADG_E_INVALID && dtmin == -1.0);

  /* the pipelined calls: argument checks, then the state check before adg_init */
  float qf = 0.f;
  CHECK(adg_set_dofs_f32_async(NULL, &qf) == ADG_E_INVALID);
  CHECK(adg_get_dofs_f32_async(ctx, NULL) == ADG_E_INVALID);
  CHECK(adg_advance_async(ctx, -1) == ADG_E_INVALID);
  CHECK(adg_set_dofs_f32_async(ctx, &qf) == ADG_E_STATE);
  CHECK(adg_get_dofs_f32_async(ctx, &qf) == ADG_E_STATE);
  CHECK(adg_advance_async(ctx, 1) == ADG_E_STATE);
  CHECK(adg_sync(ctx) == ADG_E_STATE);

  adg_destroy(ctx);
  printf("ok %lld %d %.17g\n", (long long)nt, ncl, dt_planned);
  free(xyz); free(tets); free(tag); free(rho); free(lam); free(mu); free(dt); free(cl); free(kt);
  return 0;
}

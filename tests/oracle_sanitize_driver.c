/*
 * oracle_sanitize_driver.c -- runs every entry point of the CPU oracle on one
 * mesh and state read from a file, for a build under AddressSanitizer,
 * UndefinedBehaviorSanitizer and LeakSanitizer (tests/test_oracle_sanitizers.py).
 * Test infrastructure: it links the oracle's C sources and nothing else.
 *
 * Input (native byte order):
 *   int64 kind (0 Euler, 1 scalar), nv, nt, k, steps
 *   double xy[2 nv]; int32 tri[3 nt]; int32 canon[nv]; int8 bc[3 nt]
 *   Euler:  or_config; double u0[4 nb nt]; double t_end
 *   scalar: or_sc_config; double u0[nb nt]; double t_end
 * Output: double u[...] after `steps` steps, double t, int64 counters[4].
 * Exit status 0 when every call returned what it should.
 */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

#define CHECK(cond)                                                        \
  do {                                                                     \
    if (!(cond)) {                                                         \
      fprintf(stderr, "check failed at line %d: %s\n", __LINE__, #cond);   \
      exit(3);                                                             \
    }                                                                      \
  } while (0)

static void *read_n(FILE *f, size_t bytes) {
  void *p = malloc(bytes ? bytes : 1);
  CHECK(p != NULL);
  CHECK(fread(p, 1, bytes, f) == bytes);
  return p;
}

/* the error paths of the mesh builder: a clockwise cell and an edge shared
 * by three cells are rejected without a leak */
static void bad_meshes(void) {
  const double xy[] = {0, 0, 1, 0, 0, 1, 1, 1, -1, 0.5};
  const int32_t cw[] = {0, 2, 1};
  or_mesh *m = NULL;
  CHECK(or_mesh_create(3, xy, 1, cw, NULL, NULL, &m) == OR_EMESH && m == NULL);
  const int32_t fan[] = {0, 1, 2, 1, 3, 2, 0, 2, 4, 1, 2, 4};   /* edge {1, 2} in three cells */
  int8_t walls[12];
  memset(walls, OR_BC_REFLECT, sizeof walls);
  CHECK(or_mesh_create(5, xy, 4, fan, NULL, walls, &m) == OR_EMESH && m == NULL);
  const int32_t one[] = {0, 1, 2};   /* boundary edges without a tag */
  CHECK(or_mesh_create(3, xy, 1, one, NULL, NULL, &m) == OR_EMESH && m == NULL);
  const int32_t out_of_range[] = {0, 1, 7};
  CHECK(or_mesh_create(3, xy, 1, out_of_range, NULL, walls, &m) == OR_EMESH && m == NULL);
}

static void run_euler(FILE *f, FILE *out, int64_t nv, int64_t nt, int k, int64_t steps, or_mesh *m) {
  or_config cf;
  CHECK(fread(&cf, sizeof cf, 1, f) == 1);
  const int nb = k == 1 ? 3 : 6;
  const size_t sz = 4u * (size_t)nb * (size_t)nt;
  double *u = read_n(f, sizeof(double) * sz);
  double t_end;
  CHECK(fread(&t_end, sizeof t_end, 1, f) == 1);
  (void)nv;

  int32_t *nbr = malloc(sizeof(int32_t) * 3 * nt), *ne = malloc(sizeof(int32_t) * 3 * nt);
  double *area = malloc(sizeof(double) * nt), *len = malloc(sizeof(double) * 3 * nt);
  double *nrm = malloc(sizeof(double) * 6 * nt), *q12 = malloc(sizeof(double) * 24 * nt);
  CHECK(nbr && ne && area && len && nrm && q12);
  or_mesh_neighbors(m, nbr, ne);
  or_mesh_geometry(m, area, len, nrm);
  or_quad12_points(m, q12);
  for (int64_t K = 0; K < nt; ++K) {
    double w[3], om[2], nodes[4], cfl[2];
    int32_t nn, limv[2];
    CHECK(or_decomposition(m, k, K, w, om, nodes, &nn, cfl, limv) == OR_OK);
  }
  CHECK(or_min_cfl_area(m, k, 0) > 0.0 && or_min_cfl_area(m, k, 1) > 0.0);

  /* the stage operators, on all cells and on the odd cells */
  int64_t nodd = nt / 2;
  int64_t *odd = malloc(sizeof(int64_t) * (nodd ? nodd : 1));
  CHECK(odd != NULL);
  for (int64_t j = 0; j < nodd; ++j) odd[j] = 2 * j + 1;
  double *L = calloc(sz, sizeof(double)), *uh = calloc(sz, sizeof(double));
  double *oe = calloc(sz, sizeof(double)), *lim = calloc(sz, sizeof(double));
  double *sig = calloc(12u * (size_t)nt, sizeof(double)), *pm = calloc(2u * (size_t)nt, sizeof(double));
  CHECK(L && uh && oe && lim && sig && pm);
  const double alpha = or_alpha(m, &cf, u, 0.0);
  CHECK(alpha > 0.0);
  CHECK(or_alpha_cells(m, &cf, u, 0.0, odd, nodd) <= alpha);
  CHECK(or_L(m, &cf, u, alpha, 0.0, L, NULL, 0) == OR_OK);
  CHECK(or_L(m, &cf, u, alpha, 0.0, L, odd, nodd) == OR_OK);
  const double dt = 0.5 * or_min_cfl_area(m, k, 0) / alpha;
  CHECK(or_rk_stage(m, &cf, u, u, 0.0, 1.0, dt, alpha, 0.0, uh, NULL, 0) == OR_OK);
  double st[10], st2[10];
  CHECK(or_stats(m, &cf, uh, st) == OR_OK);
  CHECK(or_stats_cells(m, &cf, uh, odd, nodd, st2) == OR_OK);
  CHECK(st2[4] <= st[4] && st2[7] == st[7]);
  CHECK(or_oe(m, &cf, uh, dt, st, dt, oe, sig, NULL, 0) == OR_OK);
  CHECK(or_oe(m, &cf, uh, dt, st, dt, oe, NULL, odd, nodd) == OR_OK);
  int64_t cnt2[2] = {0, 0};
  CHECK(or_limit(m, &cf, oe, lim, cnt2, NULL, 0) == OR_OK);
  or_point_minima(m, &cf, lim, pm);
  double pt[4];
  or_eval(m, k, lim, 0, q12[0], q12[1], pt);

  /* the scheme */
  double t = 0.0;
  int64_t cnt[4] = {0, 0, 0, 0};
  CHECK(or_advance(m, &cf, u, &t, t_end, steps, cnt) == OR_OK);
  CHECK(fwrite(u, sizeof(double), sz, out) == sz);
  CHECK(fwrite(&t, sizeof t, 1, out) == 1);
  CHECK(fwrite(cnt, sizeof(int64_t), 4, out) == 4);
  /* a step at t = t_end does nothing */
  double dt0 = -1.0;
  CHECK(or_step(m, &cf, u, &t, t, &dt0, cnt) == OR_OK && dt0 == 0.0);

  free(odd); free(L); free(uh); free(oe); free(lim); free(sig); free(pm);
  free(nbr); free(ne); free(area); free(len); free(nrm); free(q12); free(u);
}

static void run_scalar(FILE *f, FILE *out, int64_t nt, int k, int64_t steps, or_mesh *m) {
  or_sc_config cf;
  CHECK(fread(&cf, sizeof cf, 1, f) == 1);
  const int nb = (k + 1) * (k + 2) / 2;
  const size_t sz = (size_t)nb * (size_t)nt;
  double *u = read_n(f, sizeof(double) * sz);
  double t_end;
  CHECK(fread(&t_end, sizeof t_end, 1, f) == 1);
  double *L = calloc(sz, sizeof(double)), *oe = calloc(sz, sizeof(double));
  double *sig = calloc((size_t)(k + 1) * (size_t)nt, sizeof(double)), *vals = malloc(sizeof(double) * 12 * nt);
  double *pr = calloc(sz, sizeof(double));
  CHECK(L && oe && sig && vals && pr);
  const double alpha = or_sc_alpha(m, &cf, u);
  CHECK(or_sc_L(m, &cf, u, alpha, L) == OR_OK);
  double st[3];
  or_sc_stats(m, &cf, u, st);
  CHECK(or_sc_oe(m, &cf, u, 1e-3, st, oe, sig) == OR_OK);
  CHECK(or_sc_dt_base(m, k) > 0.0);
  for (int64_t i = 0; i < 12 * nt; ++i) vals[i] = 1.0 + 1e-3 * (double)(i % 17);
  CHECK(or_sc_project(m, k, vals, pr) == OR_OK);
  double d = or_sc_deriv(m, k, u, 0, 0.0, 0.0, 1, 0) + or_sc_eval(m, k, u, 0, 0.0, 0.0);
  (void)d;
  double b[10];
  or_sc_basis(0.25, 0.25, 1, 1, b);
  double t = 0.0;
  int64_t n = 0;
  CHECK(or_sc_advance(m, &cf, u, &t, t_end, steps, &n) == OR_OK);
  int64_t cnt[4] = {n, 0, 0, 0};
  CHECK(fwrite(u, sizeof(double), sz, out) == sz);
  CHECK(fwrite(&t, sizeof t, 1, out) == 1);
  CHECK(fwrite(cnt, sizeof(int64_t), 4, out) == 4);
  free(L); free(oe); free(sig); free(vals); free(pr); free(u);
}

int main(int argc, char **argv) {
  CHECK(argc == 3);
  FILE *f = fopen(argv[1], "rb"), *out = fopen(argv[2], "wb");
  CHECK(f && out);
  int64_t hdr[5];
  CHECK(fread(hdr, sizeof(int64_t), 5, f) == 5);
  const int64_t kind = hdr[0], nv = hdr[1], nt = hdr[2], steps = hdr[4];
  const int k = (int)hdr[3];
  double *xy = read_n(f, sizeof(double) * 2 * nv);
  int32_t *tri = read_n(f, sizeof(int32_t) * 3 * nt), *canon = read_n(f, sizeof(int32_t) * nv);
  int8_t *bc = read_n(f, 3 * (size_t)nt);
  or_mesh *m = NULL;
  CHECK(or_mesh_create(nv, xy, nt, tri, canon, bc, &m) == OR_OK && m != NULL);
  CHECK(or_mesh_nt(m) == nt);
  double psi[6], dpsi[12], d2psi[18], mc[6];
  or_basis(0.2, 0.3, psi, dpsi, d2psi);
  or_mass_constants(k > 2 ? 2 : k, mc);
  if (kind == 0) run_euler(f, out, nv, nt, k, steps, m);
  else run_scalar(f, out, nt, k, steps, m);
  or_mesh_destroy(m);
  bad_meshes();
  free(xy); free(tri); free(canon); free(bc);
  fclose(f);
  CHECK(fclose(out) == 0);
  return 0;
}

/*
 * oracle.c -- plain FP64 CPU oracle of the bound-preserving, rotation-
 * invariant OEDG scheme on triangles for the 2D Euler equations
 * (Ding, Cui & Wu, "Robust DG Schemes on Unstructured Triangular Meshes:
 * Oscillation Elimination and Bound Preservation via Optimal Convex
 * Decomposition", arXiv 2409.09620).
 *
 * TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU-baseline
 * leg of the benchmark are the only users.  Nothing here is shared with the
 * CUDA path.
 *
 * Every quantity is evaluated the slow, direct way: a polynomial is
 * evaluated at a PHYSICAL point by mapping it back to the reference triangle
 * of the cell that owns the polynomial; neighbour traces are found by
 * evaluating the neighbour's own polynomial at the same physical point (or
 * at its periodic translate); derivatives are physical derivatives by the
 * chain rule.  Loops follow the order of the paper's formulas.
 *
 * Readings of the paper where it is silent or garbled (each is also listed
 * in the design notes of the repository):
 *  - edge e_i is opposite vertex v_i (Fig. 1); its endpoints in counter-
 *    clockwise order are v_c = v_{i+1}, v_d = v_{i+2};
 *  - the edge Gauss map of Appendix B uses nodes on [-1, 1]; they are mapped
 *    to s = (1 + x_nu) / 2 on the edge with weights w_nu / 2 (sum 1);
 *  - alpha of the LF flux is the maximum wave speed over the edge Gauss
 *    points of the stage input (eq. 1250), boundary ghost states included;
 *    dt is fixed per step from the first stage's alpha (Sec. 5);
 *  - the exterior state of a transmissive (outflow) edge is the cell's own
 *    average, a constant: in the flux, in alpha and in the OE jumps (zero
 *    exterior derivatives); the interior trace itself would add no
 *    dissipation at the edge, and gas at rest next to such an edge then
 *    amplifies round-off;
 *  - the OE jumps on a boundary edge are taken against the same exterior
 *    state as the flux: the mirror polynomial on a reflecting wall, the cell
 *    average on a transmissive edge, a constant state on a Dirichlet / shock
 *    edge;
 *  - the wave speed R(u, n) is +inf for rho <= 0 and uses max(p, 0) in the
 *    sound speed (it is evaluated at vertices that the limiter does not
 *    control); a term beta/h * delta with delta = 0 contributes 0;
 *  - the BP limiter for P2 checks rho and the internal energy at the two
 *    internal nodes of the optimal decomposition (the paper's E_* formula is
 *    only an upper bound of E at the weighted internal state, because E is
 *    concave); for P1 it uses the vertices v1, v2 as the paper does;
 *  - the moving-shock and Dirichlet ghosts are evaluated at the stage time
 *    t^n + c_s dt, c = (0, 1, 1/2) for fluxes, and at the time of the stage
 *    result for the OE jumps.
 */
#include "oracle.h"
#include "oracle_mesh.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Orthogonal modal basis, eq. (basisfunc): Psi^(0..5)                       */
/* ------------------------------------------------------------------------ */
void or_basis(double xi, double eta, double *psi, double *dpsi, double *d2psi) {
  psi[0] = 1.0;
  psi[1] = 4.0 * xi + 2.0 * eta - 2.0;
  psi[2] = 3.0 * eta - 1.0;
  psi[3] = 24.0 * xi * xi + 24.0 * xi * eta + 4.0 * eta * eta - 24.0 * xi - 8.0 * eta + 4.0;
  psi[4] = 20.0 * xi * eta + 10.0 * eta * eta - 4.0 * xi - 12.0 * eta + 2.0;
  psi[5] = 10.0 * eta * eta - 8.0 * eta + 1.0;
  if (dpsi) {
    /* d/dxi, d/deta */
    dpsi[0] = 0.0;                          dpsi[1] = 0.0;
    dpsi[2] = 4.0;                          dpsi[3] = 2.0;
    dpsi[4] = 0.0;                          dpsi[5] = 3.0;
    dpsi[6] = 48.0 * xi + 24.0 * eta - 24.0; dpsi[7] = 24.0 * xi + 8.0 * eta - 8.0;
    dpsi[8] = 20.0 * eta - 4.0;             dpsi[9] = 20.0 * xi + 20.0 * eta - 12.0;
    dpsi[10] = 0.0;                         dpsi[11] = 20.0 * eta - 8.0;
  }
  if (d2psi) {
    /* d2/dxi2, d2/dxi deta, d2/deta2 */
    for (int i = 0; i < 9; ++i) d2psi[i] = 0.0;
    d2psi[9] = 48.0;  d2psi[10] = 24.0; d2psi[11] = 8.0;
    d2psi[12] = 0.0;  d2psi[13] = 20.0; d2psi[14] = 20.0;
    d2psi[15] = 0.0;  d2psi[16] = 0.0;  d2psi[17] = 20.0;
  }
}

static int nbasis(int k) { return k == 1 ? 3 : 6; }
static int mode_degree(int l) { return l == 0 ? 0 : (l <= 2 ? 1 : 2); }

/* N-point volume rule for degree k: N = 3 (k = 1) or 6 (k = 2), Sec. 2.1 */
static int vol_rule(int k, const double (**b)[3], const double **w) {
  if (k == 1) { *b = Q3_B; *w = Q3_W; return 3; }
  *b = Q6_B; *w = Q6_W; return 6;
}

/* Q = k + 1 Gauss points on an edge: parameter s in (0, 1) and weight summing to 1 */
static int edge_rule(int k, double *s, double *w) {
  if (k == 1) {
    double x = 1.0 / sqrt(3.0);
    s[0] = 0.5 * (1.0 - x); s[1] = 0.5 * (1.0 + x);
    w[0] = 0.5; w[1] = 0.5;
    return 2;
  }
  double x = sqrt(3.0 / 5.0);
  s[0] = 0.5 * (1.0 - x); s[1] = 0.5; s[2] = 0.5 * (1.0 + x);
  w[0] = 5.0 / 18.0; w[1] = 8.0 / 18.0; w[2] = 5.0 / 18.0;
  return 3;
}

static void bary_point(const cellgeo *g, const double b[3], double *x, double *y) {
  *x = b[0] * g->v[0][0] + b[1] * g->v[1][0] + b[2] * g->v[2][0];
  *y = b[0] * g->v[0][1] + b[1] * g->v[1][1] + b[2] * g->v[2][1];
}

/* a_K^(l) / |K| = integral of Psi_l^2 over K divided by |K| (12-point rule, exact to degree 6) */
void or_mass_constants(int k, double *c) {
  int nb = nbasis(k);
  for (int l = 0; l < nb; ++l) c[l] = 0.0;
  for (int mu = 0; mu < 12; ++mu) {
    double psi[6];
    or_basis(Q12_B[mu][1], Q12_B[mu][2], psi, NULL, NULL); /* (xi, eta) = (b2, b3) */
    for (int l = 0; l < nb; ++l) c[l] += Q12_W[mu] * psi[l] * psi[l];
  }
}

/* ------------------------------------------------------------------------ */
/* Evaluation of a cell polynomial at a physical point                      */
/* ------------------------------------------------------------------------ */
static inline double coef(const double *u, int64_t nt, int nb, int c, int l, int64_t K) {
  return u[((int64_t)c * nb + l) * nt + K];
}

static void eval_at(const or_mesh *m, int k, const double *u, int64_t K, const cellgeo *g,
                    double x, double y, double out[4]) {
  int nb = nbasis(k);
  double xi, eta, psi[6];
  ref_coords(g, x, y, &xi, &eta);
  or_basis(xi, eta, psi, NULL, NULL);
  for (int c = 0; c < 4; ++c) {
    double s = 0.0;
    for (int l = 0; l < nb; ++l) s += coef(u, m->nt, nb, c, l, K) * psi[l];
    out[c] = s;
  }
}

void or_eval(const or_mesh *m, int k, const double *u, int64_t K, double x, double y, double *out4) {
  cellgeo g;
  cell_geo(m, K, &g);
  eval_at(m, k, u, K, &g, x, y, out4);
}

/* value, physical gradient (d/dx, d/dy) and Hessian (xx, xy, yy) of all 4 components */
static void eval_derivs(const or_mesh *m, int k, const double *u, int64_t K, const cellgeo *g,
                        double x, double y, double val[4], double grad[4][2], double hess[4][3]) {
  int nb = nbasis(k);
  double xi, eta, psi[6], dpsi[12], d2psi[18];
  ref_coords(g, x, y, &xi, &eta);
  or_basis(xi, eta, psi, dpsi, d2psi);
  double xx = g->jinv[0][0], xy_ = g->jinv[0][1]; /* d xi / dx, d xi / dy */
  double ex = g->jinv[1][0], ey = g->jinv[1][1];  /* d eta / dx, d eta / dy */
  for (int c = 0; c < 4; ++c) {
    val[c] = 0.0;
    grad[c][0] = grad[c][1] = 0.0;
    hess[c][0] = hess[c][1] = hess[c][2] = 0.0;
  }
  for (int l = 0; l < nb; ++l) {
    double px = dpsi[2 * l] * xx + dpsi[2 * l + 1] * ex;
    double py = dpsi[2 * l] * xy_ + dpsi[2 * l + 1] * ey;
    double a = d2psi[3 * l], b = d2psi[3 * l + 1], cc = d2psi[3 * l + 2];
    double pxx = a * xx * xx + 2.0 * b * xx * ex + cc * ex * ex;
    double pxy = a * xx * xy_ + b * (xx * ey + xy_ * ex) + cc * ex * ey;
    double pyy = a * xy_ * xy_ + 2.0 * b * xy_ * ey + cc * ey * ey;
    for (int c = 0; c < 4; ++c) {
      double q = coef(u, m->nt, nb, c, l, K);
      val[c] += q * psi[l];
      grad[c][0] += q * px;
      grad[c][1] += q * py;
      hess[c][0] += q * pxx;
      hess[c][1] += q * pxy;
      hess[c][2] += q * pyy;
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Euler physics, eq. (eq:euler) and eq. (G:Euler)                           */
/* ------------------------------------------------------------------------ */
static double pressure(const double u[4], double gamma) {
  return (gamma - 1.0) * (u[3] - (u[1] * u[1] + u[2] * u[2]) / (2.0 * u[0]));
}

/* rho-weighted internal energy E - |m|^2 / (2 rho) of eq. (G:Euler) */
static double int_energy(const double u[4]) { return u[3] - (u[1] * u[1] + u[2] * u[2]) / (2.0 * u[0]); }

static void euler_flux(const double u[4], double gamma, double f1[4], double f2[4]) {
  double rho = u[0], v1 = u[1] / rho, v2 = u[2] / rho;
  double p = pressure(u, gamma);
  f1[0] = u[1];       f2[0] = u[2];
  f1[1] = u[1] * v1 + p; f2[1] = u[1] * v2;
  f1[2] = u[2] * v1;  f2[2] = u[2] * v2 + p;
  f1[3] = (u[3] + p) * v1; f2[3] = (u[3] + p) * v2;
}

/* spectral radius of F'(u) . n: |v . n| + sound speed */
static double wave_speed(const double u[4], const double n[2], double gamma) {
  if (!(u[0] > 0.0)) return INFINITY;
  double p = pressure(u, gamma);
  if (p < 0.0) p = 0.0;
  return fabs(u[1] * n[0] + u[2] * n[1]) / u[0] + sqrt(gamma * p / u[0]);
}

/* Lax-Friedrichs flux, eq. (fluxLF) */
static void lf_flux(const double uin[4], const double uex[4], const double n[2], double alpha,
                    double gamma, double out[4]) {
  double f1i[4], f2i[4], f1e[4], f2e[4];
  euler_flux(uin, gamma, f1i, f2i);
  euler_flux(uex, gamma, f1e, f2e);
  for (int c = 0; c < 4; ++c)
    out[c] = 0.5 * ((f1i[c] * n[0] + f2i[c] * n[1]) + (f1e[c] * n[0] + f2e[c] * n[1]) -
                    alpha * (uex[c] - uin[c]));
}

static double shock_position(const or_config *cf, double y, double t) {
  return cf->shock_x0 + y / tan(cf->shock_angle) + cf->shock_speed * t / sin(cf->shock_angle);
}

/* exterior state at a boundary point from the interior state uin and the
 * cell average ubar */
static void ghost_state(const or_config *cf, int tag, const double uin[4], const double ubar[4],
                        const double n[2], double x, double y, double t, double out[4]) {
  if (tag == OR_BC_REFLECT) {
    double mn = uin[1] * n[0] + uin[2] * n[1];
    out[0] = uin[0];
    out[1] = uin[1] - 2.0 * mn * n[0];
    out[2] = uin[2] - 2.0 * mn * n[1];
    out[3] = uin[3];
  } else if (tag >= OR_BC_DIRICHLET0 && tag < OR_BC_DIRICHLET0 + 4) {
    for (int c = 0; c < 4; ++c) out[c] = cf->bc_state[tag - OR_BC_DIRICHLET0][c];
  } else if (tag == OR_BC_SHOCK) {
    int s = x < shock_position(cf, y, t) ? cf->shock_post : cf->shock_pre;
    for (int c = 0; c < 4; ++c) out[c] = cf->bc_state[s][c];
  } else { /* transmissive: the cell average */
    for (int c = 0; c < 4; ++c) out[c] = ubar[c];
  }
}

/* cell average of cell K (mode 0) */
static void cell_average(const or_mesh *m, int k, const double *u, int64_t K, double ubar[4]) {
  for (int c = 0; c < 4; ++c) ubar[c] = coef(u, m->nt, nbasis(k), c, 0, K);
}

/* exterior trace at the physical point (x, y) of edge i of cell K */
static void exterior_trace(const or_mesh *m, const or_config *cf, const double *u, int64_t K, int i,
                           const double n[2], double x, double y, double t, const double uin[4],
                           double uex[4]) {
  int32_t nb_cell = m->nbr[3 * K + i];
  if (nb_cell >= 0) {
    cellgeo gn;
    cell_geo(m, nb_cell, &gn);
    eval_at(m, cf->k, u, nb_cell, &gn, x + m->shift[6 * K + 2 * i], y + m->shift[6 * K + 2 * i + 1], uex);
  } else {
    double ubar[4];
    cell_average(m, cf->k, u, K, ubar);
    ghost_state(cf, m->bc[3 * K + i], uin, ubar, n, x, y, t, uex);
  }
}

/* ------------------------------------------------------------------------ */
/* Mesh construction: adjacency through (canonical) vertex pairs            */
/* ------------------------------------------------------------------------ */
typedef struct { int32_t lo, hi; int64_t K; int32_t i; } edge_rec;

static int edge_cmp(const void *pa, const void *pb) {
  const edge_rec *a = pa, *b = pb;
  if (a->lo != b->lo) return a->lo < b->lo ? -1 : 1;
  if (a->hi != b->hi) return a->hi < b->hi ? -1 : 1;
  if (a->K != b->K) return a->K < b->K ? -1 : 1;
  return a->i - b->i;
}

void or_mesh_destroy(or_mesh *m) {
  if (!m) return;
  free(m->xy); free(m->tri); free(m->canon); free(m->bc);
  free(m->nbr); free(m->nbr_edge); free(m->shift);
  free(m);
}

int or_mesh_create(int64_t nv, const double *xy, int64_t nt, const int32_t *tri,
                   const int32_t *canon, const int8_t *bc, or_mesh **out) {
  *out = NULL;
  if (nv <= 0 || nt <= 0 || !xy || !tri) return OR_EINVAL;
  or_mesh *m = calloc(1, sizeof(or_mesh));
  if (!m) return OR_ENOMEM;
  m->nv = nv; m->nt = nt;
  m->xy = malloc(sizeof(double) * 2 * nv);
  m->tri = malloc(sizeof(int32_t) * 3 * nt);
  m->canon = malloc(sizeof(int32_t) * nv);
  m->bc = malloc(3 * nt);
  m->nbr = malloc(sizeof(int32_t) * 3 * nt);
  m->nbr_edge = malloc(sizeof(int32_t) * 3 * nt);
  m->shift = calloc(6 * nt, sizeof(double));
  edge_rec *rec = malloc(sizeof(edge_rec) * 3 * nt);
  if (!m->xy || !m->tri || !m->canon || !m->bc || !m->nbr || !m->nbr_edge || !m->shift || !rec) {
    free(rec); or_mesh_destroy(m); return OR_ENOMEM;
  }
  memcpy(m->xy, xy, sizeof(double) * 2 * nv);
  memcpy(m->tri, tri, sizeof(int32_t) * 3 * nt);
  for (int64_t v = 0; v < nv; ++v) m->canon[v] = canon ? canon[v] : (int32_t)v;
  for (int64_t e = 0; e < 3 * nt; ++e) m->bc[e] = bc ? bc[e] : 0;
  int rc = OR_OK;
  for (int64_t e = 0; e < 3 * nt; ++e) {
    if (m->tri[e] < 0 || m->tri[e] >= nv) { rc = OR_EMESH; goto done; }
    m->nbr[e] = -1; m->nbr_edge[e] = -1;
  }
  for (int64_t K = 0; K < nt; ++K) {
    cellgeo g;
    cell_geo(m, K, &g);
    if (!(g.area > 0.0)) { rc = OR_EMESH; goto done; }
    for (int i = 0; i < 3; ++i) {
      int32_t a = m->canon[m->tri[3 * K + (i + 1) % 3]], b = m->canon[m->tri[3 * K + (i + 2) % 3]];
      if (a < 0 || a >= nv || b < 0 || b >= nv || a == b) { rc = OR_EMESH; goto done; }
      rec[3 * K + i].lo = a < b ? a : b;
      rec[3 * K + i].hi = a < b ? b : a;
      rec[3 * K + i].K = K;
      rec[3 * K + i].i = i;
    }
  }
  qsort(rec, 3 * nt, sizeof(edge_rec), edge_cmp);
  for (int64_t e = 0; e < 3 * nt;) {
    int64_t f = e + 1;
    while (f < 3 * nt && rec[f].lo == rec[e].lo && rec[f].hi == rec[e].hi) ++f;
    if (f - e > 2) { rc = OR_EMESH; goto done; }   /* non-manifold */
    if (f - e == 2) {
      int64_t K0 = rec[e].K, K1 = rec[e + 1].K;
      int i0 = rec[e].i, i1 = rec[e + 1].i;
      int32_t a0 = m->tri[3 * K0 + (i0 + 1) % 3], b0 = m->tri[3 * K0 + (i0 + 2) % 3];
      int32_t a1 = m->tri[3 * K1 + (i1 + 1) % 3], b1 = m->tri[3 * K1 + (i1 + 2) % 3];
      /* the shared edge is traversed in opposite directions by the two cells */
      if (m->canon[a0] != m->canon[b1] || m->canon[b0] != m->canon[a1]) { rc = OR_EMESH; goto done; }
      double sx = m->xy[2 * b1] - m->xy[2 * a0], sy = m->xy[2 * b1 + 1] - m->xy[2 * a0 + 1];
      double tx = m->xy[2 * a1] - m->xy[2 * b0], ty = m->xy[2 * a1 + 1] - m->xy[2 * b0 + 1];
      double scale = 1.0 + fabs(sx) + fabs(sy);
      if (fabs(sx - tx) > 1e-9 * scale || fabs(sy - ty) > 1e-9 * scale) { rc = OR_EMESH; goto done; }
      m->nbr[3 * K0 + i0] = (int32_t)K1; m->nbr_edge[3 * K0 + i0] = i1;
      m->nbr[3 * K1 + i1] = (int32_t)K0; m->nbr_edge[3 * K1 + i1] = i0;
      m->shift[6 * K0 + 2 * i0] = sx;  m->shift[6 * K0 + 2 * i0 + 1] = sy;
      m->shift[6 * K1 + 2 * i1] = -sx; m->shift[6 * K1 + 2 * i1 + 1] = -sy;
    } else {
      int8_t tag = m->bc[3 * rec[e].K + rec[e].i];
      if (tag < OR_BC_REFLECT || tag > OR_BC_SHOCK) { rc = OR_EMESH; goto done; }
    }
    e = f;
  }
done:
  free(rec);
  if (rc != OR_OK) { or_mesh_destroy(m); return rc; }
  *out = m;
  return OR_OK;
}

int64_t or_mesh_nt(const or_mesh *m) { return m->nt; }

void or_mesh_neighbors(const or_mesh *m, int32_t *nbr, int32_t *nbr_edge) {
  memcpy(nbr, m->nbr, sizeof(int32_t) * 3 * m->nt);
  memcpy(nbr_edge, m->nbr_edge, sizeof(int32_t) * 3 * m->nt);
}

void or_mesh_geometry(const or_mesh *m, double *area, double *len, double *normal) {
  for (int64_t K = 0; K < m->nt; ++K) {
    cellgeo g;
    cell_geo(m, K, &g);
    area[K] = g.area;
    for (int i = 0; i < 3; ++i) {
      len[3 * K + i] = g.len[i];
      normal[6 * K + 2 * i] = g.n[i][0];
      normal[6 * K + 2 * i + 1] = g.n[i][1];
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Optimal convex decomposition, eqs. (1040) and (1139); BP CFL numbers      */
/* eqs. (1692), (1713); classical ZXS CFL numbers (Sec. 4.3 remarks)         */
/* ------------------------------------------------------------------------ */
/* relabelling with l1 >= l2 >= l3 (Sec. 4.2); ties keep the original order */
static void sort_edges(const cellgeo *g, int perm[3]) {
  perm[0] = 0; perm[1] = 1; perm[2] = 2;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 2 - a; ++b)
      if (g->len[perm[b]] < g->len[perm[b + 1]]) { int t = perm[b]; perm[b] = perm[b + 1]; perm[b + 1] = t; }
}

int or_decomposition(const or_mesh *m, int k, int64_t K, double *w, double *omega, double *nodes,
                     int32_t *n_nodes, double *cfl, int32_t *limv) {
  if (K < 0 || K >= m->nt || (k != 1 && k != 2)) return OR_EINVAL;
  cellgeo g;
  cell_geo(m, K, &g);
  int p[3];
  sort_edges(&g, p);
  /* sorted labels: edge s (longest first) is original edge p[s]; its opposite vertex is p[s] */
  double l1 = g.len[p[0]], l2 = g.len[p[1]], l3 = g.len[p[2]];
  const double *V1 = g.v[p[0]], *V2 = g.v[p[1]], *V3 = g.v[p[2]];
  double lbar = (l1 + l2 + l3) / 3.0;
  limv[0] = p[0];
  limv[1] = p[1];
  nodes[0] = nodes[1] = nodes[2] = nodes[3] = 0.0;
  omega[0] = omega[1] = 0.0;
  if (k == 1) {
    for (int i = 0; i < 3; ++i) w[i] = 2.0 * g.len[i] / (3.0 * l1 + 3.0 * l2);
    omega[0] = (l1 + l2 - 2.0 * l3) / (3.0 * l1 + 3.0 * l2);
    double den = l1 + l2 - 2.0 * l3;
    if (den > 0.0) {
      nodes[0] = ((l1 - l3) * V1[0] + (l2 - l3) * V2[0]) / den;
      nodes[1] = ((l1 - l3) * V1[1] + (l2 - l3) * V2[1]) / den;
      *n_nodes = 1;
    } else {
      *n_nodes = 0;   /* equilateral: omega_1 = 0, no internal node */
    }
    cfl[0] = 2.0 / (3.0 * (l1 + l2));
    cfl[1] = 1.0 / (9.0 * lbar);
    return OR_OK;
  }
  /* P2, eq. (1139) and (1703) */
  double lhat = sqrt(l1 * l1 + l2 * l2 + l3 * l3 - (2.0 / 3.0) * (l1 * l2 + l2 * l3 + l3 * l1));
  for (int i = 0; i < 3; ++i) w[i] = 2.0 * g.len[i] / (9.0 * lbar + 3.0 * lhat);
  omega[0] = omega[1] = (lbar + lhat) / (6.0 * lbar + 2.0 * lhat);
  const double r3 = sqrt(3.0);
  double c[2][3] = {
      {3 * l1 + 3 * l2 + r3 * l2 - r3 * l3, 6 * l2 + r3 * l3 - r3 * l1, 3 * l2 + 3 * l3 + r3 * l1 - r3 * l2},
      {3 * l1 + 3 * l2 + r3 * l3 - r3 * l2, 6 * l2 + r3 * l1 - r3 * l3, 3 * l2 + 3 * l3 + r3 * l2 - r3 * l1}};
  double M[2][3][3][3] = {
      {{{6, 1, -2}, {1, 2 * r3 + 6, -r3 - 2}, {-2, -r3 - 2, 6}},
       {{6, -r3 - 2, -2}, {-r3 - 2, 12, r3 - 2}, {-2, r3 - 2, 6}},
       {{6, r3 - 2, -2}, {r3 - 2, 6 - 2 * r3, 1}, {-2, 1, 6}}},
      {{{6, 1, -2}, {1, 6 - 2 * r3, r3 - 2}, {-2, r3 - 2, 6}},
       {{6, r3 - 2, -2}, {r3 - 2, 12, -r3 - 2}, {-2, -r3 - 2, 6}},
       {{6, -r3 - 2, -2}, {-r3 - 2, 2 * r3 + 6, 1}, {-2, 1, 6}}}};
  double lv[3] = {l1, l2, l3};
  double den = 18.0 * (lbar + lhat) * (l2 + lhat);
  for (int s = 0; s < 2; ++s) {
    double beta[3];
    for (int i = 0; i < 3; ++i) {
      double q = 0.0;
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) q += lv[a] * M[s][i][a][b] * lv[b];
      beta[i] = (q + 2.0 * c[s][i] * lhat) / den;
    }
    nodes[2 * s] = beta[0] * V1[0] + beta[1] * V2[0] + beta[2] * V3[0];
    nodes[2 * s + 1] = beta[0] * V1[1] + beta[1] * V2[1] + beta[2] * V3[1];
  }
  *n_nodes = 2;
  cfl[0] = 2.0 / (9.0 * lbar + 3.0 * lhat);
  cfl[1] = 1.0 / (27.0 * lbar);
  return OR_OK;
}

double or_min_cfl_area(const or_mesh *m, int k, int decomp) {
  double best = INFINITY;
  for (int64_t K = 0; K < m->nt; ++K) {
    double w[3], om[2], nd[4], cfl[2];
    int32_t nn, lv[2];
    or_decomposition(m, k, K, w, om, nd, &nn, cfl, lv);
    cellgeo g;
    cell_geo(m, K, &g);
    double v = cfl[decomp ? 1 : 0] * g.area;
    if (v < best) best = v;
  }
  return best;
}

/* ------------------------------------------------------------------------ */
/* Initial data: L2 projection with the 12-point rule (Appendix A)           */
/* ------------------------------------------------------------------------ */
void or_quad12_points(const or_mesh *m, double *xy) {
  for (int64_t K = 0; K < m->nt; ++K) {
    cellgeo g;
    cell_geo(m, K, &g);
    for (int mu = 0; mu < 12; ++mu) bary_point(&g, Q12_B[mu], &xy[(K * 12 + mu) * 2], &xy[(K * 12 + mu) * 2 + 1]);
  }
}

int or_project(const or_mesh *m, int k, const double *vals, double *coeffs) {
  if (k != 1 && k != 2) return OR_EINVAL;
  int nb = nbasis(k);
  double cm[6];
  or_mass_constants(k, cm);
#pragma omp parallel for schedule(static)
  for (int64_t K = 0; K < m->nt; ++K) {
    double acc[4][6] = {{0}};
    for (int mu = 0; mu < 12; ++mu) {
      double psi[6];
      or_basis(Q12_B[mu][1], Q12_B[mu][2], psi, NULL, NULL);
      for (int c = 0; c < 4; ++c)
        for (int l = 0; l < nb; ++l) acc[c][l] += Q12_W[mu] * vals[(K * 12 + mu) * 4 + c] * psi[l];
    }
    for (int c = 0; c < 4; ++c)
      for (int l = 0; l < nb; ++l) coeffs[((int64_t)c * nb + l) * m->nt + K] = acc[c][l] / cm[l];
  }
  return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Viscosity coefficient, eq. (1250): max over edge Gauss points            */
/* ------------------------------------------------------------------------ */
static double cell_alpha(const or_mesh *m, const or_config *cf, const double *u, int64_t K, double t) {
  cellgeo g;
  cell_geo(m, K, &g);
  double s[3], w[3];
  int Q = edge_rule(cf->k, s, w);
  double best = 0.0;
  for (int i = 0; i < 3; ++i) {
    int a = (i + 1) % 3, b = (i + 2) % 3;
    for (int nu = 0; nu < Q; ++nu) {
      double x = g.v[a][0] + (g.v[b][0] - g.v[a][0]) * s[nu];
      double y = g.v[a][1] + (g.v[b][1] - g.v[a][1]) * s[nu];
      double uin[4];
      eval_at(m, cf->k, u, K, &g, x, y, uin);
      double r = wave_speed(uin, g.n[i], cf->gamma);
      if (r > best || r != r) best = r;
      if (m->nbr[3 * K + i] < 0) {
        double uex[4], ubar[4];
        cell_average(m, cf->k, u, K, ubar);
        ghost_state(cf, m->bc[3 * K + i], uin, ubar, g.n[i], x, y, t, uex);
        double re = wave_speed(uex, g.n[i], cf->gamma);
        if (re > best || re != re) best = re;
      }
    }
  }
  return best;
}

double or_alpha_cells(const or_mesh *m, const or_config *cf, const double *u, double t,
                      const int64_t *cells, int64_t ncells) {
  int64_t n = cells ? ncells : m->nt;
  double *a = malloc(sizeof(double) * (n > 0 ? n : 1));
#pragma omp parallel for schedule(static)
  for (int64_t j = 0; j < n; ++j) a[j] = cell_alpha(m, cf, u, cells ? cells[j] : j, t);
  double best = 0.0;
  for (int64_t j = 0; j < n; ++j)
    if (a[j] > best || a[j] != a[j]) best = a[j];
  free(a);
  return best;
}

double or_alpha(const or_mesh *m, const or_config *cf, const double *u, double t) {
  return or_alpha_cells(m, cf, u, t, NULL, 0);
}

/* ------------------------------------------------------------------------ */
/* DG operator, eq. (DGSystem:Dis)                                          */
/* ------------------------------------------------------------------------ */
static void cell_L(const or_mesh *m, const or_config *cf, const double *u, double alpha, double t,
                   int64_t K, double Lout[4][6]) {
  int k = cf->k, nb = nbasis(k);
  cellgeo g;
  cell_geo(m, K, &g);
  double acc[4][6] = {{0}};
  /* volume term: |K| sum_mu w_mu F(u(x_mu)) . grad Psi_l(x_mu) */
  const double (*B)[3];
  const double *W;
  int N = vol_rule(k, &B, &W);
  for (int mu = 0; mu < N; ++mu) {
    double x, y, val[4], grad[4][2], hess[4][3], f1[4], f2[4];
    bary_point(&g, B[mu], &x, &y);
    eval_derivs(m, k, u, K, &g, x, y, val, grad, hess);
    euler_flux(val, cf->gamma, f1, f2);
    double xi, eta, psi[6], dpsi[12];
    ref_coords(&g, x, y, &xi, &eta);
    or_basis(xi, eta, psi, dpsi, NULL);
    for (int l = 0; l < nb; ++l) {
      double px = dpsi[2 * l] * g.jinv[0][0] + dpsi[2 * l + 1] * g.jinv[1][0];
      double py = dpsi[2 * l] * g.jinv[0][1] + dpsi[2 * l + 1] * g.jinv[1][1];
      for (int c = 0; c < 4; ++c) acc[c][l] += g.area * W[mu] * (f1[c] * px + f2[c] * py);
    }
  }
  /* edge term: sum_i l_i sum_nu w_nu Fhat(u_int, u_ext, n_i) Psi_l(x_i,nu) */
  double s[3], w[3];
  int Q = edge_rule(k, s, w);
  for (int i = 0; i < 3; ++i) {
    int a = (i + 1) % 3, b = (i + 2) % 3;
    for (int nu = 0; nu < Q; ++nu) {
      double x = g.v[a][0] + (g.v[b][0] - g.v[a][0]) * s[nu];
      double y = g.v[a][1] + (g.v[b][1] - g.v[a][1]) * s[nu];
      double uin[4], uex[4], fh[4];
      eval_at(m, k, u, K, &g, x, y, uin);
      exterior_trace(m, cf, u, K, i, g.n[i], x, y, t, uin, uex);
      lf_flux(uin, uex, g.n[i], alpha, cf->gamma, fh);
      double xi, eta, psi[6];
      ref_coords(&g, x, y, &xi, &eta);
      or_basis(xi, eta, psi, NULL, NULL);
      for (int l = 0; l < nb; ++l)
        for (int c = 0; c < 4; ++c) acc[c][l] -= g.len[i] * w[nu] * fh[c] * psi[l];
    }
  }
  /* divide by the mass a_K^(l) */
  double cm[6];
  or_mass_constants(k, cm);
  for (int c = 0; c < 4; ++c)
    for (int l = 0; l < nb; ++l) Lout[c][l] = acc[c][l] / (cm[l] * g.area);
}

int or_L(const or_mesh *m, const or_config *cf, const double *u, double alpha, double t, double *L,
         const int64_t *cells, int64_t ncells) {
  if (cf->k != 1 && cf->k != 2) return OR_EINVAL;
  int nb = nbasis(cf->k);
  int64_t n = cells ? ncells : m->nt;
#pragma omp parallel for schedule(static)
  for (int64_t j = 0; j < n; ++j) {
    int64_t K = cells ? cells[j] : j;
    double Lc[4][6];
    cell_L(m, cf, u, alpha, t, K, Lc);
    for (int c = 0; c < 4; ++c)
      for (int l = 0; l < nb; ++l) L[((int64_t)c * nb + l) * m->nt + K] = Lc[c][l];
  }
  return OR_OK;
}

/* SSP-RK3 stage combination, eq. (RKTime) with the OE / BP steps of Sec. 4.5 */
int or_rk_stage(const or_mesh *m, const or_config *cf, const double *un, const double *v, double a,
                double b, double dt, double alpha, double t, double *uh, const int64_t *cells,
                int64_t ncells) {
  if (cf->k != 1 && cf->k != 2) return OR_EINVAL;
  int nb = nbasis(cf->k);
  int64_t n = cells ? ncells : m->nt;
#pragma omp parallel for schedule(static)
  for (int64_t j = 0; j < n; ++j) {
    int64_t K = cells ? cells[j] : j;
    double Lc[4][6];
    cell_L(m, cf, v, alpha, t, K, Lc);
    for (int c = 0; c < 4; ++c)
      for (int l = 0; l < nb; ++l) {
        int64_t idx = ((int64_t)c * nb + l) * m->nt + K;
        uh[idx] = a * un[idx] + b * (v[idx] + dt * Lc[c][l]);
      }
  }
  return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Global statistics of the OE procedure (eqs. OEScalar:Coef2, normOmg,      */
/* RIOESys:Coef1): domain means and sup deviations at the volume points      */
/* ------------------------------------------------------------------------ */
int or_stats_cells(const or_mesh *m, const or_config *cf, const double *u, const int64_t *cells,
                   int64_t ncells, double *stats) {
  int k = cf->k, nb = nbasis(k);
  int64_t n = cells ? ncells : m->nt;
  double sum[4] = {0, 0, 0, 0}, omega = 0.0;
  for (int64_t K = 0; K < m->nt; ++K) {
    cellgeo g;
    cell_geo(m, K, &g);
    omega += g.area;
    for (int c = 0; c < 4; ++c) sum[c] += g.area * coef(u, m->nt, nb, c, 0, K);
  }
  double mean[4];
  for (int c = 0; c < 4; ++c) mean[c] = sum[c] / omega;
  double *dev = malloc(sizeof(double) * 5 * (n > 0 ? n : 1));
#pragma omp parallel for schedule(static)
  for (int64_t j = 0; j < n; ++j) {
    const int64_t K = cells ? cells[j] : j;
    cellgeo g;
    cell_geo(m, K, &g);
    const double (*B)[3];
    const double *W;
    int N = vol_rule(k, &B, &W);
    double d[5] = {0, 0, 0, 0, 0};
    for (int mu = 0; mu < N; ++mu) {
      double x, y, val[4];
      bary_point(&g, B[mu], &x, &y);
      eval_at(m, k, u, K, &g, x, y, val);
      double dr = fabs(val[0] - mean[0]);
      double dm = sqrt((val[1] - mean[1]) * (val[1] - mean[1]) + (val[2] - mean[2]) * (val[2] - mean[2]));
      double de = fabs(val[3] - mean[3]);
      double d1 = fabs(val[1] - mean[1]), d2 = fabs(val[2] - mean[2]);
      if (dr > d[0]) d[0] = dr;
      if (dm > d[1]) d[1] = dm;
      if (de > d[2]) d[2] = de;
      if (d1 > d[3]) d[3] = d1;
      if (d2 > d[4]) d[4] = d2;
    }
    for (int q = 0; q < 5; ++q) dev[5 * j + q] = d[q];
  }
  double D[5] = {0, 0, 0, 0, 0};
  for (int64_t j = 0; j < n; ++j)
    for (int q = 0; q < 5; ++q)
      if (dev[5 * j + q] > D[q]) D[q] = dev[5 * j + q];
  free(dev);
  for (int c = 0; c < 4; ++c) stats[c] = mean[c];
  stats[4] = D[0];
  stats[5] = D[1];
  stats[6] = D[2];
  stats[7] = omega;
  stats[8] = D[3];
  stats[9] = D[4];
  return OR_OK;
}

int or_stats(const or_mesh *m, const or_config *cf, const double *u, double *stats) {
  return or_stats_cells(m, cf, u, NULL, 0, stats);
}

/* ------------------------------------------------------------------------ */
/* OE procedure: eqs. (oe:sys), (OEScalar:Coef1), (OEScalar:Coef2),          */
/* (oe:sysdelta2), (RIOESys:CoefM/Coef1/Coef2) with the trapezoidal rule     */
/* ------------------------------------------------------------------------ */
/* ghost derivatives on a boundary edge (val, grad, hess of the 4 components) */
static void ghost_derivs(const or_config *cf, int tag, const double ubar[4], const double n[2], double x,
                         double y, double t, const double val[4], const double grad[4][2], const double hess[4][3],
                         double gv[4], double gg[4][2], double gh[4][3]) {
  if (tag == OR_BC_REFLECT) {
    /* mirror polynomial: q_g(x) = q(Rx) for rho, E; m_g(x) = R m(Rx); R = I - 2 n n^T */
    double R[2][2] = {{1.0 - 2.0 * n[0] * n[0], -2.0 * n[0] * n[1]},
                      {-2.0 * n[1] * n[0], 1.0 - 2.0 * n[1] * n[1]}};
    double H[4][2][2], Gm[2][2];
    for (int c = 0; c < 4; ++c) {
      H[c][0][0] = hess[c][0]; H[c][0][1] = H[c][1][0] = hess[c][1]; H[c][1][1] = hess[c][2];
    }
    /* R H R of every component */
    double RHR[4][2][2];
    for (int c = 0; c < 4; ++c)
      for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
          double s = 0.0;
          for (int p = 0; p < 2; ++p)
            for (int q = 0; q < 2; ++q) s += R[a][p] * H[c][p][q] * R[q][b];
          RHR[c][a][b] = s;
        }
    for (int c = 0; c < 4; c += 3) { /* rho and E */
      gv[c] = val[c];
      gg[c][0] = R[0][0] * grad[c][0] + R[0][1] * grad[c][1];
      gg[c][1] = R[1][0] * grad[c][0] + R[1][1] * grad[c][1];
      gh[c][0] = RHR[c][0][0]; gh[c][1] = RHR[c][0][1]; gh[c][2] = RHR[c][1][1];
    }
    /* momentum: value R m, gradient matrix R G R, Hessians sum_l R_kl (R H_l R) */
    for (int a = 0; a < 2; ++a) {
      gv[1 + a] = R[a][0] * val[1] + R[a][1] * val[2];
    }
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) {
        double s = 0.0;
        for (int p = 0; p < 2; ++p)
          for (int q = 0; q < 2; ++q) s += R[a][p] * grad[1 + p][q] * R[q][b];
        Gm[a][b] = s;
      }
    for (int a = 0; a < 2; ++a) {
      gg[1 + a][0] = Gm[a][0];
      gg[1 + a][1] = Gm[a][1];
      gh[1 + a][0] = R[a][0] * RHR[1][0][0] + R[a][1] * RHR[2][0][0];
      gh[1 + a][1] = R[a][0] * RHR[1][0][1] + R[a][1] * RHR[2][0][1];
      gh[1 + a][2] = R[a][0] * RHR[1][1][1] + R[a][1] * RHR[2][1][1];
    }
  } else { /* constant exterior states: Dirichlet, moving shock, the transmissive cell average */
    double st[4];
    ghost_state(cf, tag, val, ubar, n, x, y, t, st);
    for (int c = 0; c < 4; ++c) {
      gv[c] = st[c];
      gg[c][0] = gg[c][1] = 0.0;
      gh[c][0] = gh[c][1] = gh[c][2] = 0.0;
    }
  }
}

/* derivative d^alpha q with |alpha| = j listed as alpha_1 = j, j-1, ..., 0
 * (x-derivatives first), for a component given by value / grad / hess */
static int derivs_of_order(int j, double val, const double grad[2], const double hess[3], double out[3]) {
  if (j == 0) { out[0] = val; return 1; }
  if (j == 1) { out[0] = grad[0]; out[1] = grad[1]; return 2; }
  out[0] = hess[0]; out[1] = hess[1]; out[2] = hess[2];
  return 3;
}

static double binom(int j, int a) {
  double r = 1.0;
  for (int i = 1; i <= a; ++i) r = r * (j - a + i) / i;
  return r;
}

static double factorial(int j) { double r = 1.0; for (int i = 2; i <= j; ++i) r *= i; return r; }

/* sigma[c][j] of cell K, c in (rho, m1, m2, E), j = 0..k */
static void cell_sigma(const or_mesh *m, const or_config *cf, const double *u, const double *stats,
                       double t, int64_t K, double sigma[4][3]) {
  int k = cf->k;
  cellgeo g;
  cell_geo(m, K, &g);
  const double eps = 1e-12;
  double mean[4] = {stats[0], stats[1], stats[2], stats[3]};
  double mnorm = sqrt(mean[1] * mean[1] + mean[2] * mean[2]);
  /* normalisers and "constant component" tests (remark on round-off, Sec. 2.3 / 3.3) */
  double Drho = stats[4], Dm = stats[5], DE = stats[6], Dm1 = stats[8], Dm2 = stats[9];
  int const_rho = Drho <= eps * fmax(1.0, fabs(mean[0]));
  int const_E = DE <= eps * fmax(1.0, fabs(mean[3]));
  int const_m = Dm <= eps * fmax(1.0, mnorm);
  int const_m1 = Dm1 <= eps * fmax(1.0, fabs(mean[1]));
  int const_m2 = Dm2 <= eps * fmax(1.0, fabs(mean[2]));
  for (int c = 0; c < 4; ++c)
    for (int j = 0; j < 3; ++j) sigma[c][j] = 0.0;

  for (int i = 0; i < 3; ++i) {
    const double *n = g.n[i];
    double h = 2.0 * g.area / g.len[i];   /* sup distance to edge i: the altitude */
    int vc = (i + 1) % 3, vd = (i + 2) % 3;
    /* J[q][j]: trapezoidal approximation of (1/l) int sum_alpha C_j^a [d^alpha q]^2 ds;
     * q = 0 rho, 1 m_n, 2 m_t, 3 E, 4 m1, 5 m2 */
    double Jq[6][3] = {{0}};
    double beta = 0.0;
    for (int e = 0; e < 2; ++e) {
      int vv = e == 0 ? vc : vd;
      double x = g.v[vv][0], y = g.v[vv][1];
      double val[4], grad[4][2], hess[4][3];
      double ov[4], og[4][2], oh[4][3];
      eval_derivs(m, k, u, K, &g, x, y, val, grad, hess);
      int32_t nbc = m->nbr[3 * K + i];
      if (nbc >= 0) {
        cellgeo gn;
        cell_geo(m, nbc, &gn);
        eval_derivs(m, k, u, nbc, &gn, x + m->shift[6 * K + 2 * i], y + m->shift[6 * K + 2 * i + 1], ov, og, oh);
      } else {
        double ubar[4];
        cell_average(m, k, u, K, ubar);
        ghost_derivs(cf, m->bc[3 * K + i], ubar, n, x, y, t, val, grad, hess, ov, og, oh);
      }
      /* beta_K^(i): max spectral radius over both sides at both endpoints */
      double r1 = wave_speed(val, n, cf->gamma), r2 = wave_speed(ov, n, cf->gamma);
      if (r1 > beta || r1 != r1) beta = r1;
      if (r2 > beta || r2 != r2) beta = r2;
      /* jumps of the conservative components and of m_n, m_t (K's normal on both sides) */
      double jv[6], jg[6][2], jh[6][3];
      for (int c = 0; c < 4; ++c) {
        int q = c == 0 ? 0 : (c == 3 ? 3 : 3 + c); /* rho -> 0, m1 -> 4, m2 -> 5, E -> 3 */
        jv[q] = val[c] - ov[c];
        jg[q][0] = grad[c][0] - og[c][0];
        jg[q][1] = grad[c][1] - og[c][1];
        for (int r = 0; r < 3; ++r) jh[q][r] = hess[c][r] - oh[c][r];
      }
      /* m_n = m . n, m_t = -m1 n2 + m2 n1 (linear: the jump of m_n is n . jump of m) */
      jv[1] = jv[4] * n[0] + jv[5] * n[1];
      jv[2] = -jv[4] * n[1] + jv[5] * n[0];
      for (int r = 0; r < 2; ++r) {
        jg[1][r] = jg[4][r] * n[0] + jg[5][r] * n[1];
        jg[2][r] = -jg[4][r] * n[1] + jg[5][r] * n[0];
      }
      for (int r = 0; r < 3; ++r) {
        jh[1][r] = jh[4][r] * n[0] + jh[5][r] * n[1];
        jh[2][r] = -jh[4][r] * n[1] + jh[5][r] * n[0];
      }
      for (int q = 0; q < 6; ++q)
        for (int j = 0; j <= k; ++j) {
          double d[3];
          int cnt = derivs_of_order(j, jv[q], jg[q], jh[q], d);
          for (int a = 0; a < cnt; ++a) {
            int alpha1 = j - a;   /* listed x-derivatives first */
            Jq[q][j] += 0.5 * binom(j, alpha1) * d[a] * d[a];
          }
        }
    }
    for (int j = 0; j <= k; ++j) {
      double A = (2.0 * j + 1.0) / ((2.0 * k - 1.0) * factorial(j));
      double hj = pow(h, (double)j);
      double drho = const_rho ? 0.0 : A * hj * sqrt(Jq[0][j]) / Drho;
      double dE = const_E ? 0.0 : A * hj * sqrt(Jq[3][j]) / DE;
      double dm1, dm2;
      if (cf->oe == 2) { /* component-wise: each momentum component with its own normaliser */
        dm1 = const_m1 ? 0.0 : A * hj * sqrt(Jq[4][j]) / Dm1;
        dm2 = const_m2 ? 0.0 : A * hj * sqrt(Jq[5][j]) / Dm2;
      } else {           /* rotation invariant: max of the normal and tangential parts */
        double dmn = const_m ? 0.0 : A * hj * sqrt(Jq[1][j]) / Dm;
        double dmt = const_m ? 0.0 : A * hj * sqrt(Jq[2][j]) / Dm;
        dm1 = dm2 = dmn > dmt ? dmn : dmt;
      }
      double dd[4] = {drho, dm1, dm2, dE};
      for (int c = 0; c < 4; ++c)
        if (dd[c] != 0.0) sigma[c][j] += beta / h * dd[c];
    }
  }
}

int or_oe(const or_mesh *m, const or_config *cf, const double *u, double dt, const double *stats,
          double t, double *out, double *sigma, const int64_t *cells, int64_t ncells) {
  int k = cf->k, nb = nbasis(k);
  if (k != 1 && k != 2) return OR_EINVAL;
  int64_t n = cells ? ncells : m->nt;
#pragma omp parallel for schedule(static)
  for (int64_t jj = 0; jj < n; ++jj) {
    int64_t K = cells ? cells[jj] : jj;
    double sg[4][3];
    cell_sigma(m, cf, u, stats, t, K, sg);
    if (sigma)
      for (int c = 0; c < 4; ++c)
        for (int j = 0; j < 3; ++j) sigma[((int64_t)c * 3 + j) * m->nt + K] = sg[c][j];
    for (int c = 0; c < 4; ++c)
      for (int l = 0; l < nb; ++l) {
        int64_t idx = ((int64_t)c * nb + l) * m->nt + K;
        int deg = mode_degree(l);
        if (deg == 0) { out[idx] = u[idx]; continue; }   /* eq. (OE:m0) */
        double s = 0.0;
        for (int j = 0; j <= deg; ++j) s += sg[c][j];
        out[idx] = u[idx] * exp(-dt * s);
      }
  }
  return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Simplified BP limiter (Sec. 4.4, eqs. 1944 / 1981)                        */
/* ------------------------------------------------------------------------ */
/* points of the limiter: all edge Gauss points, then the decomposition's
 * extra points (P1: vertices v1, v2 of the sorted labelling; P2: the two
 * internal nodes); returns the number of points */
static int limiter_points(const or_mesh *m, const or_config *cf, int64_t K, const cellgeo *g,
                          double px[16], double py[16], int *n_edge_pts) {
  double s[3], w[3];
  int Q = edge_rule(cf->k, s, w), np = 0;
  for (int i = 0; i < 3; ++i) {
    int a = (i + 1) % 3, b = (i + 2) % 3;
    for (int nu = 0; nu < Q; ++nu) {
      px[np] = g->v[a][0] + (g->v[b][0] - g->v[a][0]) * s[nu];
      py[np] = g->v[a][1] + (g->v[b][1] - g->v[a][1]) * s[nu];
      ++np;
    }
  }
  *n_edge_pts = np;
  if (cf->decomp != 0) return np;   /* classical decomposition: edge points (+ u_* below) */
  double wd[3], om[2], nd[4], cfl[2];
  int32_t nn, lv[2];
  or_decomposition(m, cf->k, K, wd, om, nd, &nn, cfl, lv);
  if (cf->k == 1) {
    px[np] = g->v[lv[0]][0]; py[np] = g->v[lv[0]][1]; ++np;
    px[np] = g->v[lv[1]][0]; py[np] = g->v[lv[1]][1]; ++np;
  } else {
    px[np] = nd[0]; py[np] = nd[1]; ++np;
    px[np] = nd[2]; py[np] = nd[3]; ++np;
  }
  return np;
}

/* classical decomposition for P2: the weighted internal state u_* of Sec. 4.1
 * (edge weights w_i = 2 w_1^GL / 3 = 1/9) computed from edge Gauss values */
static void zxs_internal_state(const or_config *cf, const double *ubar, double pts[][4], double out[4]) {
  double s[3], w[3];
  int Q = edge_rule(cf->k, s, w);
  const double we = 1.0 / 9.0;
  for (int c = 0; c < 4; ++c) {
    double acc = 0.0;
    for (int i = 0; i < 3; ++i)
      for (int nu = 0; nu < Q; ++nu) acc += we * w[nu] * pts[i * Q + nu][c];
    out[c] = (ubar[c] - acc) / (1.0 - 3.0 * we);
  }
}

static int cell_limit(const or_mesh *m, const or_config *cf, const double *u, int64_t K, double *out,
                      int *nonphys) {
  int k = cf->k, nb = nbasis(k);
  cellgeo g;
  cell_geo(m, K, &g);
  double px[16], py[16];
  int ne, np = limiter_points(m, cf, K, &g, px, py, &ne);
  double c_[4][6];
  for (int c = 0; c < 4; ++c)
    for (int l = 0; l < nb; ++l) c_[c][l] = coef(u, m->nt, nb, c, l, K);
  double ubar[4] = {c_[0][0], c_[1][0], c_[2][0], c_[3][0]};
  *nonphys = 0;
  int limited = 0;
  double Ebar = int_energy(ubar);
  if (!(ubar[0] > 0.0) || !(Ebar > 0.0)) {
    *nonphys = 1;
  } else {
    /* Step 1: density */
    double pts[16][4];
    for (int p = 0; p < np; ++p) eval_at(m, k, u, K, &g, px[p], py[p], pts[p]);
    double rmin = INFINITY;
    for (int p = 0; p < np; ++p) rmin = fmin(rmin, pts[p][0]);
    if (cf->decomp != 0 && k == 2) {
      double us[4];
      zxs_internal_state(cf, ubar, pts, us);
      rmin = fmin(rmin, us[0]);
    }
    double eps1 = fmin(ubar[0], 1e-13);
    double th1 = 1.0;
    if (rmin < eps1) th1 = (ubar[0] - eps1) / (ubar[0] - rmin);
    if (th1 < 1.0) {
      limited = 1;
      for (int l = 1; l < nb; ++l) c_[0][l] *= th1;
    }
    /* Step 2: internal energy of the density-limited polynomial */
    double Emin = INFINITY;
    double tp[16][4];
    for (int p = 0; p < np; ++p) {
      double xi, eta, psi[6];
      ref_coords(&g, px[p], py[p], &xi, &eta);
      or_basis(xi, eta, psi, NULL, NULL);
      for (int c = 0; c < 4; ++c) {
        double sacc = 0.0;
        for (int l = 0; l < nb; ++l) sacc += c_[c][l] * psi[l];
        tp[p][c] = sacc;
      }
      Emin = fmin(Emin, int_energy(tp[p]));
    }
    if (cf->decomp != 0 && k == 2) {
      double us[4];
      zxs_internal_state(cf, ubar, tp, us);
      Emin = fmin(Emin, int_energy(us));
    }
    double eps2 = fmin(Ebar, 1e-13);
    double th2 = 1.0;
    if (Emin < eps2) th2 = (Ebar - eps2) / (Ebar - Emin);
    if (th2 < 1.0) {
      limited = 1;
      for (int c = 0; c < 4; ++c)
        for (int l = 1; l < nb; ++l) c_[c][l] *= th2;
    }
  }
  for (int c = 0; c < 4; ++c)
    for (int l = 0; l < nb; ++l) out[((int64_t)c * nb + l) * m->nt + K] = c_[c][l];
  return limited;
}

int or_limit(const or_mesh *m, const or_config *cf, const double *u, double *out, int64_t *counters,
             const int64_t *cells, int64_t ncells) {
  if (cf->k != 1 && cf->k != 2) return OR_EINVAL;
  int64_t n = cells ? ncells : m->nt;
  int64_t lim = 0, bad = 0;
#pragma omp parallel for schedule(static) reduction(+ : lim, bad)
  for (int64_t j = 0; j < n; ++j) {
    int64_t K = cells ? cells[j] : j;
    int np_ = 0;
    lim += cell_limit(m, cf, u, K, out, &np_);
    bad += np_;
  }
  if (counters) { counters[0] += lim; counters[1] += bad; }
  return OR_OK;
}

void or_point_minima(const or_mesh *m, const or_config *cf, const double *u, double *out) {
#pragma omp parallel for schedule(static)
  for (int64_t K = 0; K < m->nt; ++K) {
    cellgeo g;
    cell_geo(m, K, &g);
    double px[16], py[16];
    int ne, np = limiter_points(m, cf, K, &g, px, py, &ne);
    double rmin = INFINITY, emin = INFINITY;
    for (int p = 0; p < np; ++p) {
      double v[4];
      eval_at(m, cf->k, u, K, &g, px[p], py[p], v);
      rmin = fmin(rmin, v[0]);
      emin = fmin(emin, int_energy(v));
    }
    out[2 * K] = rmin;
    out[2 * K + 1] = emin;
  }
}

/* ------------------------------------------------------------------------ */
/* Fully discrete BP OEDG scheme (Sec. 4.5) with the BP time step (Sec. 5)   */
/* ------------------------------------------------------------------------ */
int or_step(const or_mesh *m, const or_config *cf, double *u, double *t, double t_end, double *dt_out,
            int64_t *counters) {
  int k = cf->k, nb = nbasis(k);
  if (k != 1 && k != 2) return OR_EINVAL;
  *dt_out = 0.0;
  if (!(*t < t_end)) return OR_OK;
  int64_t sz = 4 * (int64_t)nb * m->nt;
  double *un = malloc(sizeof(double) * sz), *v = malloc(sizeof(double) * sz);
  double *uh = malloc(sizeof(double) * sz), *tmp = malloc(sizeof(double) * sz);
  if (!un || !v || !uh || !tmp) { free(un); free(v); free(uh); free(tmp); return OR_ENOMEM; }
  memcpy(un, u, sizeof(double) * sz);
  memcpy(v, u, sizeof(double) * sz);
  const double A[3] = {0.0, 0.75, 1.0 / 3.0}, B[3] = {1.0, 0.25, 2.0 / 3.0};
  const double C_IN[3] = {0.0, 1.0, 0.5}, C_OUT[3] = {1.0, 0.5, 1.0};
  double min_ca = or_min_cfl_area(m, k, cf->decomp);
  double alpha1 = or_alpha(m, cf, un, *t);
  double dt = cf->cfl * min_ca / alpha1;   /* C_SSP = 1 for SSP-RK3 */
  int clamped = 0;
  if (*t + dt >= t_end) { dt = t_end - *t; clamped = 1; }
  int rc = OR_OK;
  int64_t lim[2] = {0, 0};
  for (int s = 0; s < 3; ++s) {
    double alpha = s == 0 ? alpha1 : or_alpha(m, cf, v, *t + C_IN[s] * dt);
    if (alpha * dt > min_ca * (1.0 + 1e-12) && counters) counters[2] += 1;
    or_rk_stage(m, cf, un, v, A[s], B[s], dt, alpha, *t + C_IN[s] * dt, uh, NULL, 0);
    if (cf->oe) {
      double stats[10];
      or_stats(m, cf, uh, stats);
      or_oe(m, cf, uh, dt, stats, *t + C_OUT[s] * dt, tmp, NULL, NULL, 0);
    } else {
      memcpy(tmp, uh, sizeof(double) * sz);
    }
    if (cf->bp) or_limit(m, cf, tmp, v, lim, NULL, 0);
    else memcpy(v, tmp, sizeof(double) * sz);
  }
  memcpy(u, v, sizeof(double) * sz);
  *t = clamped ? t_end : *t + dt;
  *dt_out = dt;
  if (counters) { counters[0] += lim[0]; counters[1] += lim[1]; counters[3] += 1; }
  if (lim[1] > 0) rc = OR_ENONPHYS;
  free(un); free(v); free(uh); free(tmp);
  return rc;
}

int or_advance(const or_mesh *m, const or_config *cf, double *u, double *t, double t_end, int64_t max_steps,
               int64_t *counters) {
  for (int64_t s = 0; s < max_steps && *t < t_end; ++s) {
    double dt;
    int rc = or_step(m, cf, u, t, t_end, &dt, counters);
    if (rc != OR_OK) return rc;
  }
  return OR_OK;
}

int or_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void or_set_num_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

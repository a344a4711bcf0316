/*
 * scalar.c -- plain FP64 oracle of the OEDG scheme for scalar conservation
 * laws u_t + div F(u) = 0 on triangles (Ding, Cui & Wu, arXiv 2409.09620,
 * Sec. 2), degrees k = 1, 2, 3.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite and the benchmark's CPU legs
 * load this library; it shares nothing with the CUDA path.
 *
 * Followed step by step:
 *   basis                 eq. (basisfunc), Psi^(0..9), kept as monomial tables
 *                         so that every derivative is exact
 *   DG operator L(u)      eq. (DGScalar:Dis) with the LF flux (fluxLF); N = 3,
 *                         6, 12 volume points (Appendix A) and Q = k + 1 Gauss
 *                         points per edge (Appendix B)
 *   OE procedure          eqs. (oe:scalar), (OEScalar:Coef1), (OEScalar:beta),
 *                         (OEScalar:Coef2) with the trapezoidal rule and the
 *                         round-off guard of Sec. 2.3; normaliser (normOmg)
 *   time stepping         SSP-RK(2,2) or SSP-RK(3,3) (eq. RKTime) with the OE
 *                         after every stage, the time step of Sec. 5
 *
 * State layout: u[l * nt + K], mode l in 0..nb-1 (nb = 3, 6, 10).
 * Readings where the paper is silent (the same as the CUDA path takes):
 * alpha^LF is the maximum of |F'(u) . n| over all edge Gauss points and both
 * traces of the stage input; the time step is fixed per step from the first
 * stage's alpha; the initial state is the L2 projection (no initial OE);
 * boundary edges: periodic through the mesh, transmissive = own trace,
 * constant state (tags 3..6) = bc_state, with zero derivatives in the OE.
 */
#include "oracle.h"
#include "oracle_mesh.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define SC_NB_MAX 10

/* ---- basis of eq. (basisfunc) as sums of c xi^p eta^q --------------------- */
typedef struct { double c; int p, q; } mono;
static const mono PSI0[] = {{1, 0, 0}};
static const mono PSI1[] = {{4, 1, 0}, {2, 0, 1}, {-2, 0, 0}};
static const mono PSI2[] = {{3, 0, 1}, {-1, 0, 0}};
static const mono PSI3[] = {{24, 2, 0}, {24, 1, 1}, {4, 0, 2}, {-24, 1, 0}, {-8, 0, 1}, {4, 0, 0}};
static const mono PSI4[] = {{20, 1, 1}, {10, 0, 2}, {-4, 1, 0}, {-12, 0, 1}, {2, 0, 0}};
static const mono PSI5[] = {{10, 0, 2}, {-8, 0, 1}, {1, 0, 0}};
static const mono PSI6[] = {{160, 3, 0}, {240, 2, 1}, {96, 1, 2}, {8, 0, 3}, {-240, 2, 0},
                            {-192, 1, 1}, {-24, 0, 2}, {96, 1, 0}, {24, 0, 1}, {-8, 0, 0}};
static const mono PSI7[] = {{168, 2, 1}, {168, 1, 2}, {28, 0, 3}, {-24, 2, 0}, {-192, 1, 1},
                            {-60, 0, 2}, {24, 1, 0}, {36, 0, 1}, {-4, 0, 0}};
static const mono PSI8[] = {{84, 1, 2}, {42, 0, 3}, {-48, 1, 1}, {-66, 0, 2}, {4, 1, 0}, {26, 0, 1}, {-2, 0, 0}};
static const mono PSI9[] = {{35, 0, 3}, {-45, 0, 2}, {15, 0, 1}, {-1, 0, 0}};
static const mono *const PSI[SC_NB_MAX] = {PSI0, PSI1, PSI2, PSI3, PSI4, PSI5, PSI6, PSI7, PSI8, PSI9};
static const int PSI_N[SC_NB_MAX] = {1, 3, 2, 6, 5, 3, 10, 9, 7, 4};

static int sc_nb(int k) { return (k + 1) * (k + 2) / 2; }
static int sc_degree(int l) { return l == 0 ? 0 : l <= 2 ? 1 : l <= 5 ? 2 : 3; }

static double falling(int n, int r) {   /* n (n-1) ... (n-r+1) */
  double f = 1.0;
  for (int i = 0; i < r; ++i) f *= (double)(n - i);
  return f;
}

/* d^(r+s) Psi_l / d xi^r d eta^s at (xi, eta) */
static double psi_d(int l, int r, int s, double xi, double eta) {
  double v = 0.0;
  for (int t = 0; t < PSI_N[l]; ++t) {
    const mono mo = PSI[l][t];
    if (mo.p < r || mo.q < s) continue;
    v += mo.c * falling(mo.p, r) * falling(mo.q, s) * pow(xi, mo.p - r) * pow(eta, mo.q - s);
  }
  return v;
}

void or_sc_basis(double xi, double eta, int r, int s, double *out) {
  for (int l = 0; l < SC_NB_MAX; ++l) out[l] = psi_d(l, r, s, xi, eta);
}

/* a_K^(l) / |K|: integral of Psi_l^2 by the 12-point rule (exact to degree 6) */
void or_sc_mass_constants(int k, double *c) {
  int nb = sc_nb(k);
  for (int l = 0; l < nb; ++l) c[l] = 0.0;
  for (int mu = 0; mu < 12; ++mu)
    for (int l = 0; l < nb; ++l) {
      double p = psi_d(l, 0, 0, Q12_B[mu][1], Q12_B[mu][2]);
      c[l] += Q12_W[mu] * p * p;
    }
}

/* ---- quadrature ------------------------------------------------------------- */
static int sc_vol_rule(int k, const double (**b)[3], const double **w) {
  if (k == 1) { *b = Q3_B; *w = Q3_W; return 3; }
  if (k == 2) { *b = Q6_B; *w = Q6_W; return 6; }
  *b = Q12_B; *w = Q12_W; return 12;
}

/* Q = k + 1 Gauss-Legendre points on [-1, 1] mapped to s = (1 + x) / 2, w / 2 */
static int sc_edge_rule(int k, double *s, double *w) {
  double x[4], ww[4];
  int q = k + 1;
  if (q == 2) {
    x[0] = -1.0 / sqrt(3.0); x[1] = -x[0]; ww[0] = ww[1] = 1.0;
  } else if (q == 3) {
    x[0] = -sqrt(0.6); x[1] = 0.0; x[2] = sqrt(0.6); ww[0] = ww[2] = 5.0 / 9.0; ww[1] = 8.0 / 9.0;
  } else {
    double a = sqrt(3.0 / 7.0 - 2.0 / 7.0 * sqrt(6.0 / 5.0)), b = sqrt(3.0 / 7.0 + 2.0 / 7.0 * sqrt(6.0 / 5.0));
    x[0] = -b; x[1] = -a; x[2] = a; x[3] = b;
    ww[0] = ww[3] = (18.0 - sqrt(30.0)) / 36.0;
    ww[1] = ww[2] = (18.0 + sqrt(30.0)) / 36.0;
  }
  for (int i = 0; i < q; ++i) { s[i] = 0.5 * (1.0 + x[i]); w[i] = 0.5 * ww[i]; }
  return q;
}

/* ---- evaluation ---------------------------------------------------------------- */
static double sc_eval_ref(int k, const double *u, int64_t nt, int64_t K, double xi, double eta) {
  double v = 0.0;
  for (int l = 0; l < sc_nb(k); ++l) v += u[l * nt + K] * psi_d(l, 0, 0, xi, eta);
  return v;
}

static double sc_eval_phys(const or_mesh *m, int k, const double *u, int64_t K, double x, double y) {
  cellgeo g;
  cell_geo(m, K, &g);
  double xi, eta;
  ref_coords(&g, x, y, &xi, &eta);
  return sc_eval_ref(k, u, m->nt, K, xi, eta);
}

double or_sc_eval(const or_mesh *m, int k, const double *u, int64_t K, double x, double y) {
  return sc_eval_phys(m, k, u, K, x, y);
}

/* Physical derivative d^(p+q) u / dx^p dy^q of cell K's polynomial at (x, y).
 * The map is affine: d/dx = xi_x d/dxi + eta_x d/deta, d/dy = xi_y d/dxi +
 * eta_y d/deta, so d^p/dx^p d^q/dy^q is the product of these operators,
 * expanded here into coefficients of d^r/dxi^r d^(n-r)/deta^(n-r). */
static double sc_phys_deriv(const or_mesh *m, int k, const double *u, int64_t K, const cellgeo *g, double x,
                            double y, int p, int q) {
  double co[4] = {1.0, 0.0, 0.0, 0.0}, nx[4];   /* co[r]: coefficient of Dxi^r Deta^(deg - r) */
  int deg = 0;
  for (int f = 0; f < p + q; ++f) {
    const double a = f < p ? g->jinv[0][0] : g->jinv[0][1];   /* xi_x or xi_y */
    const double b = f < p ? g->jinv[1][0] : g->jinv[1][1];   /* eta_x or eta_y */
    for (int r = 0; r <= deg + 1; ++r) nx[r] = 0.0;
    for (int r = 0; r <= deg; ++r) {
      nx[r + 1] += a * co[r];    /* times a Dxi */
      nx[r] += b * co[r];        /* times b Deta */
    }
    ++deg;
    for (int r = 0; r <= deg; ++r) co[r] = nx[r];
  }
  double xi, eta;
  ref_coords(g, x, y, &xi, &eta);
  double v = 0.0;
  for (int r = 0; r <= deg; ++r) {
    if (co[r] == 0.0) continue;
    double d = 0.0;
    for (int l = 0; l < sc_nb(k); ++l) d += u[l * m->nt + K] * psi_d(l, r, deg - r, xi, eta);
    v += co[r] * d;
  }
  return v;
}

double or_sc_deriv(const or_mesh *m, int k, const double *u, int64_t K, double x, double y, int p, int q) {
  cellgeo g;
  cell_geo(m, K, &g);
  return sc_phys_deriv(m, k, u, K, &g, x, y, p, q);
}

/* ---- physics ---------------------------------------------------------------------- */
static void sc_flux(const or_sc_config *cf, double u, double f[2]) {
  if (cf->flux == 0) { f[0] = cf->ax * u; f[1] = cf->ay * u; }
  else { f[0] = 0.5 * u * u; f[1] = 0.5 * u * u; }
}

/* F'(u) . n */
static double sc_speed(const or_sc_config *cf, double u, const double n[2]) {
  return cf->flux == 0 ? cf->ax * n[0] + cf->ay * n[1] : u * (n[0] + n[1]);
}

/* exterior value at the physical point (x, y) of edge i of cell K */
static double sc_exterior(const or_mesh *m, const or_sc_config *cf, const double *u, int64_t K, int i, double x,
                          double y, double uin) {
  int32_t nbc = m->nbr[3 * K + i];
  if (nbc >= 0) return sc_eval_phys(m, cf->k, u, nbc, x + m->shift[6 * K + 2 * i], y + m->shift[6 * K + 2 * i + 1]);
  int tag = m->bc[3 * K + i];
  if (tag >= OR_BC_DIRICHLET0 && tag < OR_BC_DIRICHLET0 + 4) return cf->bc_state[tag - OR_BC_DIRICHLET0];
  return uin;   /* transmissive */
}

static int sc_check(const or_mesh *m, const or_sc_config *cf) {
  if (cf->k < 1 || cf->k > 3 || (cf->flux != 0 && cf->flux != 1) || (cf->rk != 2 && cf->rk != 3)) return OR_EINVAL;
  for (int64_t t = 0; t < 3 * m->nt; ++t)
    if (m->nbr[t] < 0 && !(m->bc[t] == OR_BC_TRANSMISSIVE ||
                           (m->bc[t] >= OR_BC_DIRICHLET0 && m->bc[t] < OR_BC_DIRICHLET0 + 4)))
      return OR_EINVAL;
  return OR_OK;
}

/* ---- alpha^LF: max |F'(u) . n| over the edge Gauss points, both traces ------------ */
double or_sc_alpha(const or_mesh *m, const or_sc_config *cf, const double *u) {
  double s[4], w[4];
  int q = sc_edge_rule(cf->k, s, w);
  double amax = 0.0;
#pragma omp parallel for reduction(max : amax) schedule(static)
  for (int64_t K = 0; K < m->nt; ++K) {
    cellgeo g;
    cell_geo(m, K, &g);
    for (int i = 0; i < 3; ++i) {
      int a = (i + 1) % 3, b = (i + 2) % 3;
      for (int nu = 0; nu < q; ++nu) {
        double x = g.v[a][0] + s[nu] * (g.v[b][0] - g.v[a][0]), y = g.v[a][1] + s[nu] * (g.v[b][1] - g.v[a][1]);
        double ui = sc_eval_phys(m, cf->k, u, K, x, y);
        double ue = sc_exterior(m, cf, u, K, i, x, y, ui);
        double r = fmax(fabs(sc_speed(cf, ui, g.n[i])), fabs(sc_speed(cf, ue, g.n[i])));
        if (r > amax) amax = r;
      }
    }
  }
  return amax;
}

/* ---- DG operator, eq. (DGScalar:Dis) ------------------------------------------------ */
static void sc_cell_L(const or_mesh *m, const or_sc_config *cf, const double *u, double alpha, int64_t K,
                      const double *cmass, double *Lout) {
  const int k = cf->k, nb = sc_nb(k);
  cellgeo g;
  cell_geo(m, K, &g);
  double acc[SC_NB_MAX] = {0};
  const double (*B)[3];
  const double *W;
  int nv = sc_vol_rule(k, &B, &W);
  for (int mu = 0; mu < nv; ++mu) {
    double xi = B[mu][1], eta = B[mu][2];
    double f[2];
    sc_flux(cf, sc_eval_ref(k, u, m->nt, K, xi, eta), f);
    for (int l = 0; l < nb; ++l) {
      double gx = psi_d(l, 1, 0, xi, eta) * g.jinv[0][0] + psi_d(l, 0, 1, xi, eta) * g.jinv[1][0];
      double gy = psi_d(l, 1, 0, xi, eta) * g.jinv[0][1] + psi_d(l, 0, 1, xi, eta) * g.jinv[1][1];
      acc[l] += g.area * W[mu] * (f[0] * gx + f[1] * gy);
    }
  }
  double s[4], w[4];
  int q = sc_edge_rule(k, s, w);
  for (int i = 0; i < 3; ++i) {
    int a = (i + 1) % 3, b = (i + 2) % 3;
    for (int nu = 0; nu < q; ++nu) {
      double x = g.v[a][0] + s[nu] * (g.v[b][0] - g.v[a][0]), y = g.v[a][1] + s[nu] * (g.v[b][1] - g.v[a][1]);
      double ui = sc_eval_phys(m, k, u, K, x, y);
      double ue = sc_exterior(m, cf, u, K, i, x, y, ui);
      double fi[2], fe[2];
      sc_flux(cf, ui, fi);
      sc_flux(cf, ue, fe);
      double fhat = 0.5 * ((fi[0] + fe[0]) * g.n[i][0] + (fi[1] + fe[1]) * g.n[i][1] - alpha * (ue - ui));
      double xi, eta;
      ref_coords(&g, x, y, &xi, &eta);
      for (int l = 0; l < nb; ++l) acc[l] -= g.len[i] * w[nu] * fhat * psi_d(l, 0, 0, xi, eta);
    }
  }
  for (int l = 0; l < nb; ++l) Lout[l] = acc[l] / (cmass[l] * g.area);
}

int or_sc_L(const or_mesh *m, const or_sc_config *cf, const double *u, double alpha, double *L) {
  int rc = sc_check(m, cf);
  if (rc) return rc;
  const int nb = sc_nb(cf->k);
  double cmass[SC_NB_MAX];
  or_sc_mass_constants(cf->k, cmass);
#pragma omp parallel for schedule(static)
  for (int64_t K = 0; K < m->nt; ++K) {
    double Lc[SC_NB_MAX];
    sc_cell_L(m, cf, u, alpha, K, cmass, Lc);
    for (int l = 0; l < nb; ++l) L[l * m->nt + K] = Lc[l];
  }
  return OR_OK;
}

/* ---- OE statistics: domain mean and the normaliser of eq. (normOmg) ---------------- */
void or_sc_stats(const or_mesh *m, const or_sc_config *cf, const double *u, double *stats) {
  double sum = 0.0, area = 0.0;
  for (int64_t K = 0; K < m->nt; ++K) {
    cellgeo g;
    cell_geo(m, K, &g);
    sum += g.area * u[K];
    area += g.area;
  }
  const double mean = sum / area;
  const double (*B)[3];
  const double *W;
  int nv = sc_vol_rule(cf->k, &B, &W);
  double dev = 0.0;
  for (int64_t K = 0; K < m->nt; ++K)
    for (int mu = 0; mu < nv; ++mu) dev = fmax(dev, fabs(sc_eval_ref(cf->k, u, m->nt, K, B[mu][1], B[mu][2]) - mean));
  stats[0] = mean;
  stats[1] = dev;
  stats[2] = area;
}

/* ---- OE procedure, eqs. (oe:scalar), (OEScalar:Coef1/beta/Coef2) -------------------- */
static void sc_cell_sigma(const or_mesh *m, const or_sc_config *cf, const double *u, const double *stats,
                          int64_t K, double sigma[4]) {
  const int k = cf->k;
  cellgeo g;
  cell_geo(m, K, &g);
  const double mean = stats[0], D = stats[1];
  const int constant = D <= 1e-12 * fmax(1.0, fabs(mean));
  for (int j = 0; j <= k; ++j) sigma[j] = 0.0;
  if (constant) return;
  for (int i = 0; i < 3; ++i) {
    const int vc = (i + 1) % 3, vd = (i + 2) % 3;
    const int32_t nbc = m->nbr[3 * K + i];
    const int tag = m->bc[3 * K + i];
    const double h = 2.0 * g.area / g.len[i];
    cellgeo gn;
    if (nbc >= 0) cell_geo(m, nbc, &gn);
    double J[4] = {0, 0, 0, 0}, beta = 0.0;
    for (int e = 0; e < 2; ++e) {
      const int v = e == 0 ? vc : vd;
      const double x = g.v[v][0], y = g.v[v][1];
      const double xs = x + (nbc >= 0 ? m->shift[6 * K + 2 * i] : 0.0);
      const double ys = y + (nbc >= 0 ? m->shift[6 * K + 2 * i + 1] : 0.0);
      for (int j = 0; j <= k; ++j) {
        for (int a1 = 0; a1 <= j; ++a1) {
          const int a2 = j - a1;
          const double own = sc_phys_deriv(m, k, u, K, &g, x, y, a1, a2);
          double ext;
          if (nbc >= 0) ext = sc_phys_deriv(m, k, u, nbc, &gn, xs, ys, a1, a2);
          else if (tag >= OR_BC_DIRICHLET0 && tag < OR_BC_DIRICHLET0 + 4)
            ext = j == 0 ? cf->bc_state[tag - OR_BC_DIRICHLET0] : 0.0;
          else ext = own;   /* transmissive: the exterior is the interior polynomial */
          const double jump = own - ext;
          /* binomial C_j^{a1} */
          double cb = 1.0;
          for (int t = 0; t < a1; ++t) cb = cb * (double)(j - t) / (double)(t + 1);
          J[j] += 0.5 * cb * jump * jump;
          if (j == 0) beta = fmax(beta, fmax(fabs(sc_speed(cf, own, g.n[i])), fabs(sc_speed(cf, ext, g.n[i]))));
        }
      }
    }
    double fact = 1.0;
    for (int j = 0; j <= k; ++j) {
      if (j > 0) fact *= (double)j;
      const double A = (2.0 * j + 1.0) / ((2.0 * k - 1.0) * fact);
      const double delta = A * pow(h, (double)j) * sqrt(J[j]) / D;
      sigma[j] += beta / h * delta;
    }
  }
}

int or_sc_oe(const or_mesh *m, const or_sc_config *cf, const double *u, double dt, const double *stats,
             double *out, double *sigma_out) {
  int rc = sc_check(m, cf);
  if (rc) return rc;
  const int k = cf->k, nb = sc_nb(k);
#pragma omp parallel for schedule(static)
  for (int64_t K = 0; K < m->nt; ++K) {
    double sig[4];
    sc_cell_sigma(m, cf, u, stats, K, sig);
    if (sigma_out)
      for (int j = 0; j <= k; ++j) sigma_out[j * m->nt + K] = sig[j];
    for (int l = 0; l < nb; ++l) {
      const int md = sc_degree(l);
      double s = 0.0;
      for (int j = 0; j <= md; ++j) s += sig[j];
      out[l * m->nt + K] = l == 0 ? u[K] : u[l * m->nt + K] * exp(-dt * s);
    }
  }
  return OR_OK;
}

/* ---- time step of Sec. 5: C_SSP / alpha * min_K |K| / ((2k + 1) sum_i l_i) ----------- */
double or_sc_dt_base(const or_mesh *m, int k) {
  double mn = INFINITY;
  for (int64_t K = 0; K < m->nt; ++K) {
    cellgeo g;
    cell_geo(m, K, &g);
    mn = fmin(mn, g.area / ((2.0 * k + 1.0) * (g.len[0] + g.len[1] + g.len[2])));
  }
  return mn;
}

/* L2 projection with the 12-point rule; vals[K * 12 + mu] are point values */
int or_sc_project(const or_mesh *m, int k, const double *vals, double *coeffs) {
  if (k < 1 || k > 3) return OR_EINVAL;
  const int nb = sc_nb(k);
  double cmass[SC_NB_MAX];
  or_sc_mass_constants(k, cmass);
  for (int64_t K = 0; K < m->nt; ++K)
    for (int l = 0; l < nb; ++l) {
      double s = 0.0;
      for (int mu = 0; mu < 12; ++mu) s += Q12_W[mu] * vals[K * 12 + mu] * psi_d(l, 0, 0, Q12_B[mu][1], Q12_B[mu][2]);
      coeffs[l * m->nt + K] = s / cmass[l];
    }
  return OR_OK;
}

/* ---- one SSP-RK step with the OE after every stage ------------------------------------ */
int or_sc_step(const or_mesh *m, const or_sc_config *cf, double *u, double *t, double t_end, double *dt_out) {
  int rc = sc_check(m, cf);
  if (rc) return rc;
  const int64_t n = (int64_t)sc_nb(cf->k) * m->nt;
  double *un = malloc(n * sizeof(double)), *v = malloc(n * sizeof(double)), *L = malloc(n * sizeof(double)),
         *uh = malloc(n * sizeof(double));
  if (!un || !v || !L || !uh) { free(un); free(v); free(L); free(uh); return OR_ENOMEM; }
  memcpy(un, u, n * sizeof(double));
  memcpy(v, u, n * sizeof(double));
  double alpha = or_sc_alpha(m, cf, v);
  double dt = cf->cfl * or_sc_dt_base(m, cf->k) / alpha;
  if (*t + dt >= t_end) dt = t_end - *t;
  static const double A3[3] = {0.0, 0.75, 1.0 / 3.0}, B3[3] = {1.0, 0.25, 2.0 / 3.0};
  static const double A2[2] = {0.0, 0.5}, B2[2] = {1.0, 0.5};
  for (int st = 0; st < cf->rk; ++st) {
    const double a = cf->rk == 3 ? A3[st] : A2[st], b = cf->rk == 3 ? B3[st] : B2[st];
    if (st > 0) alpha = or_sc_alpha(m, cf, v);
    or_sc_L(m, cf, v, alpha, L);
    for (int64_t i = 0; i < n; ++i) uh[i] = a * un[i] + b * (v[i] + dt * L[i]);
    if (cf->oe) {
      double stats[3];
      or_sc_stats(m, cf, uh, stats);
      or_sc_oe(m, cf, uh, dt, stats, v, NULL);
    } else {
      memcpy(v, uh, n * sizeof(double));
    }
  }
  memcpy(u, v, n * sizeof(double));
  *t = dt == t_end - *t ? t_end : *t + dt;
  if (dt_out) *dt_out = dt;
  free(un); free(v); free(L); free(uh);
  return OR_OK;
}

int or_sc_advance(const or_mesh *m, const or_sc_config *cf, double *u, double *t, double t_end, int64_t max_steps,
                  int64_t *steps) {
  int64_t s = 0;
  while (*t < t_end && s < max_steps) {
    int rc = or_sc_step(m, cf, u, t, t_end, NULL);
    if (rc) return rc;
    ++s;
  }
  if (steps) *steps = s;
  return OR_OK;
}

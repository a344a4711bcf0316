/*
 * oracle.h -- plain FP64 CPU oracle of the BP RI-OEDG stage for the 2D Euler
 * equations on triangles (Ding, Cui & Wu, arXiv 2409.09620).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark load this library.  It shares no code,
 * header, table or helper with the CUDA path, and it never calls it.
 *
 * Layout of a modal state: u[(c * nb + l) * nt + K] with component
 * c in (rho, m1, m2, E), mode l in 0..nb-1 (nb = 3 for P1, 6 for P2) and
 * cell K in 0..nt-1.
 */
#ifndef DG_ORACLE_H
#define DG_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define OR_OK 0
#define OR_EINVAL (-1)
#define OR_EMESH (-2)
#define OR_ENOMEM (-3)
#define OR_ENONPHYS (-4)

/* boundary tags of an edge without a neighbour */
#define OR_BC_NONE 0
#define OR_BC_REFLECT 1
#define OR_BC_TRANSMISSIVE 2
#define OR_BC_DIRICHLET0 3 /* 3..6: constant states 0..3 */
#define OR_BC_SHOCK 7

typedef struct or_config {
  int32_t k;        /* polynomial degree: 1 or 2 */
  int32_t oe;       /* 0 off, 1 rotation-invariant OE (Sec. 3.3), 2 component-wise OE (Sec. 3.2) */
  int32_t bp;       /* 0 off, 1 BP limiter at the decomposition points (Sec. 4.4) */
  int32_t decomp;   /* 0 optimal decomposition (Sec. 4.2), 1 classical Zhang-Xia-Shu */
  double gamma;     /* adiabatic index */
  double cfl;       /* multiplies the BP time step of Sec. 5 (1 = paper) */
  double bc_state[4][4];     /* conservative Dirichlet states */
  double shock_x0;           /* moving shock: foot on y = 0 at t = 0 */
  double shock_angle;        /* angle of the shock line to the x-axis */
  double shock_speed;        /* normal speed of the shock */
  int32_t shock_pre, shock_post; /* indices into bc_state */
} or_config;

typedef struct or_mesh or_mesh;

int or_mesh_create(int64_t nv, const double *xy, int64_t nt, const int32_t *tri,
                   const int32_t *canon, const int8_t *bc, or_mesh **out);
void or_mesh_destroy(or_mesh *m);
int64_t or_mesh_nt(const or_mesh *m);
/* neighbour cell and its local edge per (cell, edge); -1 on a boundary */
void or_mesh_neighbors(const or_mesh *m, int32_t *nbr, int32_t *nbr_edge);
/* per cell: area, edge lengths [3], outward normals [3][2] */
void or_mesh_geometry(const or_mesh *m, double *area, double *len, double *normal);

/* Decomposition of one cell (Sec. 4.2):
 * w[3] edge weights (original local edge order), omega[2] internal-node
 * weights, nodes[2][2] internal nodes, *n_nodes (0, 1 or 2), cfl[2] =
 * (C_DCW_{K,k}, C_ZXS_{K,k}), limv[2] = local ids of the P1 limiter vertices
 * (opposite the longest and second longest edges). */
int or_decomposition(const or_mesh *m, int k, int64_t K, double *w, double *omega,
                     double *nodes, int32_t *n_nodes, double *cfl, int32_t *limv);
/* min over cells of C_{K,k} |K| for the optimal (decomp=0) or ZXS decomposition */
double or_min_cfl_area(const or_mesh *m, int k, int decomp);

/* basis functions of eq. (basisfunc) and their reference derivatives */
void or_basis(double xi, double eta, double *psi, double *dpsi /*[6][2]*/,
              double *d2psi /*[6][3]*/);
/* mass a_K^(l) / |K| by the 12-point rule */
void or_mass_constants(int k, double *c);

/* physical points of the 12-point rule: xy[(K * 12 + mu) * 2 + d] */
void or_quad12_points(const or_mesh *m, double *xy);
/* L2 projection; vals[(K * 12 + mu) * 4 + c] are point values of the state */
int or_project(const or_mesh *m, int k, const double *vals, double *coeffs);
/* evaluate cell K's polynomial at physical (x, y) */
void or_eval(const or_mesh *m, int k, const double *u, int64_t K, double x, double y,
             double *out4);

/* alpha: max wave speed over edge Gauss points (eq. 1250) */
double or_alpha(const or_mesh *m, const or_config *cf, const double *u, double t);
/* the same maximum over a subset of the cells (cells == NULL: all); it reads
 * only those cells' own coefficients */
double or_alpha_cells(const or_mesh *m, const or_config *cf, const double *u, double t,
                      const int64_t *cells, int64_t ncells);
/* DG operator L(u) (eq. DGSystem:Dis); cells == NULL means all cells */
int or_L(const or_mesh *m, const or_config *cf, const double *u, double alpha, double t,
         double *L, const int64_t *cells, int64_t ncells);
/* u_h = a * un + b * (v + dt * L(v)) */
int or_rk_stage(const or_mesh *m, const or_config *cf, const double *un, const double *v,
                double a, double b, double dt, double alpha, double t, double *uh,
                const int64_t *cells, int64_t ncells);
/* global statistics of OE: stats[0..3] = domain means, stats[4..6] = sup
 * deviations of rho, |m - mean m| and E at the volume points, stats[7] =
 * |Omega|, stats[8..9] = sup deviations of m1 and m2 (component-wise OE) */
int or_stats(const or_mesh *m, const or_config *cf, const double *u, double *stats);
/* the same with the sup deviations taken over a subset of the cells (cells ==
 * NULL: all); the domain means still sum the cell averages (mode 0) of every
 * cell, in cell order, so only mode 0 of the other cells is read */
int or_stats_cells(const or_mesh *m, const or_config *cf, const double *u, const int64_t *cells,
                   int64_t ncells, double *stats);
/* OE procedure F_tau; sigma (nullable) receives sigma[(c * 3 + j) * nt + K] */
int or_oe(const or_mesh *m, const or_config *cf, const double *u, double dt,
          const double *stats, double t, double *out, double *sigma,
          const int64_t *cells, int64_t ncells);
/* simplified BP limiter; counters[0] += cells with theta < 1,
 * counters[1] += cells with a non-admissible average */
int or_limit(const or_mesh *m, const or_config *cf, const double *u, double *out,
             int64_t *counters, const int64_t *cells, int64_t ncells);
/* minimum of rho and of rho-weighted internal energy over the limiter point
 * set of each cell: out[2 * K + 0 / 1] */
void or_point_minima(const or_mesh *m, const or_config *cf, const double *u, double *out);
/* one SSP-RK3 step of the BP RI-OEDG scheme (Sec. 4.5); counters[0..3]:
 * limited cells, non-admissible averages, CFL breaches, steps */
int or_step(const or_mesh *m, const or_config *cf, double *u, double *t, double t_end,
            double *dt_out, int64_t *counters);
int or_advance(const or_mesh *m, const or_config *cf, double *u, double *t, double t_end,
               int64_t max_steps, int64_t *counters);
int or_num_threads(void);
/* threads of the OpenMP loops from now on (n > 0) */
void or_set_num_threads(int n);

/* ------------------------------------------------------------------------ */
/* Scalar conservation laws u_t + div F(u) = 0, P1-P3 OEDG (Sec. 2; scalar.c)
 * State layout: u[l * nt + K], nb = (k + 1)(k + 2) / 2 modes.               */
/* ------------------------------------------------------------------------ */
typedef struct or_sc_config {
  int32_t k;          /* 1, 2 or 3 */
  int32_t flux;       /* 0: linear F = (ax u, ay u); 1: Burgers F = (u^2/2, u^2/2) */
  int32_t oe;         /* 0 off, 1 OE procedure after every stage (eq. oe:scalar) */
  int32_t rk;         /* 2: SSP-RK(2,2); 3: SSP-RK(3,3) (eq. RKTime) */
  double ax, ay;      /* velocity of the linear flux */
  double cfl;         /* multiplies the time step of Sec. 5 */
  double bc_state[4]; /* values of the constant-state boundary tags 3..6 */
} or_sc_config;

/* d^(r+s) Psi_l / d xi^r d eta^s at (xi, eta), l = 0..9 (eq. basisfunc) */
void or_sc_basis(double xi, double eta, int r, int s, double *out10);
void or_sc_mass_constants(int k, double *c);
double or_sc_eval(const or_mesh *m, int k, const double *u, int64_t K, double x, double y);
/* physical derivative d^(p+q) u / dx^p dy^q of cell K's polynomial at (x, y) */
double or_sc_deriv(const or_mesh *m, int k, const double *u, int64_t K, double x, double y, int p, int q);
/* vals[K * 12 + mu]: values at the 12-point rule's points (or_quad12_points) */
int or_sc_project(const or_mesh *m, int k, const double *vals, double *coeffs);
double or_sc_alpha(const or_mesh *m, const or_sc_config *cf, const double *u);
int or_sc_L(const or_mesh *m, const or_sc_config *cf, const double *u, double alpha, double *L);
/* stats[0] = domain mean, stats[1] = sup |u - mean| at the volume points, stats[2] = |Omega| */
void or_sc_stats(const or_mesh *m, const or_sc_config *cf, const double *u, double *stats);
/* OE procedure; sigma (nullable) receives sigma[j * nt + K], j = 0..k */
int or_sc_oe(const or_mesh *m, const or_sc_config *cf, const double *u, double dt, const double *stats,
             double *out, double *sigma);
/* min_K |K| / ((2k + 1) sum_i l_K^(i)) */
double or_sc_dt_base(const or_mesh *m, int k);
int or_sc_step(const or_mesh *m, const or_sc_config *cf, double *u, double *t, double t_end, double *dt_out);
int or_sc_advance(const or_mesh *m, const or_sc_config *cf, double *u, double *t, double t_end,
                  int64_t max_steps, int64_t *steps);

#ifdef __cplusplus
}
#endif
#endif

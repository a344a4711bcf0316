/*
 * oracle_mesh.h -- internal to the oracle (TEST INFRASTRUCTURE ONLY): the mesh
 * record, the per-cell geometry of Sec. 2 and the volume quadrature rules of
 * Appendix A, shared by the Euler (oracle.c) and scalar (scalar.c) parts.
 */
#ifndef DG_ORACLE_MESH_H
#define DG_ORACLE_MESH_H
#include <math.h>
#include <stdint.h>

struct or_mesh {
  int64_t nv, nt;
  double *xy;       /* [2 nv] */
  int32_t *tri;     /* [3 nt] */
  int32_t *canon;   /* [nv] */
  int8_t *bc;       /* [3 nt] */
  int32_t *nbr;     /* [3 nt] neighbour cell or -1 */
  int32_t *nbr_edge;/* [3 nt] */
  double *shift;    /* [6 nt] neighbour copy of a point = point + shift */
};

/* ------------------------------------------------------------------------ */
/* Geometry of a cell (Sec. 2: notation, Fig. 1; affine map of Sec. 2.1)     */
/* ------------------------------------------------------------------------ */
typedef struct {
  double v[3][2];     /* vertices v1, v2, v3 (counter-clockwise) */
  double area;        /* |K| = det(J_K) / 2 */
  double jinv[2][2];  /* d(xi, eta) / d(x, y) */
  double len[3];      /* l_K^(i), edge i opposite vertex i */
  double n[3][2];     /* outward unit normal of edge i */
} cellgeo;

static inline void cell_geo(const or_mesh *m, int64_t K, cellgeo *g) {
  for (int i = 0; i < 3; ++i) {
    int32_t v = m->tri[3 * K + i];
    g->v[i][0] = m->xy[2 * v];
    g->v[i][1] = m->xy[2 * v + 1];
  }
  /* J_K = [[x2 - x1, x3 - x1], [y2 - y1, y3 - y1]] */
  double J00 = g->v[1][0] - g->v[0][0], J01 = g->v[2][0] - g->v[0][0];
  double J10 = g->v[1][1] - g->v[0][1], J11 = g->v[2][1] - g->v[0][1];
  double det = J00 * J11 - J01 * J10;
  g->area = 0.5 * det;
  g->jinv[0][0] = J11 / det;
  g->jinv[0][1] = -J01 / det;
  g->jinv[1][0] = -J10 / det;
  g->jinv[1][1] = J00 / det;
  for (int i = 0; i < 3; ++i) {
    int a = (i + 1) % 3, b = (i + 2) % 3;
    double dx = g->v[b][0] - g->v[a][0], dy = g->v[b][1] - g->v[a][1];
    double l = sqrt(dx * dx + dy * dy);
    g->len[i] = l;
    g->n[i][0] = dy / l;   /* counter-clockwise edge: outward normal is (dy, -dx) / l */
    g->n[i][1] = -dx / l;
  }
}

static inline void ref_coords(const cellgeo *g, double x, double y, double *xi, double *eta) {
  double dx = x - g->v[0][0], dy = y - g->v[0][1];
  *xi = g->jinv[0][0] * dx + g->jinv[0][1] * dy;
  *eta = g->jinv[1][0] * dx + g->jinv[1][1] * dy;
}

/* ------------------------------------------------------------------------ */
/* Quadrature rules (Appendix A tables 2th, 4th, 6th; Appendix B)            */
/* ------------------------------------------------------------------------ */
static const double Q3_B[3][3] = {
    {1.0 / 6.0, 1.0 / 6.0, 2.0 / 3.0}, {1.0 / 6.0, 2.0 / 3.0, 1.0 / 6.0}, {2.0 / 3.0, 1.0 / 6.0, 1.0 / 6.0}};
static const double Q3_W[3] = {1.0 / 3.0, 1.0 / 3.0, 1.0 / 3.0};
static const double Q6_B[6][3] = {
    {0.445948490915965, 0.445948490915965, 0.108103018168070},
    {0.445948490915965, 0.108103018168070, 0.445948490915965},
    {0.108103018168070, 0.445948490915965, 0.445948490915965},
    {0.091576213509771, 0.091576213509771, 0.816847572980458},
    {0.091576213509771, 0.816847572980458, 0.091576213509771},
    {0.816847572980458, 0.091576213509771, 0.091576213509771}};
static const double Q6_W[6] = {0.223381589678010, 0.223381589678010, 0.223381589678010,
                               0.109951743655322, 0.109951743655322, 0.109951743655322};
static const double Q12_B[12][3] = {
    {0.063089014491502, 0.063089014491502, 0.873821971016996},
    {0.063089014491502, 0.873821971016996, 0.063089014491502},
    {0.873821971016996, 0.063089014491502, 0.063089014491502},
    {0.249286745170910, 0.249286745170910, 0.501426509658180},
    {0.249286745170910, 0.501426509658180, 0.249286745170910},
    {0.501426509658180, 0.249286745170910, 0.249286745170910},
    {0.053145049844817, 0.636502499121399, 0.310352451033784},
    {0.636502499121399, 0.053145049844817, 0.310352451033784},
    {0.053145049844817, 0.310352451033784, 0.636502499121399},
    {0.636502499121399, 0.310352451033784, 0.053145049844817},
    {0.310352451033784, 0.053145049844817, 0.636502499121399},
    {0.310352451033784, 0.636502499121399, 0.053145049844817}};
static const double Q12_W[12] = {0.050844906370207, 0.050844906370207, 0.050844906370207,
                                 0.116786275726379, 0.116786275726379, 0.116786275726379,
                                 0.082851075618374, 0.082851075618374, 0.082851075618374,
                                 0.082851075618374, 0.082851075618374, 0.082851075618374};

#endif

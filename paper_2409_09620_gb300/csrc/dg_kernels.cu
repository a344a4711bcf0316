// dg_kernels.cu -- kernel instantiations and launch wrappers of the GB300
// BP RI-OEDG solver: mesh geometry / optimal convex decomposition, the three
// stage kernels and the fixed-order reductions between them.
#include "dg_internal.h"
#include <algorithm>

#include "dg_stage.cuh"

namespace dg {

struct OpMinD {
  __device__ double operator()(double a, double b) const { return a < b ? a : b; }
  template <typename T> __device__ static T ident() { return T(INFINITY); }
};

// ==========================================================================
// Geometry and optimal convex decomposition (Sec. 4.2, eqs. 1040, 1139;
// BP CFL numbers eqs. 1692, 1713; classical ZXS numbers of Sec. 4.3)
// ==========================================================================
__global__ void __launch_bounds__(TPB) k_geometry(int64_t nt, const double *__restrict__ vxy, double *area,
                                                  double *jinv, double *nrm, double *len, double *hgeo,
                                                  double *node, int8_t *limv, double *c_area, double *part_min,
                                                  float *jinv_f, float *nrm_f, float *len_f, float *hgeo_f,
                                                  double *iarea, float *node_f, double *psi_node) {
  const int64_t K = (int64_t)blockIdx.x * TPB + threadIdx.x;
  double mins[4] = {INFINITY, INFINITY, INFINITY, INFINITY};
  if (K < nt) {
    double x[3], y[3];
#pragma unroll
    for (int v = 0; v < 3; ++v) { x[v] = vxy[(2 * v) * nt + K]; y[v] = vxy[(2 * v + 1) * nt + K]; }
    const double J00 = x[1] - x[0], J01 = x[2] - x[0], J10 = y[1] - y[0], J11 = y[2] - y[0];
    const double det = J00 * J11 - J01 * J10;
    const double ar = 0.5 * det;
    area[K] = ar;
    jinv[K] = J11 / det;
    jinv[nt + K] = -J01 / det;
    jinv[2 * nt + K] = -J10 / det;
    jinv[3 * nt + K] = J00 / det;
    double l[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const int a = (i + 1) % 3, b = (i + 2) % 3;
      const double dx = x[b] - x[a], dy = y[b] - y[a];
      l[i] = sqrt(dx * dx + dy * dy);
      len[i * nt + K] = l[i];
      nrm[(2 * i) * nt + K] = dy / l[i];
      nrm[(2 * i + 1) * nt + K] = -dx / l[i];
      // h_K^(i) = sup distance of K to edge i = the altitude 2|K| / l_i (OE coefficient, Sec. 2.3)
      hgeo[i * nt + K] = 2.0 * ar / l[i];
      hgeo[(3 + i) * nt + K] = l[i] / (2.0 * ar);
    }
    // relabel edges longest first (stable)
    int p0 = 0, p1 = 1, p2 = 2, tmp;
    if (l[p0] < l[p1]) { tmp = p0; p0 = p1; p1 = tmp; }
    if (l[p1] < l[p2]) { tmp = p1; p1 = p2; p2 = tmp; }
    if (l[p0] < l[p1]) { tmp = p0; p0 = p1; p1 = tmp; }
    const double l1 = l[p0], l2 = l[p1], l3 = l[p2];
    const double lb = (l1 + l2 + l3) / 3.0;
    const double lh = sqrt(l1 * l1 + l2 * l2 + l3 * l3 - (2.0 / 3.0) * (l1 * l2 + l2 * l3 + l3 * l1));
    limv[K] = (int8_t)p0;
    limv[nt + K] = (int8_t)p1;
    // two internal nodes of the P2 decomposition as barycentric weights of the
    // sorted vertices; (xi, eta) = weights of the original vertices 2 and 3
    const double r = 1.7320508075688772;   // sqrt(3)
    // quadratic forms l^T M_{s,i} l: entries (M00, M11, M22, M01, M02, M12)
    const double Mq[2][3][6] = {
        {{6, 6 + 2 * r, 6, 1, -2, -r - 2}, {6, 12, 6, -r - 2, -2, r - 2}, {6, 6 - 2 * r, 6, r - 2, -2, 1}},
        {{6, 6 - 2 * r, 6, 1, -2, r - 2}, {6, 12, 6, r - 2, -2, -r - 2}, {6, 6 + 2 * r, 6, -r - 2, -2, 1}}};
    const double cq[2][3] = {{3 * l1 + 3 * l2 + r * (l2 - l3), 6 * l2 + r * (l3 - l1), 3 * l2 + 3 * l3 + r * (l1 - l2)},
                             {3 * l1 + 3 * l2 + r * (l3 - l2), 6 * l2 + r * (l1 - l3), 3 * l2 + 3 * l3 + r * (l2 - l1)}};
    const double den = 18.0 * (lb + lh) * (l2 + lh);
    const int perm[3] = {p0, p1, p2};
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      double bary[3] = {0.0, 0.0, 0.0};
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const double *M = Mq[s][i];
        const double qf = M[0] * l1 * l1 + M[1] * l2 * l2 + M[2] * l3 * l3 +
                          2.0 * (M[3] * l1 * l2 + M[4] * l1 * l3 + M[5] * l2 * l3);
        bary[perm[i]] = (qf + 2.0 * cq[s][i] * lh) / den;
      }
      node[(2 * s) * nt + K] = bary[1];
      node[(2 * s + 1) * nt + K] = bary[2];
      // the P2 basis at the node, for the FP64 limiter
#pragma unroll
      for (int l = 1; l < 6; ++l) psi_node[(5 * s + l - 1) * nt + K] = psi(l, bary[1], bary[2]);
    }
    iarea[K] = 1.0 / ar;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      jinv_f[q * nt + K] = float(jinv[q * nt + K]);
      node_f[q * nt + K] = float(node[q * nt + K]);
    }
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      nrm_f[q * nt + K] = float(nrm[q * nt + K]);
      hgeo_f[q * nt + K] = float(hgeo[q * nt + K]);
    }
#pragma unroll
    for (int q = 0; q < 3; ++q) len_f[q * nt + K] = float(len[q * nt + K]);
    const double cs[4] = {2.0 / (3.0 * (l1 + l2)), 1.0 / (9.0 * lb), 2.0 / (9.0 * lb + 3.0 * lh), 1.0 / (27.0 * lb)};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      c_area[q * nt + K] = cs[q] * ar;
      mins[q] = cs[q] * ar;
    }
  }
  block_reduce<4>(mins, part_min + 4 * blockIdx.x, OpMinD());
}

// ==========================================================================
// Fixed-order reductions of block partials (one block)
// ==========================================================================
__global__ void k_fin_min4(const double *part, int nblk, double *out) {
  double r[4];
  fin_reduce<4>(part, nblk, (double)INFINITY, OpMinD(), r);
  if (threadIdx.x == 0)
    for (int q = 0; q < 4; ++q) out[q] = r[q];
}

// Finalize kernels: block g reduces tile group g (TILE_GROUP tiles) of the
// stage kernel's partials; the block that takes the last top-level ticket
// reduces the group results and writes the scalars (see finish_*_top).
__global__ void __launch_bounds__(TPB) k_fin_mean(const double *part, FinBufs f, int64_t ntiles, Scalars *sc) {
  if (!sc->active) return;
  reduce_group<4>(part, blockIdx.x, ntiles, f.grp_sum, OpSum());
  finish_means_top(f, ntiles, sc);
}
__global__ void __launch_bounds__(TPB) k_fin_dev(const double *part, FinBufs f, int64_t ntiles, Scalars *sc, int cw) {
  if (!sc->active) return;
  reduce_group<5>(part, blockIdx.x, ntiles, f.grp_dev, OpMaxNN());
  finish_deviations_top(f, ntiles, sc, cw);
}
__global__ void __launch_bounds__(TPB) k_fin_alpha(const double *pa, const long long *pc, FinBufs f, int64_t ntiles,
                                                   Scalars *sc, int stage) {
  if (!sc->active) return;
  reduce_group<1>(pa, blockIdx.x, ntiles, f.grp_alpha, OpMaxNN());
  reduce_group<2>(pc, blockIdx.x, ntiles, f.grp_cnt, OpSum());
  finish_alpha_top(f, ntiles, sc, stage);
}

__global__ void k_step_begin(Scalars *sc) {
  if (threadIdx.x == 0) step_begin_thread(sc);
}

__global__ void k_set_inv_normalisers(Scalars *sc, int cw) {
  if (threadIdx.x == 0) write_inv_normalisers(sc, cw);
}

__global__ void k_set_active(Scalars *sc, int active) {
  if (threadIdx.x == 0) sc->active = active;
}

// ==========================================================================
// Launch wrappers
// ==========================================================================
static inline unsigned nblocks(int64_t nt) { return (unsigned)((nt + TPB - 1) / TPB); }

void launch_geometry(cudaStream_t s, int64_t nt, const double *vxy, const GeomPtrs &g, double *part_min,
                     double *out_min4) {
  const unsigned nb = nblocks(nt);
  k_geometry<<<nb, TPB, 0, s>>>(nt, vxy, g.area, g.jinv, g.nrm, g.len, g.hgeo, g.node, g.limv, g.c_area, part_min,
                                g.jinv_f, g.nrm_f, g.len_f, g.hgeo_f, g.iarea, g.node_f, g.psi_node);
  k_fin_min4<<<1, FIN_THREADS, 0, s>>>(part_min, (int)nb, out_min4);
}

template <int K, typename Real>
static void rk_impl(cudaStream_t s, const MeshDev &m, const Phys &ph, StateDev<Real> v, StateDev<Real> un,
                    StateDev<Real> uh, const void *tr, void *vd, void *hs, double *part_sum, const Scalars *sc,
                    double a, double b, double c_in) {
  k_rk<K, Real><<<nblocks(m.nt), TPB, 0, s>>>(m, ph, v, un, uh, (const Real *)tr, (Real *)vd, (Real *)hs, part_sum,
                                              sc, a, b, c_in);
}
template <int K, typename Real>
static void stats_impl(cudaStream_t s, const MeshDev &m, const Phys &ph, StateDev<Real> uh, double *part_dev,
                       const void *vd, const void *hs, void *ej, const Scalars *sc, double c_out) {
  k_stats<K, Real><<<nblocks(m.nt), TPB, 0, s>>>(m, ph, uh, part_dev, (const Real *)vd, (const Real *)hs, (Real *)ej,
                                                 sc, c_out);
}
template <int K, typename Real>
static void oebp_impl(cudaStream_t s, const MeshDev &m, const Phys &ph, StateDev<Real> uh, StateDev<Real> out,
                      const void *ej, void *tr, double *pa, long long *pc, const Scalars *sc, int do_oe,
                      int do_bp, double c_out, int end_of_step) {
  k_oe_bp<K, Real><<<nblocks(m.nt), TPB, 0, s>>>(m, ph, uh, out, (const Real *)ej, (Real *)tr, pa, pc, sc, do_oe,
                                                 do_bp, c_out, end_of_step);
}

#define DG_DISPATCH(K_, PREC_, CALL)                        \
  do {                                                       \
    if ((PREC_) == 0) {                                      \
      using Real = double;                                   \
      if ((K_) == 1) { constexpr int KK = 1; CALL; }         \
      else { constexpr int KK = 2; CALL; }                   \
    } else {                                                 \
      using Real = float;                                    \
      if ((K_) == 1) { constexpr int KK = 1; CALL; }         \
      else { constexpr int KK = 2; CALL; }                   \
    }                                                        \
  } while (0)

// k_rk: volume + edge fluxes + RK combination, block sums of |K| u_h^(0)
void launch_rk_only(const StageCtx &c, const StateBuf &v, const StateBuf &un, const StateBuf &uh, double a,
                    double b, double c_in) {
  DG_DISPATCH(c.k, c.prec,
              (rk_impl<KK, Real>(c.stream, c.mesh, c.phys, {v.avg, (Real *)v.hi}, {un.avg, (Real *)un.hi},
                                 {uh.avg, (Real *)uh.hi}, c.tr, c.vd, c.hs, c.part_sum, c.sc, a, b, c_in)));
}

void launch_fin_mean(const StageCtx &c) {
  const int64_t nt = nblocks(c.mesh.nt);
  k_fin_mean<<<(unsigned)num_groups(nt), TPB, 0, c.stream>>>(c.part_sum, c.fin, nt, c.sc);
}

void launch_rk(const StageCtx &c, const StateBuf &v, const StateBuf &un, const StateBuf &uh, double a, double b,
               double c_in) {
  launch_rk_only(c, v, un, uh, a, b, c_in);
  launch_fin_mean(c);
}

// k_stats: deviation maxima at the volume points and the edge OE records
void launch_stats_only(const StageCtx &c, const StateBuf &uh, double c_out) {
  DG_DISPATCH(c.k, c.prec,
              (stats_impl<KK, Real>(c.stream, c.mesh, c.phys, {uh.avg, (Real *)uh.hi}, c.part_dev, c.vd, c.hs, c.ej,
                                    c.sc, c_out)));
}

void launch_fin_dev(const StageCtx &c) {
  const int64_t nt = nblocks(c.mesh.nt);
  k_fin_dev<<<(unsigned)num_groups(nt), TPB, 0, c.stream>>>(c.part_dev, c.fin, nt, c.sc, c.phys.oe == 2);
}

void launch_stats(const StageCtx &c, const StateBuf &uh, double c_out) {
  launch_stats_only(c, uh, c_out);
  launch_fin_dev(c);
}

// k_oe_bp: RIOE + limiter + traces, block maxima of the wave speed and counters
void launch_oe_bp_only(const StageCtx &c, const StateBuf &uh, const StateBuf &out, int do_oe, int do_bp,
                       double c_out, int end_of_step) {
  DG_DISPATCH(c.k, c.prec,
              (oebp_impl<KK, Real>(c.stream, c.mesh, c.phys, {uh.avg, (Real *)uh.hi}, {out.avg, (Real *)out.hi}, c.ej,
                                   c.tr, c.part_alpha, c.part_cnt, c.sc, do_oe, do_bp, c_out, end_of_step)));
}

// alpha and counters; after stage 2 also t += dt (stage < 0: outside a step)
void launch_fin_alpha(const StageCtx &c, int stage) {
  const int64_t nt = nblocks(c.mesh.nt);
  k_fin_alpha<<<(unsigned)num_groups(nt), TPB, 0, c.stream>>>(c.part_alpha, c.part_cnt, c.fin, nt, c.sc, stage);
}

void launch_oe_bp(const StageCtx &c, const StateBuf &uh, const StateBuf &out, int do_oe, int do_bp, double c_out,
                  int stage) {
  launch_oe_bp_only(c, uh, out, do_oe, do_bp, c_out, stage == 2);
  launch_fin_alpha(c, stage);
}

void launch_step_begin(const StageCtx &c) { k_step_begin<<<1, 32, 0, c.stream>>>(c.sc); }
void launch_set_active(const StageCtx &c, int active) { k_set_active<<<1, 32, 0, c.stream>>>(c.sc, active); }
void launch_set_inv_normalisers(const StageCtx &c) {
  k_set_inv_normalisers<<<1, 32, 0, c.stream>>>(c.sc, c.phys.oe == 2);
}

int64_t num_blocks(int64_t nt) { return nblocks(nt); }

size_t stage_kernels_local_bytes(int k, int prec) {
  size_t n = 0;
  DG_DISPATCH(k, prec, (n = std::max({kernel_local_bytes(k_rk<KK, Real>), kernel_local_bytes(k_stats<KK, Real>),
                                      kernel_local_bytes(k_oe_bp<KK, Real>)})));
  return n;
}

}  // namespace dg

// dg_scalar.cu -- the OEDG scheme for scalar conservation laws
// u_t + div F(u) = 0 on triangles (Ding, Cui & Wu, arXiv 2409.09620, Sec. 2),
// P1-P3, FP64: F(u) = (a1 u, a2 u) (linear convection) or (u^2/2, u^2/2)
// (Burgers).  One thread per cell; per RK stage
//
//   k_sc_rk     volume quadrature (N = 3, 6, 12 points, Appendix A), LF
//               fluxes (eq. fluxLF) against the neighbours' traces, mass
//               inverse and RK combination (eqs. DGScalar:Dis, RKTime), and
//               block sums of |K| u^(0)
//   k_sc_stats  sup |u - mean| at the volume points (eq. normOmg) and the
//               new state's physical derivatives up to order k at the three
//               vertices
//   k_sc_oe     sigma from the vertex jumps of every edge (eqs. OEScalar:Coef1,
//               OEScalar:beta, OEScalar:Coef2 with the trapezoidal rule), the
//               exact damping (eq. oe:scalar), traces of the result at the Q =
//               k + 1 edge Gauss points and block maxima of |F'(u) . n|
//
// with finalize kernels in the fixed two-level order of the Euler path.  The
// time step is Sec. 5's C_SSP / alpha * min_K |K| / ((2k + 1) sum_i l_K^(i)).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/dg.h"
#include "dg_internal.h"

namespace dg {
namespace sc {

// --------------------------------------------------------------------------
// Basis of eq. (basisfunc), modes 0..9, and its reference derivatives.  Each
// mode is a sum of terms c xi^p eta^q; d^(r+s)/dxi^r deta^s is taken term by
// term.  constexpr, so evaluations at fixed points fold to constants.
// --------------------------------------------------------------------------
// flat (non-recursive) helpers for exponents and orders up to 3, so that the
// optimiser folds every evaluation at the fixed points into a constant
__host__ __device__ constexpr double ipow(double x, int n) {
  return n <= 0 ? 1.0 : n == 1 ? x : n == 2 ? x * x : x * x * x;
}
__host__ __device__ constexpr double fall(int n, int r) {   // n (n-1) ... (n-r+1)
  return r <= 0 ? 1.0 : r == 1 ? double(n) : r == 2 ? double(n * (n - 1)) : double(n * (n - 1) * (n - 2));
}
__host__ __device__ constexpr double term(double c, int p, int q, int r, int s, double x, double y) {
  return (r > p || s > q) ? 0.0 : c * fall(p, r) * fall(q, s) * ipow(x, p - r) * ipow(y, q - s);
}
__host__ __device__ constexpr double psi_rs(int l, int r, int s, double x, double y) {
#define T(c, p, q) term(c, p, q, r, s, x, y)
  return l == 0 ? T(1, 0, 0)
       : l == 1 ? T(4, 1, 0) + T(2, 0, 1) + T(-2, 0, 0)
       : l == 2 ? T(3, 0, 1) + T(-1, 0, 0)
       : l == 3 ? T(24, 2, 0) + T(24, 1, 1) + T(4, 0, 2) + T(-24, 1, 0) + T(-8, 0, 1) + T(4, 0, 0)
       : l == 4 ? T(20, 1, 1) + T(10, 0, 2) + T(-4, 1, 0) + T(-12, 0, 1) + T(2, 0, 0)
       : l == 5 ? T(10, 0, 2) + T(-8, 0, 1) + T(1, 0, 0)
       : l == 6 ? T(160, 3, 0) + T(240, 2, 1) + T(96, 1, 2) + T(8, 0, 3) + T(-240, 2, 0) + T(-192, 1, 1) +
                      T(-24, 0, 2) + T(96, 1, 0) + T(24, 0, 1) + T(-8, 0, 0)
       : l == 7 ? T(168, 2, 1) + T(168, 1, 2) + T(28, 0, 3) + T(-24, 2, 0) + T(-192, 1, 1) + T(-60, 0, 2) +
                      T(24, 1, 0) + T(36, 0, 1) + T(-4, 0, 0)
       : l == 8 ? T(84, 1, 2) + T(42, 0, 3) + T(-48, 1, 1) + T(-66, 0, 2) + T(4, 1, 0) + T(26, 0, 1) + T(-2, 0, 0)
                : T(35, 0, 3) + T(-45, 0, 2) + T(15, 0, 1) + T(-1, 0, 0);
#undef T
}
// a_K^(l) / |K| (exact rationals: 1, 2/3, 1/2, 16/15, 4/9, 1/3, 16/7, 4/5, 1/3, 1/4)
__host__ __device__ constexpr double sc_inv_mass(int l) {
  return l == 0 ? 1.0 : l == 1 ? 1.5 : l == 2 ? 2.0 : l == 3 ? 0.9375 : l == 4 ? 2.25 : l == 5 ? 3.0
       : l == 6 ? 7.0 / 16.0 : l == 7 ? 1.25 : l == 8 ? 3.0 : 4.0;
}
__host__ __device__ constexpr int sc_degree(int l) { return l == 0 ? 0 : l <= 2 ? 1 : l <= 5 ? 2 : 3; }

template <int K> struct SDeg {
  static constexpr int NB = (K + 1) * (K + 2) / 2;     // modes; also derivatives up to order K per vertex
  static constexpr int NQ = K + 1;                     // edge Gauss points
  static constexpr int NV = K == 1 ? 3 : K == 2 ? 6 : 12;
};

// volume rules of Appendix A (tab:2th, tab:4th, tab:6th): (xi, eta) = (b2, b3)
__host__ __device__ constexpr double q12_b(int mu, int c) {
  return mu == 0 ? (c == 1 ? 0.063089014491502 : 0.873821971016996)
       : mu == 1 ? (c == 1 ? 0.873821971016996 : 0.063089014491502)
       : mu == 2 ? 0.063089014491502
       : mu == 3 ? (c == 1 ? 0.249286745170910 : 0.501426509658180)
       : mu == 4 ? (c == 1 ? 0.501426509658180 : 0.249286745170910)
       : mu == 5 ? 0.249286745170910
       : mu == 6 ? (c == 1 ? 0.636502499121399 : 0.310352451033784)
       : mu == 7 ? (c == 1 ? 0.053145049844817 : 0.310352451033784)
       : mu == 8 ? (c == 1 ? 0.310352451033784 : 0.636502499121399)
       : mu == 9 ? (c == 1 ? 0.310352451033784 : 0.053145049844817)
       : mu == 10 ? (c == 1 ? 0.053145049844817 : 0.636502499121399)
                  : (c == 1 ? 0.636502499121399 : 0.053145049844817);
}
__host__ __device__ constexpr double q12_w(int mu) {
  return mu < 3 ? 0.050844906370207 : mu < 6 ? 0.116786275726379 : 0.082851075618374;
}
__host__ __device__ constexpr double svol_xi(int NV, int mu) { return NV == 12 ? q12_b(mu, 1) : vol_xi(NV, mu); }
__host__ __device__ constexpr double svol_eta(int NV, int mu) { return NV == 12 ? q12_b(mu, 2) : vol_eta(NV, mu); }
__host__ __device__ constexpr double svol_w(int NV, int mu) { return NV == 12 ? q12_w(mu) : vol_w(NV, mu); }

// Q-point Gauss-Legendre rule on an edge, s in (0, 1), weights summing to 1
// (Appendix B with reading R2); Q = 4: nodes +-sqrt(3/7 -+ 2/7 sqrt(6/5))
__host__ __device__ constexpr double sgauss_s(int Q, int nu) {
  return Q < 4 ? gauss_s(Q, nu)
       : nu == 0 ? 0.069431844202973713 : nu == 1 ? 0.33000947820757187 : nu == 2 ? 0.66999052179242813
                 : 0.93056815579702629;
}
__host__ __device__ constexpr double sgauss_w(int Q, int nu) {
  return Q < 4 ? gauss_w(Q, nu) : (nu == 0 || nu == 3) ? 0.17392742256872693 : 0.32607257743127307;
}

// ---- device scalars of one solver ------------------------------------------------
struct ScScalars {
  double t, t_end, dt, alpha, cfl, dt_base, mean, area_total, dev, inv_dev;
  long long steps;
  int active, clamped;
};

struct ScPhys {
  int flux;            // 0 linear, 1 Burgers
  double ax, ay;
  double bc[4];        // constant-state boundary values (tags 3..6)
};

__device__ __forceinline__ void sflux(const ScPhys &ph, double u, double &f0, double &f1) {
  if (ph.flux == 0) { f0 = ph.ax * u; f1 = ph.ay * u; }
  else { f0 = f1 = 0.5 * u * u; }
}
__device__ __forceinline__ double sspeed(const ScPhys &ph, double u, double nx, double ny) {
  return ph.flux == 0 ? ph.ax * nx + ph.ay * ny : u * (nx + ny);
}
// exterior value at a boundary edge (tag > 0): constant state or the interior value
__device__ __forceinline__ double sghost(const ScPhys &ph, int tag, double uin) {
  return (tag >= DG_BC_DIRICHLET0 && tag < DG_BC_DIRICHLET0 + 4) ? ph.bc[tag - DG_BC_DIRICHLET0] : uin;
}

// record of the derivatives d^j u / dx^a dy^(j-a) at a vertex: index of (j, a)
__host__ __device__ constexpr int didx(int j, int a) { return j * (j + 1) / 2 + (j - a); }

// ---- K1: volume + edge fluxes + RK combination ------------------------------------
template <int K>
__global__ void __launch_bounds__(TPB) k_sc_rk(MeshDev m, ScPhys ph, const double *__restrict__ v,
                                               const double *__restrict__ un, double *__restrict__ uh,
                                               const double *__restrict__ tr, double *part, const ScScalars *sc,
                                               double a, double b) {
  constexpr int NB = SDeg<K>::NB, NQ = SDeg<K>::NQ, NV = SDeg<K>::NV;
  if (!sc->active) return;
  const int64_t nt = m.nt;
  const int64_t Kc = (int64_t)blockIdx.x * TPB + threadIdx.x;
  double mass[1] = {0.0};
  if (Kc < nt) {
    const double dt = sc->dt, alpha = sc->alpha;
    const double area = m.area[Kc];
    const double jx = m.jinv[Kc], jy = m.jinv[nt + Kc], ex = m.jinv[2 * nt + Kc], ey = m.jinv[3 * nt + Kc];
    double c[NB], acc[NB];
#pragma unroll
    for (int l = 0; l < NB; ++l) { c[l] = v[l * nt + Kc]; acc[l] = 0.0; }
    // volume: |K| sum_mu w_mu F(u(x_mu)) . grad Psi_l
#pragma unroll
    for (int mu = 0; mu < NV; ++mu) {
      const double xi = svol_xi(NV, mu), eta = svol_eta(NV, mu), w = svol_w(NV, mu);
      double u = 0.0;
#pragma unroll
      for (int l = 0; l < NB; ++l) u = cfma(psi_rs(l, 0, 0, xi, eta), c[l], u);
      double f0, f1;
      sflux(ph, u, f0, f1);
      const double g1 = f0 * jx + f1 * jy, g2 = f0 * ex + f1 * ey;   // F . grad xi, F . grad eta
#pragma unroll
      for (int l = 1; l < NB; ++l) {
        acc[l] = cfma(w * psi_rs(l, 1, 0, xi, eta), g1, acc[l]);
        acc[l] = cfma(w * psi_rs(l, 0, 1, xi, eta), g2, acc[l]);
      }
    }
#pragma unroll
    for (int l = 1; l < NB; ++l) acc[l] *= area;
    // edges: - sum_i l_i sum_nu w_nu Fhat Psi_l
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const int32_t cn = m.conn[i * nt + Kc];
      const double nx = m.nrm[(2 * i) * nt + Kc], ny = m.nrm[(2 * i + 1) * nt + Kc], li = m.len[i * nt + Kc];
#pragma unroll
      for (int nu = 0; nu < NQ; ++nu) {
        const double um = tr[(Kc * 3 + i) * NQ + nu];
        const double up = cn >= 0 ? tr[((int64_t)(cn >> 2) * 3 + (cn & 3)) * NQ + (NQ - 1 - nu)] : sghost(ph, -cn, um);
        double fm0, fm1, fp0, fp1;
        sflux(ph, um, fm0, fm1);
        sflux(ph, up, fp0, fp1);
        const double fh = 0.5 * ((fm0 + fp0) * nx + (fm1 + fp1) * ny - alpha * (up - um));
        const double tv = li * sgauss_w(NQ, nu) * fh;
        const double s = sgauss_s(NQ, nu);
#pragma unroll
        for (int l = 0; l < NB; ++l) acc[l] = cfma(-psi_rs(l, 0, 0, edge_xi(i, s), edge_eta(i, s)), tv, acc[l]);
      }
    }
    // mass inverse and SSP-RK combination
    const double dta = dt / area;
    double h[NB];
#pragma unroll
    for (int l = 0; l < NB; ++l) {
      h[l] = a * un[l * nt + Kc] + b * (c[l] + dta * sc_inv_mass(l) * acc[l]);
      uh[l * nt + Kc] = h[l];
    }
    mass[0] = area * h[0];
  }
  block_reduce<1>(mass, part + blockIdx.x, OpSum());
}

// ---- K2: sup |u - mean| at the volume points; vertex derivative records ----------------
// The records hold d^j u / dx^p dy^(j-p), j <= K, at the three vertices (the
// affine map gives d/dx = xi_x d/dxi + eta_x d/deta, d/dy = xi_y d/dxi +
// eta_y d/deta), for the OE jumps of the neighbours and the cell itself.
template <int K>
__global__ void __launch_bounds__(TPB) k_sc_stats(MeshDev m, const double *__restrict__ u, double *__restrict__ vr,
                                                  double *part, const ScScalars *sc) {
  constexpr int NB = SDeg<K>::NB, NV = SDeg<K>::NV;
  if (!sc->active) return;
  const int64_t nt = m.nt;
  const int64_t Kc = (int64_t)blockIdx.x * TPB + threadIdx.x;
  double d[1] = {0.0};
  if (Kc < nt) {
    const double mean = sc->mean;
    double c[NB];
#pragma unroll
    for (int l = 0; l < NB; ++l) c[l] = u[l * nt + Kc];
#pragma unroll
    for (int mu = 0; mu < NV; ++mu) {
      double s = c[0] - mean;
#pragma unroll
      for (int l = 1; l < NB; ++l) s = cfma(psi_rs(l, 0, 0, svol_xi(NV, mu), svol_eta(NV, mu)), c[l], s);
      d[0] = max_nn(d[0], fabs(s));
    }
    const double jx = m.jinv[Kc], jy = m.jinv[nt + Kc], ex = m.jinv[2 * nt + Kc], ey = m.jinv[3 * nt + Kc];
    double *vo = vr + Kc * 3 * NB;
#pragma unroll
    for (int vv = 0; vv < 3; ++vv) {
      const double xi = vert_xi(vv), eta = vert_eta(vv);
#pragma unroll
      for (int j = 0; j <= K; ++j)
#pragma unroll
        for (int p = j; p >= 0; --p) {
          // expand (jx Dxi + ex Deta)^p (jy Dxi + ey Deta)^(j-p): co[r] multiplies Dxi^r Deta^(j-r)
          double co[K + 1];
#pragma unroll
          for (int r = 0; r <= K; ++r) co[r] = r == 0 ? 1.0 : 0.0;
#pragma unroll
          for (int f = 0; f < j; ++f) {
            const double fa = f < p ? jx : jy, fb = f < p ? ex : ey;
#pragma unroll
            for (int r = K; r >= 0; --r) co[r] = (r > 0 ? fa * co[r - 1] : 0.0) + fb * co[r];
          }
          double dv = 0.0;
#pragma unroll
          for (int r = 0; r <= j; ++r) {
            double ref = 0.0;   // d^j u / dxi^r deta^(j-r) at the vertex
#pragma unroll
            for (int l = 0; l < NB; ++l) ref = cfma(psi_rs(l, r, j - r, xi, eta), c[l], ref);
            dv += co[r] * ref;
          }
          vo[vv * NB + didx(j, p)] = dv;
        }
    }
  }
  block_reduce<1>(d, part + blockIdx.x, OpMaxNN());
}

// ---- K3: OE damping, traces and wave speeds ---------------------------------------------
template <int K>
__global__ void __launch_bounds__(TPB) k_sc_oe(MeshDev m, ScPhys ph, const double *__restrict__ uh,
                                               double *__restrict__ out, const double *__restrict__ vr,
                                               double *__restrict__ tr, double *part, const ScScalars *sc,
                                               int do_oe) {
  constexpr int NB = SDeg<K>::NB, NQ = SDeg<K>::NQ;
  if (!sc->active) return;
  const int64_t nt = m.nt;
  const int64_t Kc = (int64_t)blockIdx.x * TPB + threadIdx.x;
  double amax = 0.0;
  if (Kc < nt) {
    double c[NB];
#pragma unroll
    for (int l = 0; l < NB; ++l) c[l] = uh[l * nt + Kc];
    if (do_oe && sc->inv_dev != 0.0) {
      const double inv_dev = sc->inv_dev, dt = sc->dt;
      double sig[K + 1];
#pragma unroll
      for (int j = 0; j <= K; ++j) sig[j] = 0.0;
      const double *vme = vr + Kc * 3 * NB;
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const int32_t cn = m.conn[i * nt + Kc];
        const double nx = m.nrm[(2 * i) * nt + Kc], ny = m.nrm[(2 * i + 1) * nt + Kc];
        const double h = m.hgeo[i * nt + Kc], ih = m.hgeo[(3 + i) * nt + Kc];
        double J[K + 1];
#pragma unroll
        for (int j = 0; j <= K; ++j) J[j] = 0.0;
        double beta = 0.0;
#pragma unroll
        for (int ev = 0; ev < 2; ++ev) {
          const int ov = (i + 1 + ev) % 3;                 // v_c, then v_d
          const double *own = vme + ov * NB;
          const double *oth = cn >= 0 ? vr + ((int64_t)(cn >> 2) * 3 + ((cn & 3) + 2 - ev) % 3) * NB : nullptr;
          const bool dir = cn < 0 && (-cn) >= DG_BC_DIRICHLET0 && (-cn) < DG_BC_DIRICHLET0 + 4;
          const double u_own = own[0];
          const double u_ext = cn >= 0 ? oth[0] : (dir ? ph.bc[-cn - DG_BC_DIRICHLET0] : u_own);
          beta = max_nn(beta, max_nn(fabs(sspeed(ph, u_own, nx, ny)), fabs(sspeed(ph, u_ext, nx, ny))));
#pragma unroll
          for (int j = 0; j <= K; ++j) {
#pragma unroll
            for (int a = j; a >= 0; --a) {
              // C_j^a for the derivative d^j / dx^a dy^(j-a)
              double cb = 1.0;
#pragma unroll
              for (int t = 0; t < a; ++t) cb = cb * double(j - t) / double(t + 1);
              const double o = own[didx(j, a)];
              const double x = cn >= 0 ? oth[didx(j, a)] : (dir ? (j == 0 ? u_ext : 0.0) : o);
              const double jump = o - x;
              J[j] += 0.5 * cb * jump * jump;
            }
          }
        }
        // delta^j = A^{k,j} h^j sqrt(J_j) / D, sigma^j += beta / h delta^j
        double hj = 1.0, fact = 1.0;
#pragma unroll
        for (int j = 0; j <= K; ++j) {
          if (j > 0) fact *= double(j);
          const double A = (2.0 * j + 1.0) / ((2.0 * K - 1.0) * fact);
          sig[j] += beta * ih * (A * hj * sqrt(J[j]) * inv_dev);
          hj *= h;
        }
      }
      double fac[K + 1];
      double sacc = sig[0];
#pragma unroll
      for (int md = 1; md <= K; ++md) {
        sacc += sig[md];
        fac[md] = exp_neg(dt * sacc);
      }
#pragma unroll
      for (int l = 1; l < NB; ++l) c[l] *= fac[sc_degree(l)];
    }
#pragma unroll
    for (int l = 0; l < NB; ++l) out[l * nt + Kc] = c[l];
    // traces of the result at the edge Gauss points; wave speeds of the next stage's input
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const int32_t cn = m.conn[i * nt + Kc];
      const double nx = m.nrm[(2 * i) * nt + Kc], ny = m.nrm[(2 * i + 1) * nt + Kc];
#pragma unroll
      for (int nu = 0; nu < NQ; ++nu) {
        const double s = sgauss_s(NQ, nu);
        double u = 0.0;
#pragma unroll
        for (int l = 0; l < NB; ++l) u = cfma(psi_rs(l, 0, 0, edge_xi(i, s), edge_eta(i, s)), c[l], u);
        tr[(Kc * 3 + i) * NQ + nu] = u;
        amax = max_nn(amax, fabs(sspeed(ph, u, nx, ny)));
        if (cn < 0) amax = max_nn(amax, fabs(sspeed(ph, sghost(ph, -cn, u), nx, ny)));
      }
    }
  }
  double av[1] = {amax};
  block_reduce<1>(av, part + blockIdx.x, OpMaxNN());
}

// ---- finalize kernels (two-level fixed order) and the time step -------------------------
struct ScFin {
  double *grp;          // [ng]
  unsigned *tick;       // [3][ng + 1]
};

__global__ void __launch_bounds__(TPB) k_sc_fin(const double *part, ScFin f, int64_t ntiles, ScScalars *sc, int kind,
                                                int stage, int rk) {
  if (!sc->active) return;
  const int64_t ng = num_groups(ntiles);
  if (kind == 0) reduce_group<1>(part, blockIdx.x, ntiles, f.grp, OpSum());
  else reduce_group<1>(part, blockIdx.x, ntiles, f.grp, OpMaxNN());
  if (!take_ticket(f.tick + kind * (ng + 1) + ng, (unsigned)ng)) return;
  double r[1];
  if (kind == 0) reduce_top<1>(f.grp, ng, OpSum(), r);
  else reduce_top<1>(f.grp, ng, OpMaxNN(), r);
  if (threadIdx.x != 0) return;
  if (kind == 0) {
    sc->mean = r[0] / sc->area_total;
  } else if (kind == 1) {
    sc->dev = r[0];
    sc->inv_dev = r[0] <= 1e-12 * fmax(1.0, fabs(sc->mean)) ? 0.0 : 1.0 / r[0];   // Sec. 2.3 round-off guard
  } else {
    sc->alpha = r[0];
    if (stage == rk - 1) {
      sc->t = sc->clamped ? sc->t_end : sc->t + sc->dt;
      sc->steps += 1;
    }
  }
}

__global__ void k_sc_step_begin(ScScalars *sc) {
  if (threadIdx.x != 0) return;
  if (sc->t < sc->t_end) {
    double dt = sc->cfl * sc->dt_base / sc->alpha;
    int clamped = 0;
    if (sc->t + dt >= sc->t_end) { dt = sc->t_end - sc->t; clamped = 1; }
    sc->dt = dt;
    sc->clamped = clamped;
    sc->active = 1;
  } else {
    sc->dt = 0.0;
    sc->active = 0;
  }
}

struct ScOpMin {
  __device__ double operator()(double a, double b) const { return a < b ? a : b; }
  template <typename T> __device__ static T ident() { return T(INFINITY); }
};

// min_K |K| / ((2k + 1) sum_i l_i): block minima
__global__ void __launch_bounds__(TPB) k_sc_dt_base(MeshDev m, int k, double *part) {
  const int64_t Kc = (int64_t)blockIdx.x * TPB + threadIdx.x;
  double v[1] = {INFINITY};
  if (Kc < m.nt)
    v[0] = m.area[Kc] / ((2.0 * k + 1.0) * (m.len[Kc] + m.len[m.nt + Kc] + m.len[2 * m.nt + Kc]));
  block_reduce<1>(v, part + blockIdx.x, ScOpMin());
}

// errors against exact values at the 12-point rule's points: block partials of
// sum |K| w |e|, sum |K| w e^2, max |e|
template <int K>
__global__ void __launch_bounds__(TPB) k_sc_errors(MeshDev m, const double *__restrict__ u,
                                                   const double *__restrict__ exact, double *part) {
  constexpr int NB = SDeg<K>::NB;
  const int64_t nt = m.nt;
  const int64_t Kc = (int64_t)blockIdx.x * TPB + threadIdx.x;
  double e1[1] = {0.0}, e2[1] = {0.0}, ei[1] = {0.0};
  if (Kc < nt) {
    double c[NB];
#pragma unroll
    for (int l = 0; l < NB; ++l) c[l] = u[l * nt + Kc];
    const double area = m.area[Kc];
#pragma unroll
    for (int mu = 0; mu < 12; ++mu) {
      double s = 0.0;
#pragma unroll
      for (int l = 0; l < NB; ++l) s = cfma(psi_rs(l, 0, 0, q12_b(mu, 1), q12_b(mu, 2)), c[l], s);
      const double e = s - exact[Kc * 12 + mu];
      e1[0] += area * q12_w(mu) * fabs(e);
      e2[0] += area * q12_w(mu) * e * e;
      ei[0] = max_nn(ei[0], fabs(e));
    }
  }
  block_reduce<1>(e1, part + 3 * blockIdx.x, OpSum());
  block_reduce<1>(e2, part + 3 * blockIdx.x + 1, OpSum());
  block_reduce<1>(ei, part + 3 * blockIdx.x + 2, OpMaxNN());
}

#define SC_DISPATCH(K_, CALL)                                  \
  do {                                                          \
    if ((K_) == 1) { constexpr int KK = 1; CALL; }              \
    else if ((K_) == 2) { constexpr int KK = 2; CALL; }         \
    else { constexpr int KK = 3; CALL; }                        \
  } while (0)

}  // namespace sc
}  // namespace dg

using namespace dg;
using namespace dg::sc;

struct dg_scalar {
  const dg_mesh *mesh = nullptr;
  dg_scalar_config cfg{};
  int nb = 0;
  int64_t nt = 0, ntiles = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  MeshDev md{};
  ScPhys ph{};
  double *un = nullptr, *us = nullptr, *uh = nullptr, *tr = nullptr, *vr = nullptr, *part = nullptr;
  ScFin fin{};
  ScScalars *sc = nullptr;
  cudaGraphExec_t exec = nullptr;
  ~dg_scalar() {
    if (stream) cudaStreamSynchronize(stream);
    if (exec) cudaGraphExecDestroy(exec);
    cudaFree(un); cudaFree(us); cudaFree(uh); cudaFree(tr); cudaFree(vr); cudaFree(part);
    cudaFree(fin.grp); cudaFree(fin.tick); cudaFree(sc);
    if (own_stream && stream) cudaStreamDestroy(stream);
  }
};

namespace {

const double RK3_A[3] = {0.0, 0.75, 1.0 / 3.0}, RK3_B[3] = {1.0, 0.25, 2.0 / 3.0};
const double RK2_A[2] = {0.0, 0.5}, RK2_B[2] = {1.0, 0.5};

unsigned nblk(int64_t nt) { return (unsigned)((nt + TPB - 1) / TPB); }

void launch_fin(dg_scalar *s, int kind, int stage) {
  k_sc_fin<<<(unsigned)num_groups(s->ntiles), TPB, 0, s->stream>>>(s->part, s->fin, s->ntiles, s->sc, kind, stage,
                                                                   s->cfg.rk);
}

// traces and alpha of `src` written to `dst` (OE off): the state a step starts from
void launch_oe(dg_scalar *s, const double *src, double *dst, int do_oe, int stage) {
  SC_DISPATCH(s->cfg.k, (k_sc_oe<KK><<<nblk(s->nt), TPB, 0, s->stream>>>(s->md, s->ph, src, dst, s->vr, s->tr,
                                                                         s->part, s->sc, do_oe)));
  launch_fin(s, 2, stage);
}

// one SSP-RK step (Sec. 2.2) with the OE after every stage
void enqueue_step(dg_scalar *s) {
  k_sc_step_begin<<<1, 32, 0, s->stream>>>(s->sc);
  const int rk = s->cfg.rk;
  for (int st = 0; st < rk; ++st) {
    const double a = rk == 3 ? RK3_A[st] : RK2_A[st], b = rk == 3 ? RK3_B[st] : RK2_B[st];
    const double *v = st == 0 ? s->un : s->us;
    SC_DISPATCH(s->cfg.k, (k_sc_rk<KK><<<nblk(s->nt), TPB, 0, s->stream>>>(s->md, s->ph, v, s->un, s->uh, s->tr,
                                                                           s->part, s->sc, a, b)));
    launch_fin(s, 0, st);
    if (s->cfg.oe) {
      SC_DISPATCH(s->cfg.k,
                  (k_sc_stats<KK><<<nblk(s->nt), TPB, 0, s->stream>>>(s->md, s->uh, s->vr, s->part, s->sc)));
      launch_fin(s, 1, st);
    }
    launch_oe(s, s->uh, st == rk - 1 ? s->un : s->us, s->cfg.oe, st);
  }
}

int32_t read_sc(const dg_scalar *s, ScScalars *h) {
  cudaError_t e = cudaMemcpyAsync(h, s->sc, sizeof(ScScalars), cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return set_error(DG_ECUDA, cudaGetErrorString(e));
  return DG_OK;
}
int32_t write_sc(dg_scalar *s, const ScScalars *h) {
  cudaError_t e = cudaMemcpyAsync(s->sc, h, sizeof(ScScalars), cudaMemcpyHostToDevice, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return set_error(DG_ECUDA, cudaGetErrorString(e));
  return DG_OK;
}

}  // namespace

extern "C" int32_t dg_scalar_project(const dg_mesh *mesh, int32_t k, const double *vals, double *coeffs) {
  if (!mesh || !vals || !coeffs || k < 1 || k > 3) return set_error(DG_EINVAL, "dg_scalar_project: bad argument");
  int64_t nt = 0;
  const double *area = nullptr;
  double at = 0.0;
  mesh_view(mesh, &nt, &area, &at);
  const int nb = (k + 1) * (k + 2) / 2;
  for (int64_t K = 0; K < nt; ++K)
    for (int l = 0; l < nb; ++l) {
      double acc = 0.0;
      for (int mu = 0; mu < 12; ++mu) acc += q12_w(mu) * psi_rs(l, 0, 0, q12_b(mu, 1), q12_b(mu, 2)) * vals[K * 12 + mu];
      coeffs[(int64_t)l * nt + K] = acc * sc_inv_mass(l);
    }
  return DG_OK;
}

extern "C" int32_t dg_scalar_init(const dg_mesh *mesh, const dg_scalar_config *cfg, const double *coeffs,
                                  void *cuda_stream, dg_scalar **out) {
  if (!out) return set_error(DG_EINVAL, "out is NULL");
  *out = nullptr;
  if (!mesh || !cfg || !coeffs) return set_error(DG_EINVAL, "NULL argument");
  if (cfg->k < 1 || cfg->k > 3 || (cfg->flux != DG_FLUX_LINEAR && cfg->flux != DG_FLUX_BURGERS) ||
      (cfg->rk != 2 && cfg->rk != 3) || (cfg->oe != 0 && cfg->oe != 1) || !(cfg->cfl > 0.0))
    return set_error(DG_EINVAL, "dg_scalar_init: k in 1..3, flux linear or Burgers, rk 2 or 3, oe 0/1, cfl > 0");
  auto s = new (std::nothrow) dg_scalar();
  if (!s) return set_error(DG_ENOMEM, "host allocation failed");
  s->mesh = mesh;
  s->cfg = *cfg;
  s->nb = (cfg->k + 1) * (cfg->k + 2) / 2;
  s->md = mesh_device_view(mesh);
  s->nt = s->md.nt;
  s->ntiles = (int64_t)nblk(s->nt);
  if (!mesh_boundary_tags_ok(mesh, /*scalar=*/1)) {
    delete s;
    return set_error(DG_EINVAL, "dg_scalar_init: boundary edges must be transmissive or constant-state (tags 2..6)");
  }
  s->ph.flux = cfg->flux;
  s->ph.ax = cfg->ax;
  s->ph.ay = cfg->ay;
  for (int i = 0; i < 4; ++i) s->ph.bc[i] = cfg->bc_state[i];
  const int64_t nt = s->nt, nb = s->nb, nq = cfg->k + 1, ng = num_groups(s->ntiles);
  cudaError_t e = cudaSuccess;
  int32_t rc = DG_OK;
#define SCTRY(x)                                                                                           \
  if ((e = (x)) != cudaSuccess) {                                                                          \
    rc = set_error(e == cudaErrorMemoryAllocation ? DG_ENOMEM : DG_ECUDA, cudaGetErrorString(e));          \
    delete s;                                                                                              \
    return rc;                                                                                             \
  }
  if (cuda_stream) {
    s->stream = (cudaStream_t)cuda_stream;
  } else {
    SCTRY(cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking));
    s->own_stream = true;
  }
  SCTRY(cudaMalloc(&s->un, sizeof(double) * nb * nt));
  SCTRY(cudaMalloc(&s->us, sizeof(double) * nb * nt));
  SCTRY(cudaMalloc(&s->uh, sizeof(double) * nb * nt));
  SCTRY(cudaMalloc(&s->tr, sizeof(double) * nt * 3 * nq));
  SCTRY(cudaMalloc(&s->vr, sizeof(double) * nt * 3 * nb));
  SCTRY(cudaMalloc(&s->part, sizeof(double) * 3 * s->ntiles));
  SCTRY(cudaMalloc(&s->fin.grp, sizeof(double) * ng));
  SCTRY(cudaMalloc(&s->fin.tick, sizeof(unsigned) * 3 * (ng + 1)));
  SCTRY(cudaMemsetAsync(s->fin.tick, 0, sizeof(unsigned) * 3 * (ng + 1), s->stream));
  SCTRY(cudaMalloc(&s->sc, sizeof(ScScalars)));
  // time-step geometry factor
  k_sc_dt_base<<<nblk(nt), TPB, 0, s->stream>>>(s->md, cfg->k, s->part);
  std::vector<double> mins(s->ntiles);
  SCTRY(cudaMemcpyAsync(mins.data(), s->part, sizeof(double) * s->ntiles, cudaMemcpyDeviceToHost, s->stream));
  SCTRY(cudaStreamSynchronize(s->stream));
  ScScalars h{};
  h.dt_base = *std::min_element(mins.begin(), mins.end());
  const double *area = nullptr;
  int64_t ntv = 0;
  mesh_view(mesh, &ntv, &area, &h.area_total);
  h.t = 0.0;
  h.t_end = INFINITY;
  h.cfl = cfg->cfl;
  h.active = 1;
  if ((rc = write_sc(s, &h)) != DG_OK) { delete s; return rc; }
  SCTRY(cudaMemcpyAsync(s->uh, coeffs, sizeof(double) * nb * nt, cudaMemcpyHostToDevice, s->stream));
  launch_oe(s, s->uh, s->un, 0, -1);   // traces and alpha of the initial state
  SCTRY(cudaGetLastError());
  // one step as a CUDA graph, with stack room for its kernels
  size_t need = 0;
  SC_DISPATCH(cfg->k, (need = std::max({kernel_local_bytes(k_sc_rk<KK>), kernel_local_bytes(k_sc_stats<KK>),
                                        kernel_local_bytes(k_sc_oe<KK>)})));
  if ((rc = ensure_stack_limit(need)) != DG_OK) { delete s; return rc; }
  cudaGraph_t graph = nullptr;
  SCTRY(cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal));
  enqueue_step(s);
  e = cudaStreamEndCapture(s->stream, &graph);
  if (e == cudaSuccess) e = cudaGraphInstantiate(&s->exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  SCTRY(e);
  SCTRY(cudaStreamSynchronize(s->stream));
  *out = s;
  return DG_OK;
#undef SCTRY
}

extern "C" int32_t dg_scalar_advance(dg_scalar *s, double t_end, int64_t max_steps, dg_stats *stats) {
  if (!s || max_steps < 0) return set_error(DG_EINVAL, "bad argument");
  ScScalars h{};
  int32_t rc;
  if ((rc = read_sc(s, &h)) != DG_OK) return rc;
  h.t_end = t_end;
  h.active = 1;
  if ((rc = write_sc(s, &h)) != DG_OK) return rc;
  const long long start = h.steps;
  int64_t done = 0;
  while (done < max_steps) {
    const int64_t chunk = std::min<int64_t>(32, max_steps - done);
    for (int64_t i = 0; i < chunk; ++i)
      if (cudaGraphLaunch(s->exec, s->stream) != cudaSuccess) return set_error(DG_ECUDA, "scalar step launch");
    done += chunk;
    if ((rc = read_sc(s, &h)) != DG_OK) return rc;
    if (!(h.t < h.t_end)) break;
  }
  if ((rc = read_sc(s, &h)) != DG_OK) return rc;
  if (stats) {
    std::memset(stats, 0, sizeof(*stats));
    stats->steps = h.steps - start;
    stats->t = h.t;
    stats->dt_last = h.dt;
    stats->alpha = h.alpha;
  }
  if (!std::isfinite(h.alpha)) return set_error(DG_ENONPHYS, "scalar solver: the state is no longer finite");
  return DG_OK;
}

extern "C" int32_t dg_scalar_advance_async(dg_scalar *s, int64_t n) {
  if (!s || n < 0) return set_error(DG_EINVAL, "bad argument");
  ScScalars h{};
  int32_t rc;
  if ((rc = read_sc(s, &h)) != DG_OK) return rc;
  h.t_end = INFINITY;
  h.active = 1;
  if ((rc = write_sc(s, &h)) != DG_OK) return rc;
  for (int64_t i = 0; i < n; ++i)
    if (cudaGraphLaunch(s->exec, s->stream) != cudaSuccess) return set_error(DG_ECUDA, "scalar step launch");
  return DG_OK;
}

extern "C" void *dg_scalar_stream(const dg_scalar *s) { return s ? (void *)s->stream : nullptr; }

extern "C" int32_t dg_scalar_get_state(const dg_scalar *s, double *coeffs, size_t len, double *t) {
  if (!s || !coeffs) return set_error(DG_EINVAL, "NULL argument");
  if (len < (size_t)(s->nb * s->nt)) return set_error(DG_EINVAL, "output too small");
  if (cudaMemcpyAsync(coeffs, s->un, sizeof(double) * s->nb * s->nt, cudaMemcpyDeviceToHost, s->stream) != cudaSuccess)
    return set_error(DG_ECUDA, "state download");
  ScScalars h{};
  int32_t rc = read_sc(s, &h);
  if (rc != DG_OK) return rc;
  if (t) *t = h.t;
  return DG_OK;
}

extern "C" int32_t dg_scalar_errors(const dg_scalar *s, const double *exact, double *out3) {
  if (!s || !exact || !out3) return set_error(DG_EINVAL, "NULL argument");
  double *d_exact = nullptr, *d_part = nullptr;
  const int64_t nt = s->nt, nbk = s->ntiles;
  if (cudaMalloc(&d_exact, sizeof(double) * 12 * nt) != cudaSuccess) return set_error(DG_ENOMEM, "errors: exact values");
  if (cudaMalloc(&d_part, sizeof(double) * 3 * nbk) != cudaSuccess) {
    cudaFree(d_exact);
    return set_error(DG_ENOMEM, "errors: partials");
  }
  std::vector<double> part(3 * nbk);
  cudaError_t e = cudaMemcpyAsync(d_exact, exact, sizeof(double) * 12 * nt, cudaMemcpyHostToDevice, s->stream);
  if (e == cudaSuccess) {
    SC_DISPATCH(s->cfg.k, (k_sc_errors<KK><<<nblk(nt), TPB, 0, s->stream>>>(s->md, s->un, d_exact, d_part)));
    e = cudaMemcpyAsync(part.data(), d_part, sizeof(double) * 3 * nbk, cudaMemcpyDeviceToHost, s->stream);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  cudaFree(d_exact);
  cudaFree(d_part);
  if (e != cudaSuccess) return set_error(DG_ECUDA, cudaGetErrorString(e));
  double l1 = 0.0, l2 = 0.0, li = 0.0;
  for (int64_t b = 0; b < nbk; ++b) {
    l1 += part[3 * b];
    l2 += part[3 * b + 1];
    li = std::max(li, part[3 * b + 2]);
  }
  out3[0] = l1;
  out3[1] = std::sqrt(l2);
  out3[2] = li;
  return DG_OK;
}

extern "C" void dg_scalar_destroy(dg_scalar *s) { delete s; }

// dg_stage.cuh -- the per-stage kernels of the SSP-RK3 BP RI-OEDG scheme
// (Ding, Cui & Wu, arXiv 2409.09620, Sec. 4.5), one thread per cell.
//
//   k_rk      volume quadrature + edge LF fluxes + mass inverse + RK combine
//             (eqs. DGSystem:Dis, fluxLF, RKTime); publishes the vertex
//             derivatives of u_h and block sums of |K| u_h^(0)
//   k_stats   sup deviations from the domain mean at the volume points
//             (eqs. normOmg, RIOESys:Coef1)
//   k_oe_bp   RIOE damping (eqs. oe:sys, OEScalar:Coef1/Coef2, oe:sysdelta2,
//             RIOESys:CoefM) + BP limiter (Sec. 4.4) + traces, F.n and the
//             maximum wave speed of the limited state at the edge Gauss points
//             (eq. 1250) for the next stage
#pragma once
#include <type_traits>

#include "dg_common.cuh"

namespace dg {

// Resident blocks per SM requested from the register allocator (FP32 / FP64
// instantiations).  Higher occupancy hides the latency of the neighbour
// gathers and of the FP64 pipe better than the few spilled registers cost.
#ifndef RK_MINB_F
#define RK_MINB_F 4
#endif
#ifndef STATS_MINB_F
#define STATS_MINB_F 6
#endif
#ifndef OEBP_MINB_F
#define OEBP_MINB_F 4
#endif
#ifndef RK_MINB_D
#define RK_MINB_D 3
#endif
#ifndef STATS_MINB_D
#define STATS_MINB_D 3
#endif
#ifndef OEBP_MINB_D
#define OEBP_MINB_D 3
#endif

// A cell's state.  The FP64 form keeps the modes component- and mode-major
// ([4][NB-1][nt]); the mixed form keeps each cell's 4 (NB - 1) FP32 modes
// together (80 bytes for P2, 32 for P1, both multiples of 16), so that a cell
// -- its own or a neighbour's -- comes in (NB - 1) 16-byte loads from one
// address instead of 4 (NB - 1) scattered ones.
template <typename Real, int NB>
__device__ __forceinline__ void load_state(const StateDev<Real> &s, int64_t nt, int64_t K, double avg[4],
                                           Real hi[4][NB]) {
#pragma unroll
  for (int c = 0; c < 4; ++c) avg[c] = s.avg[c * nt + K];
  if constexpr (sizeof(Real) == sizeof(float)) {
    constexpr int NM = 4 * (NB - 1);
    const float4 *p = reinterpret_cast<const float4 *>(s.hi + K * NM);
    float v[NM];
#pragma unroll
    for (int j = 0; j < NM / 4; ++j) {
      const float4 q = p[j];
      v[4 * j] = q.x; v[4 * j + 1] = q.y; v[4 * j + 2] = q.z; v[4 * j + 3] = q.w;
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      hi[c][0] = Real(0);
#pragma unroll
      for (int l = 1; l < NB; ++l) hi[c][l] = v[c * (NB - 1) + l - 1];
    }
  } else {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      hi[c][0] = Real(0);
#pragma unroll
      for (int l = 1; l < NB; ++l) hi[c][l] = s.hi[(c * (NB - 1) + (l - 1)) * nt + K];
    }
  }
}
// store the modes of cell K in the mixed form's per-cell record
template <int NB>
__device__ __forceinline__ void store_modes_mixed(const StateDev<float> &s, int64_t K, const float hi[4][NB]) {
  constexpr int NM = 4 * (NB - 1);
  float4 *p = reinterpret_cast<float4 *>(s.hi + K * NM);
#pragma unroll
  for (int j = 0; j < NM / 4; ++j) {
    float q[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) q[r] = hi[(4 * j + r) / (NB - 1)][(4 * j + r) % (NB - 1) + 1];
    p[j] = make_float4(q[0], q[1], q[2], q[3]);
  }
}

// value of the cell polynomial at a fixed reference point (compile-time after unrolling)
template <typename Real, int NB, typename A>
__device__ __forceinline__ void eval_fixed(const A avg[4], const Real hi[4][NB], double xi, double eta,
                                           Real out[4]) {
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    Real s = Real(avg[c]);
#pragma unroll
    for (int l = 1; l < NB; ++l) s = cfma(psi(l, xi, eta), hi[c][l], s);
    out[c] = s;
  }
}

// The averages in the working precision (plain copies in the FP64 form; the
// mixed form's passes in dg_stage_mixed.cuh convert their own), and an FP64
// average reloaded from memory where a converted copy was let go.
template <typename Real>
__device__ __forceinline__ void to_real(const double a[4], Real r[4]) {
#pragma unroll
  for (int c = 0; c < 4; ++c) r[c] = Real(a[c]);
}
__device__ __forceinline__ double reload_avg(const double *p) { return __ldcg(p); }

// The mixed-precision form has its own tile functions without exchange
// buffers (dg_stage_mixed.cuh); the generic tile functions hand FP32 work to
// them.
template <int K>
__device__ __forceinline__ void rk_tile_mixed(const MeshDev &m, const Phys &ph, StateDev<float> v, StateDev<float> un,
                                              StateDev<float> uh, double *part_sum, const Scalars *sc, double a,
                                              double b, double c_in, int64_t tile);
template <int K>
__device__ __forceinline__ void oe_bp_tile_mixed(const MeshDev &m, const Phys &ph, StateDev<float> uh,
                                                 StateDev<float> out, double *part_alpha, long long *part_cnt,
                                                 const Scalars *sc, int do_oe, int do_bp, double c_out, int end_of_step,
                                                 int64_t tile);

// ==========================================================================
// K1: u_h = a u_n + b (v + dt L(v))
// ==========================================================================
// one tile of TPB cells starting at cell tile * TPB; block partial -> part_sum[4 * tile]
template <int K, typename Real>
__device__ __forceinline__ void rk_tile(const MeshDev &m, const Phys &ph, StateDev<Real> v, StateDev<Real> un,
                                        StateDev<Real> uh, const Real *__restrict__ tr, Real *__restrict__ vdo,
                                        Real *__restrict__ hso, double *part_sum,
                                        const Scalars *sc, double a, double b, double c_in,
                                        int64_t tile) {
  if constexpr (sizeof(Real) == sizeof(float)) {
    rk_tile_mixed<K>(m, ph, v, un, uh, part_sum, sc, a, b, c_in, tile);
    return;
  }
  constexpr int NB = Deg<K>::NB, NQ = Deg<K>::NQ, NV = Deg<K>::NV;
  const int64_t nt = m.nt;
  const int64_t Kc = tile * TPB + threadIdx.x;
  double mass[4] = {0.0, 0.0, 0.0, 0.0};
  if (Kc < nt) {
    const double dt = sc->dt, alpha_d = sc->alpha, t_in = fma(c_in, sc->dt, sc->t);
    const Real alpha = Real(alpha_d), gm1 = phys_gm1<Real>(ph);
    const double area = m.area[Kc];
    const Real *gj = Geo<Real>::jinv(m);
    const Real jx = gj[Kc], jy = gj[nt + Kc], ex = gj[2 * nt + Kc], ey = gj[3 * nt + Kc];
    double v0[4];
    Real cv[4][NB];
    load_state<Real, NB>(v, nt, Kc, v0, cv);
    Real v0r[4];
    to_real(v0, v0r);

    // ---- volume term: |K| sum_mu w_mu F(u(x_mu)) . grad Psi_l ---------------
    Real acc[4][NB];
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
      for (int l = 0; l < NB; ++l) acc[c][l] = Real(0);
#pragma unroll
    for (int mu = 0; mu < NV; ++mu) {
      const double xi = vol_xi(NV, mu), eta = vol_eta(NV, mu), w = vol_w(NV, mu);
      Real u[4], g1[4], g2[4];
      eval_fixed<Real, NB>(v0r, cv, xi, eta, u);
      // F . grad Psi = (F . grad xi) dPsi/dxi + (F . grad eta) dPsi/deta
      flux_dir2(u, jx, jy, ex, ey, gm1, g1, g2);
#pragma unroll
      for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int l = 1; l < NB; ++l) {
          acc[c][l] = cfma(w * psi_x(l, xi, eta), g1[c], acc[c][l]);
          acc[c][l] = cfma(w * psi_y(l, xi, eta), g2[c], acc[c][l]);
        }
    }
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
      for (int l = 1; l < NB; ++l) acc[c][l] *= Real(area);

    // ---- edge term: - sum_i l_i sum_nu w_nu Fhat Psi_l -------------------------
    double acc0[4] = {0.0, 0.0, 0.0, 0.0};
    Real tv0[NQ][4];   // mixed form: per-point mode-0 contributions of one edge
    float s_hi[4] = {0.0f, 0.0f, 0.0f, 0.0f}, s_lo[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const int32_t cn = m.conn[i * nt + Kc];
      const Real nx = Geo<Real>::nrm(m)[(2 * i) * nt + Kc], ny = Geo<Real>::nrm(m)[(2 * i + 1) * nt + Kc];
      const Real li = Geo<Real>::len(m)[i * nt + Kc];
#pragma unroll
      for (int nu = 0; nu < NQ; ++nu) {
        constexpr int TS = TraceStride<Real>::value;
        Real ow[TS], um[4], fm[4], up[4], fp[4];
        vload<TS>(tr + ((Kc * 3 + i) * NQ + nu) * TS, ow);
#pragma unroll
        for (int q = 0; q < 4; ++q) um[q] = ow[q];
        if constexpr (TS == 8) {
#pragma unroll
          for (int q = 0; q < 4; ++q) fm[q] = ow[4 + q];
        } else {
          flux_dir(um, nx, ny, gm1, fm);
        }
        if (cn >= 0) {
          const int64_t nb = cn >> 2;
          const int j = cn & 3;
          Real ot[TS];
          vload<TS>(tr + ((nb * 3 + j) * NQ + (NQ - 1 - nu)) * TS, ot);
#pragma unroll
          for (int q = 0; q < 4; ++q) up[q] = ot[q];
          if constexpr (TS == 8) {
#pragma unroll
            for (int q = 0; q < 4; ++q) fp[q] = -ot[4 + q];
          } else {
            flux_dir(up, nx, ny, gm1, fp);   // = -F(u+).n of the neighbour, n+ = -n exactly
          }
        } else {
          double px = 0.0, py = 0.0;
          if (cn == -7) {
            const double s = gauss_s(NQ, nu);
            const double xa = m.vxy[(2 * ((i + 1) % 3)) * nt + Kc], ya = m.vxy[(2 * ((i + 1) % 3) + 1) * nt + Kc];
            const double xb = m.vxy[(2 * ((i + 2) % 3)) * nt + Kc], yb = m.vxy[(2 * ((i + 2) % 3) + 1) * nt + Kc];
            px = fma(xb - xa, s, xa);
            py = fma(yb - ya, s, ya);
          }
          ghost_state(-cn, um, v0r, nx, ny, px, py, t_in, ph, up);
          flux_dir(up, nx, ny, gm1, fp);
        }
        // l_i w_nu / 2: the 1/2 of the LF flux rides on the weight (a power of
        // two, so the products are bitwise those of scaling the flux)
        const Real lw = li * Real(0.5 * gauss_w(NQ, nu));
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const Real fh = fma(-alpha, up[c] - um[c], fm[c] + fp[c]);
          const Real tv = lw * fh;
          if constexpr (sizeof(Real) == sizeof(double)) {
            acc0[c] -= double(tv);
          } else {
            tv0[nu][c] = tv;
          }
#pragma unroll
          for (int l = 1; l < NB; ++l)
            acc[c][l] = cfma(-psi(l, edge_xi(i, gauss_s(NQ, nu)), edge_eta(i, gauss_s(NQ, nu))), tv, acc[c][l]);
        }
      }
      if constexpr (sizeof(Real) != sizeof(double)) {
        // FP32 edge contributions summed in an order that is symmetric under
        // the neighbour's reversed point order, so the neighbour's sum is the
        // exact negation.  The three edge sums are added as an unevaluated
        // FP32 pair (Knuth's TwoSum: hi + lo holds each partial sum exactly,
        // the last lo addition rounds at 2^-48 of the sum) on the FP32 pipe,
        // and the FP64 average takes hi + lo once.
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const float se = NQ == 3 ? (tv0[0][c] + tv0[2][c]) + tv0[1][c] : tv0[0][c] + tv0[NQ - 1][c];
          const float x = -se, sum = s_hi[c] + x, bv = sum - s_hi[c];
          const float err = (s_hi[c] - (sum - bv)) + (x - bv);
          s_hi[c] = sum;
          s_lo[c] += err;
        }
      }
    }
    if constexpr (sizeof(Real) != sizeof(double)) {
#pragma unroll
      for (int c = 0; c < 4; ++c) acc0[c] = double(s_hi[c]) + double(s_lo[c]);
    }

    // ---- mass inverse and SSP-RK combination -----------------------------------
    const double dta = dt * m.iarea[Kc];
    double h0[4];
    Real hh[4][NB];
    Real h0r[4];
    // a u_n + b (v + dt L(v)); the first stage (a = 0, b = 1, v = u_n) skips
    // the zero term and the load of u_n (equal up to the sign of a zero)
    auto combine = [&](auto first_stage) {
      constexpr bool FIRST = decltype(first_stage)::value;
      double un0[4] = {0.0, 0.0, 0.0, 0.0};
      Real cu[4][NB];
      if constexpr (!FIRST) load_state<Real, NB>(un, nt, Kc, un0, cu);
      // the stage coefficients in the working precision, converted once
      const Real ar = Real(a), br = Real(b), dtar = Real(dta);
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const double v0c = sizeof(Real) == sizeof(double) ? v0[c] : reload_avg(v.avg + c * nt + Kc);
        if constexpr (FIRST) h0[c] = fma(dta, acc0[c], v0c);
        else h0[c] = fdot2(a, un0[c], b, fma(dta, acc0[c], v0c));
        uh.avg[c * nt + Kc] = h0[c];
        mass[c] = area * h0[c];
        h0r[c] = Real(h0[c]);
        hh[c][0] = Real(0);
#pragma unroll
        for (int l = 1; l < NB; ++l) {
          const Real s = sizeof(Real) == sizeof(double) ? Real(dta * inv_mass_c(l)) : dtar * Real(inv_mass_c(l));
          if constexpr (FIRST) hh[c][l] = fma(s, acc[c][l], cv[c][l]);
          else hh[c][l] = fdot2(ar, cu[c][l], br, fma(s, acc[c][l], cv[c][l]));
          uh.hi[(c * (NB - 1) + (l - 1)) * nt + Kc] = hh[c][l];
        }
      }
    };
    if (a == 0.0 && b == 1.0) combine(std::true_type{});
    else combine(std::false_type{});

    // ---- vertex derivatives of u_h for the OE jumps ------------------------------
    // u_h is a polynomial of degree K in the reference coordinates, so with
    // its value u0, reference gradient (gx0, ge0) at vertex 0 = (0, 0) and its
    // (constant) reference Hessian (hxx, hxe, hee):
    //   vertex 1 = (1, 0): u0 + gx0 + hxx / 2, gradient (gx0 + hxx, ge0 + hxe)
    //   vertex 2 = (0, 1): u0 + ge0 + hee / 2, gradient (gx0 + hxe, ge0 + hee)
    Real u0[4], gx0[4], ge0[4], hxx[4], hxe[4], hee[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      u0[c] = h0r[c];
      gx0[c] = Real(0);
      ge0[c] = Real(0);
      hxx[c] = Real(0);
      hxe[c] = Real(0);
      hee[c] = Real(0);
#pragma unroll
      for (int l = 1; l < NB; ++l) {
        u0[c] = cfma(psi(l, 0.0, 0.0), hh[c][l], u0[c]);
        gx0[c] = cfma(psi_x(l, 0.0, 0.0), hh[c][l], gx0[c]);
        ge0[c] = cfma(psi_y(l, 0.0, 0.0), hh[c][l], ge0[c]);
      }
#pragma unroll
      for (int l = 3; l < NB; ++l) {
        hxx[c] = cfma(psi_2(l, 0), hh[c][l], hxx[c]);
        hxe[c] = cfma(psi_2(l, 1), hh[c][l], hxe[c]);
        hee[c] = cfma(psi_2(l, 2), hh[c][l], hee[c]);
      }
    }
    Real *vo = vdo + Kc * VD_CELL;
    const Real gamma = phys_gamma<Real>(ph);
#pragma unroll
    for (int vv = 0; vv < 3; ++vv) {
      Real rec[VD_STRIDE];
      Real val4[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        Real val, gx, ge;
        if (vv == 0) {
          val = u0[c]; gx = gx0[c]; ge = ge0[c];
        } else if (vv == 1) {
          val = fma(Real(0.5), hxx[c], u0[c] + gx0[c]); gx = gx0[c] + hxx[c]; ge = ge0[c] + hxe[c];
        } else {
          val = fma(Real(0.5), hee[c], u0[c] + ge0[c]); gx = gx0[c] + hxe[c]; ge = ge0[c] + hee[c];
        }
        val4[c] = val;
        rec[c] = val;
        rec[4 + 2 * c] = fdot2(gx, jx, ge, ex);
        rec[5 + 2 * c] = fdot2(gx, jy, ge, ey);
      }
      // 1/rho and sound speed at the vertex, for the wave speeds beta of the OE (+inf for rho <= 0)
      Real ri = Real(0), cs = Real(INFINITY);
      if (gt0(val4[0])) {
        ri = Real(1) / val4[0];
        Real p = gm1 * fma(Real(-0.5) * fdot2(val4[1], val4[1], val4[2], val4[2]), ri, val4[3]);
        p = gt0(p) ? p : Real(0);
        cs = sqrt(gamma * p * ri);
      }
      rec[12] = ri;
      rec[13] = cs;
      rec[14] = Real(0);
      rec[15] = Real(0);
      vstore<VD_STRIDE>(vo + vv * VD_STRIDE, rec);
    }
    if (K == 2) {
      Real ho[12];
      // physical second derivatives from the reference ones: the factors of
      // J^-T H J^-1, shared by the four components
      const Real gxx0 = jx * jx, gxe0 = Real(2) * jx * ex, gee0 = ex * ex;
      const Real gxx1 = jx * jy, gxe1 = fdot2(jx, ey, jy, ex), gee1 = ex * ey;
      const Real gxx2 = jy * jy, gxe2 = Real(2) * jy * ey, gee2 = ey * ey;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        ho[3 * c + 0] = fma(hxx[c], gxx0, fdot2(hxe[c], gxe0, hee[c], gee0));
        ho[3 * c + 1] = fma(hxx[c], gxx1, fdot2(hxe[c], gxe1, hee[c], gee1));
        ho[3 * c + 2] = fma(hxx[c], gxx2, fdot2(hxe[c], gxe2, hee[c], gee2));
      }
      vstore<12>(hso + Kc * 12, ho);   // 16-byte vector stores
    }
  }
  block_reduce<4>(mass, part_sum + 4 * tile, OpSum());
}

template <int K, typename Real>
__global__ void __launch_bounds__(TPB, sizeof(Real) == 4 ? RK_MINB_F : RK_MINB_D)
    k_rk(MeshDev m, Phys ph, StateDev<Real> v, StateDev<Real> un, StateDev<Real> uh, const Real *__restrict__ tr,
         Real *__restrict__ vdo, Real *__restrict__ hso, double *part_sum, const Scalars *sc, double a, double b,
         double c_in) {
  if (!sc->active) return;
  rk_tile<K, Real>(m, ph, v, un, uh, tr, vdo, hso, part_sum, sc, a, b, c_in, blockIdx.x);
}

// ==========================================================================
// K2: sup deviations from the domain mean at the volume points
// ==========================================================================
template <int K, typename Real>
__device__ __forceinline__ void stats_tile(const MeshDev &m, StateDev<Real> uh, double *part_dev,
                                           const Scalars *sc, int64_t tile) {
  constexpr int NB = Deg<K>::NB, NV = Deg<K>::NV;
  const int64_t nt = m.nt;
  const int64_t Kc = tile * TPB + threadIdx.x;
  // deviations in the working precision, reduced in it; one conversion per block
  Real dr[5] = {Real(0), Real(0), Real(0), Real(0), Real(0)};
  if (Kc < nt) {
    double a0[4];
    Real hi[4][NB];
    load_state<Real, NB>(uh, nt, Kc, a0, hi);
    double off[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) off[c] = a0[c] - sc->mean[c];   // deviation of the cell mean
#pragma unroll
    for (int mu = 0; mu < NV; ++mu) {
      Real u[4];
      eval_fixed<Real, NB>(off, hi, vol_xi(NV, mu), vol_eta(NV, mu), u);
      dr[0] = max_nn(dr[0], fabs(u[0]));
      dr[1] = max_nn(dr[1], fdot2(u[1], u[1], u[2], u[2]));   // squared: one square root per cell below
      dr[2] = max_nn(dr[2], fabs(u[3]));
      dr[3] = max_nn(dr[3], fabs(u[1]));
      dr[4] = max_nn(dr[4], fabs(u[2]));
    }
    // sqrt is monotonic and correctly rounded: sqrt(max) = max(sqrt), bit for bit
    dr[1] = sqrt(dr[1]);
  }
  block_reduce<5>(dr, part_dev + 5 * tile, OpMaxNN());
}



// ==========================================================================
// K3: RIOE + BP limiter + traces / alpha of the limited state
// ==========================================================================
// exterior vertex data of a boundary edge: value, gradient (x, y) and Hessian (xx, xy, yy)
template <typename Real>
__device__ __forceinline__ void ghost_vertex(int tag, const Real val[4], const Real grd[8], const Real hes[12],
                                             const Real avg[4], Real nx, Real ny, double px, double py, double t,
                                             const Phys &ph, Real ov[4], Real og[8], Real oh[12]) {
  if (tag == 1) {
    // mirror polynomial: q(Rx) for rho, E and R m(Rx) for the momentum, R = I - 2 n n^T
    // with the fused products fixed (left to the compiler, the fusion could
    // differ between the kernels that inline this, and a batch would not
    // reproduce its solves bit for bit)
    const Real R00 = fma(Real(-2) * nx, nx, Real(1)), R01 = Real(-2) * nx * ny, R11 = fma(Real(-2) * ny, ny, Real(1));
    Real RHR[4][3];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const Real hxx = hes[3 * c], hxy = hes[3 * c + 1], hyy = hes[3 * c + 2];
      // (R H R)_ab with R symmetric
      const Real a0 = fdot2(R00, hxx, R01, hxy), a1 = fdot2(R00, hxy, R01, hyy);   // row 0 of R H
      const Real b0 = fdot2(R01, hxx, R11, hxy), b1 = fdot2(R01, hxy, R11, hyy);   // row 1 of R H
      RHR[c][0] = fdot2(a0, R00, a1, R01);
      RHR[c][1] = fdot2(a0, R01, a1, R11);
      RHR[c][2] = fdot2(b0, R01, b1, R11);
    }
#pragma unroll
    for (int c = 0; c < 4; c += 3) {
      ov[c] = val[c];
      og[2 * c] = fdot2(R00, grd[2 * c], R01, grd[2 * c + 1]);
      og[2 * c + 1] = fdot2(R01, grd[2 * c], R11, grd[2 * c + 1]);
      oh[3 * c] = RHR[c][0]; oh[3 * c + 1] = RHR[c][1]; oh[3 * c + 2] = RHR[c][2];
    }
    ov[1] = fdot2(R00, val[1], R01, val[2]);
    ov[2] = fdot2(R01, val[1], R11, val[2]);
    // gradient matrix G[a][b] = d m_a / d x_b -> R G R
    const Real G00 = grd[2], G01 = grd[3], G10 = grd[4], G11 = grd[5];
    const Real A00 = fdot2(R00, G00, R01, G10), A01 = fdot2(R00, G01, R01, G11);
    const Real A10 = fdot2(R01, G00, R11, G10), A11 = fdot2(R01, G01, R11, G11);
    og[2] = fdot2(A00, R00, A01, R01); og[3] = fdot2(A00, R01, A01, R11);
    og[4] = fdot2(A10, R00, A11, R01); og[5] = fdot2(A10, R01, A11, R11);
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      oh[3 + r] = fdot2(R00, RHR[1][r], R01, RHR[2][r]);
      oh[6 + r] = fdot2(R01, RHR[1][r], R11, RHR[2][r]);
    }
  } else {   // constant exterior states (Dirichlet, moving shock, the transmissive cell average): no derivatives
    Real st[4];
    ghost_state(tag, val, avg, nx, ny, px, py, t, ph, st);
#pragma unroll
    for (int c = 0; c < 4; ++c) ov[c] = st[c];
#pragma unroll
    for (int q = 0; q < 8; ++q) og[q] = Real(0);
#pragma unroll
    for (int q = 0; q < 12; ++q) oh[q] = Real(0);
  }
}

// --------------------------------------------------------------------------
// OE jump data of one edge, computed once for both cells that share it: beta
// (max spectral radius of both sides at both endpoints) and sqrt(2 J) for the
// trapezoidal sums J = 1/2 sum_{|alpha| = j} C_j^alpha1 [d^alpha q]^2 over
// the two endpoints (eqs. OEScalar:Coef2 with the trapezoidal rule,
// RIOESys:Coef1/Coef2), seen from the owning cell.  Jump sums are even in the
// sign of the jump and of the normal, so both cells share them.
// Edges [etile[tile], etile[tile + 1]) are processed in chunks of TPB.
// --------------------------------------------------------------------------
template <int K, typename Real>
__device__ __forceinline__ void edge_tile(const MeshDev &m, const Phys &ph, const double *__restrict__ avg,
                                          const Real *__restrict__ vdi, const Real *__restrict__ hsi,
                                          Real *__restrict__ ej, const Scalars *sc, double c_out, int64_t tile) {
  if constexpr (sizeof(Real) == sizeof(float)) return;   // the mixed form forms its jumps in K3
  const int64_t nt = m.nt;
  const int64_t e0 = m.etile[tile], e1 = m.etile[tile + 1];
  const double t_out = fma(c_out, sc->dt, sc->t);
  const Real gamma = phys_gamma<Real>(ph);
  const int cw = ph.oe == 2;
  for (int64_t e = e0 + threadIdx.x; e < e1; e += TPB) {
    const int64_t Kc = m.e_cell[e];
    const int i = m.e_loc[e];
    const int32_t cn = m.conn[i * nt + Kc];
    const Real nx = Geo<Real>::nrm(m)[(2 * i) * nt + Kc], ny = Geo<Real>::nrm(m)[(2 * i + 1) * nt + Kc];
    const Real *vme = vdi + Kc * VD_CELL;
    Real hme[12], hot[12];
#pragma unroll
    for (int q = 0; q < 12; ++q) hme[q] = Real(0);
    if (K == 2) vload<12>(hsi + Kc * 12, hme);
    const Real *vnb = nullptr;
    int jn = 0;
    if (cn >= 0) {
      vnb = vdi + (int64_t)(cn >> 2) * VD_CELL;
      jn = cn & 3;
#pragma unroll
      for (int q = 0; q < 12; ++q) hot[q] = Real(0);
      if (K == 2) vload<12>(hsi + (int64_t)(cn >> 2) * 12, hot);
    }
    Real Jq[4][K + 1];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int j = 0; j <= K; ++j) Jq[q][j] = Real(0);
    Real beta = Real(0);
#pragma unroll
    for (int ev = 0; ev < 2; ++ev) {
      const int ov = (i + 1 + ev) % 3;                 // v_c then v_d
      Real rec[VD_STRIDE], val[4], grd[8], xv[4], xg[8], xh[12];
      vload<VD_STRIDE>(vme + ov * VD_STRIDE, rec);
#pragma unroll
      for (int c = 0; c < 4; ++c) val[c] = rec[c];
#pragma unroll
      for (int q = 0; q < 8; ++q) grd[q] = rec[4 + q];
      const Real r_own = fma(fabs(fdot2(val[1], nx, val[2], ny)), rec[12], rec[13]);
      Real r_oth;
      if (cn >= 0) {
        const int xvtx = (jn + 2 - ev) % 3;            // the neighbour's copy of this vertex
        Real xr[VD_STRIDE];
        vload<VD_STRIDE>(vnb + xvtx * VD_STRIDE, xr);
#pragma unroll
        for (int c = 0; c < 4; ++c) xv[c] = xr[c];
#pragma unroll
        for (int q = 0; q < 8; ++q) xg[q] = xr[4 + q];
#pragma unroll
        for (int q = 0; q < 12; ++q) xh[q] = hot[q];
        r_oth = fma(fabs(fdot2(xv[1], nx, xv[2], ny)), xr[12], xr[13]);
      } else {
        double px = 0.0, py = 0.0;
        if (cn == -7) { px = m.vxy[(2 * ov) * nt + Kc]; py = m.vxy[(2 * ov + 1) * nt + Kc]; }
        Real ab[4];   // the cell average (the exterior state of a transmissive edge)
#pragma unroll
        for (int c = 0; c < 4; ++c) ab[c] = Real(avg[c * nt + Kc]);
        ghost_vertex(-cn, val, grd, hme, ab, nx, ny, px, py, t_out, ph, xv, xg, xh);
        // a mirror state has the same spectral radius
        r_oth = cn == -1 ? r_own : wave_speed(xv, nx, ny, gamma);
      }
      beta = max_nn(beta, max_nn(r_own, r_oth));
      // the Hessians of P2 polynomials (and of every ghost) are constant, so
      // the Hessian jump is the same at both endpoints: taken at v_c only
      const bool hess = K == 2 && ev == 0;
      Real jv[4], jg[4][2], jh[4][3];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        jv[c] = val[c] - xv[c];
        jg[c][0] = grd[2 * c] - xg[2 * c];
        jg[c][1] = grd[2 * c + 1] - xg[2 * c + 1];
#pragma unroll
        for (int r = 0; r < 3; ++r) jh[c][r] = hess ? hme[3 * c + r] - xh[3 * c + r] : Real(0);
      }
      if (!cw) {   // rotate the momentum jumps to (m_n, m_t) with the owner's normal
        Real t0 = jv[1], t1 = jv[2];
        jv[1] = fdot2(t0, nx, t1, ny); jv[2] = fdot2(t1, nx, -t0, ny);
#pragma unroll
        for (int d = 0; d < 2; ++d) {
          t0 = jg[1][d]; t1 = jg[2][d];
          jg[1][d] = fdot2(t0, nx, t1, ny); jg[2][d] = fdot2(t1, nx, -t0, ny);
        }
        if (hess) {
#pragma unroll
          for (int r = 0; r < 3; ++r) {
            t0 = jh[1][r]; t1 = jh[2][r];
            jh[1][r] = fdot2(t0, nx, t1, ny); jh[2][r] = fdot2(t1, nx, -t0, ny);
          }
        }
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        // 2 J: the 1/2 of the trapezoidal rule moves into A (sqrt(1/2))
        Jq[q][0] = fma(jv[q], jv[q], Jq[q][0]);
        Jq[q][1] = fma(jg[q][0], jg[q][0], fma(jg[q][1], jg[q][1], Jq[q][1]));
        if (hess) {   // both endpoints: twice the one value
          const Real f = fma(jh[q][0], jh[q][0], fma(jh[q][1] + jh[q][1], jh[q][1], jh[q][2] * jh[q][2]));
          Jq[q][K] = f + f;
        }
      }
    }
    Real er[EJ_STRIDE];
#pragma unroll
    for (int r = 0; r < EJ_STRIDE; ++r) er[r] = Real(0);
    er[0] = beta;
#pragma unroll
    for (int j = 0; j <= K; ++j) {
      er[ej_row(0, j, K)] = sqrt(Jq[0][j]);
      er[ej_row(3, j, K)] = sqrt(Jq[3][j]);
      if (cw) {
        er[ej_row(1, j, K)] = sqrt(Jq[1][j]);
        er[ej_row(2, j, K)] = sqrt(Jq[2][j]);
      } else {   // RIOE: delta_m = max(delta_mn, delta_mt) -> sqrt(max(J_mn, J_mt))
        er[ej_row(1, j, K)] = sqrt(max_nn(Jq[1][j], Jq[2][j]));
      }
    }
    vstore<EJ_STRIDE>(ej + e * EJ_STRIDE, er);
  }
}

template <int K, typename Real>
__device__ __forceinline__ void oe_bp_tile(const MeshDev &m, const Phys &ph, StateDev<Real> uh, StateDev<Real> out,
                                           const Real *__restrict__ ej,
                                           Real *__restrict__ tr, double *part_alpha,
                                           long long *part_cnt, const Scalars *sc,
                                           int do_oe, int do_bp, double c_out, int end_of_step, int64_t tile) {
  if constexpr (sizeof(Real) == sizeof(float)) {
    oe_bp_tile_mixed<K>(m, ph, uh, out, part_alpha, part_cnt, sc, do_oe, do_bp, c_out, end_of_step, tile);
    return;
  }
  constexpr int NB = Deg<K>::NB, NQ = Deg<K>::NQ;
  constexpr int NE = 3 * NQ;          // edge Gauss points
  const int64_t nt = m.nt;
  const int64_t Kc = tile * TPB + threadIdx.x;
  double amax = 0.0;
  long long cnt[2] = {0, 0};
  if (Kc < nt) {
    // exterior states for the next stage's alpha at the time of the stage
    // result: t + c_out dt, and after the last stage of a step clamped to
    // the end time, the end time itself (the next step starts there)
    const double dt = sc->dt, t_out = end_of_step && sc->pad ? sc->t_end : fma(c_out, sc->dt, sc->t);
    const Real gamma = phys_gamma<Real>(ph);
    double a0[4];
    Real hi[4][NB];
    load_state<Real, NB>(uh, nt, Kc, a0, hi);
    Real nxs[3], nys[3];
    int32_t cns[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      nxs[i] = Geo<Real>::nrm(m)[(2 * i) * nt + Kc];
      nys[i] = Geo<Real>::nrm(m)[(2 * i + 1) * nt + Kc];
      cns[i] = m.conn[i * nt + Kc];
    }

    // ---------------------------- RIOE ---------------------------------------
    if (do_oe) {
      const int cw = ph.oe == 2;
      // 1 / normaliser of rho, (m_n | m1), (m_t | m2), E; 0 for a constant component
      Real iD[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if constexpr (sizeof(Real) == sizeof(float)) iD[q] = sc->invDf[q]; else iD[q] = sc->invD[q];
      }
      // sigma_q^j = sum_i (beta_i / h_i) delta_{i,q}^j with delta = A^{k,j} h^j
      // sqrt(J) / D_q, A^{k,j} = (2j + 1) / ((2k - 1) j!).  The edge records hold
      // sqrt(2 J), so A carries a factor sqrt(1/2); the edge sum is taken
      // first and scaled by 1 / D_q once (a constant component, 1 / D_q = 0,
      // gets sigma = 0).  RIOE: m2 shares the momentum sums of m1.
      Real sig[4][K + 1];
#pragma unroll
      for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int j = 0; j <= K; ++j) sig[c][j] = Real(0);
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        // beta and sqrt(2 J) of this edge (edge_tile, shared by both cells)
        const int64_t eid = m.cedge[i * nt + Kc];
        const Real h = Geo<Real>::hgeo(m)[i * nt + Kc], ih = Geo<Real>::hgeo(m)[(3 + i) * nt + Kc];
        Real er[EJ_STRIDE];
        vload<EJ_STRIDE>(ej + eid * EJ_STRIDE, er);
        const Real bh = er[0] * ih;
        // a zero jump adds nothing; it is skipped only when beta / h is not
        // finite (beta = +inf at a vertex with rho <= 0), where 0 * inf would be NaN
        const bool bh_finite = is_finite_bits(bh);
        Real hj = Real(1);
#pragma unroll
        for (int j = 0; j <= K; ++j) {
          const Real F = bh * (Real((2.0 * j + 1.0) / ((2.0 * K - 1.0) * (j == 2 ? 2.0 : 1.0)) *
                                    0.70710678118654752440) * hj);
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            if (c == 2 && !cw) continue;
            const Real e = er[ej_row(c, j, K)];
            if (bh_finite || nonzero_bits(e)) sig[c][j] = fma(F, e, sig[c][j]);
          }
          hj *= h;
        }
      }
#pragma unroll
      for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int j = 0; j <= K; ++j) sig[c][j] = nonzero_bits(iD[c]) ? iD[c] * sig[c][j] : Real(0);
      // exact solution of the damping ODE: mode of degree m times exp(-dt sum_{j<=m} sigma^j)
      Real fac[4][K + 1];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        if (c == 2 && !cw) {   // RIOE: m2 shares the momentum coefficient of m1
#pragma unroll
          for (int md = 1; md <= K; ++md) fac[2][md] = fac[1][md];
          continue;
        }
        Real sacc = sig[c][0];
#pragma unroll
        for (int md = 1; md <= K; ++md) {
          sacc += sig[c][md];
          fac[c][md] = exp_neg(Real(dt) * sacc);
        }
      }
#pragma unroll
      for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int l = 1; l < NB; ++l) hi[c][l] *= fac[c][degree_of(l)];
    }

    if constexpr (sizeof(Real) == sizeof(double)) {
      // ---------------------------- BP limiter ----------------------------------
      // deviations u(x_p) - ubar at the edge Gauss points and the two extra points
      double dev[NE + 2][4];
  #pragma unroll
      for (int i = 0; i < 3; ++i)
  #pragma unroll
        for (int nu = 0; nu < NQ; ++nu) {
          const double xi = edge_xi(i, gauss_s(NQ, nu)), eta = edge_eta(i, gauss_s(NQ, nu));
  #pragma unroll
          for (int c = 0; c < 4; ++c) {
            double s = 0.0;
  #pragma unroll
            for (int l = 1; l < NB; ++l) s = cfma(psi(l, xi, eta), double(hi[c][l]), s);
            dev[i * NQ + nu][c] = s;
          }
        }
      double th_r = 1.0, th_a = 1.0;
      // A bound over the whole cell settles the usual (smooth) cell without
      // its limiter points: with |Psi_l| <= 4 on K, every point's density is
      // at least rho_bar - 4 sum |rho_l|, its energy at least E_bar -
      // 4 sum |E_l| and the L1 norm of its momentum at most |m1_bar| +
      // |m2_bar| + 4 sum (|m1_l| + |m2_l|).  If these keep rho and the
      // internal energy above the thresholds with a margin far above the
      // rounding of the point evaluations, every point passes the paper's
      // tests and theta = 1, as the points themselves would give.
      const double Ebar = int_energy(a0);
      bool settled = false;
      if (do_bp && a0[0] > 0.0 && Ebar > 0.0) {
        double D[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          double s = 0.0;
#pragma unroll
          for (int l = 1; l < NB; ++l) s += fabs(double(hi[c][l]));
          D[c] = 4.0 * s;
        }
        const double eps1 = fmin(a0[0], 1e-13), eps2 = fmin(Ebar, 1e-13);
        const double r_lo = a0[0] - D[0];
        if (r_lo >= fma(1e-12, a0[0] + D[0], eps1)) {
          const double M_hi = (fabs(a0[1]) + fabs(a0[2])) + (D[1] + D[2]);
          const double E_lo = a0[3] - D[3], E_hi = fabs(a0[3]) + D[3];
          // E_lo - M_hi^2 / (2 r_lo) >= eps2 + 1e-12 (E_hi + M_hi^2 / r_lo), times r_lo > 0
          const double M2 = M_hi * M_hi;
          settled = r_lo * (E_lo - eps2) - 1e-12 * fma(E_hi, r_lo, M2) >= 0.5 * M2;
        }
      }
      if (do_bp && !settled) {
        if (ph.decomp) {
          zxs_extra_points<K, double, NE + 2>(dev);
        } else {
          // P1: the vertices v1, v2; P2: the internal nodes, whose basis
          // values the mesh holds
          double psx[2][NB];
          if (K == 1) {
#pragma unroll
            for (int p = 0; p < 2; ++p) {
              const int vp = m.limv[p * nt + Kc];
#pragma unroll
              for (int l = 1; l < NB; ++l) psx[p][l] = psi(l, vert_xi(vp), vert_eta(vp));
            }
          } else {
#pragma unroll
            for (int p = 0; p < 2; ++p)
#pragma unroll
              for (int l = 1; l < NB; ++l) psx[p][l] = m.psi_node[(5 * p + l - 1) * nt + Kc];
          }
  #pragma unroll
          for (int p = 0; p < 2; ++p)
  #pragma unroll
            for (int c = 0; c < 4; ++c) {
              double s = 0.0;
  #pragma unroll
              for (int l = 1; l < NB; ++l) s = fma(psx[p][l], double(hi[c][l]), s);
              dev[NE + p][c] = s;
            }
        }
        if (!(a0[0] > 0.0) || !(Ebar > 0.0)) {
          cnt[1] = 1;
        } else {
          // Step 1: density
          // minimum on the integer units through order-preserving keys
          long long kmin = ord_key(a0[0] + dev[0][0]);
  #pragma unroll
          for (int p = 1; p < NE + 2; ++p) kmin = min(kmin, ord_key(a0[0] + dev[p][0]));
          const double rmin = ord_val(kmin);
          const double eps1 = fmin(a0[0], 1e-13);
          double th1 = 1.0;
          if (rmin < eps1) th1 = (a0[0] - eps1) / (a0[0] - rmin);
          // Step 2: internal energy of the density-limited polynomial
          // E - |m|^2 / (2 rho) < eps2 is tested as rho E - |m|^2 / 2 < eps2 rho (rho > 0):
          // the division is only needed at points that violate the bound
          const double eps2 = fmin(Ebar, 1e-13);
          double emin = INFINITY;
  #pragma unroll
          for (int p = 0; p < NE + 2; ++p) {
            const double w0 = fma(th1, dev[p][0], a0[0]), w1 = a0[1] + dev[p][1], w2 = a0[2] + dev[p][2],
                         w3 = a0[3] + dev[p][3];
            const double q = 0.5 * fdot2(w1, w1, w2, w2);
            if (!(w0 > 0.0) || fma(w3, w0, -q) < eps2 * w0) emin = fmin(emin, w3 - q / w0);
          }
          double th2 = 1.0;
          if (emin < eps2) th2 = (Ebar - eps2) / (Ebar - emin);
          th_r = th1 * th2;
          th_a = th2;
          if (th1 < 1.0 || th2 < 1.0) cnt[0] = 1;
        }
      }
      // ---------------------------- output ----------------------------------------
  #pragma unroll
      for (int c = 0; c < 4; ++c) out.avg[c * nt + Kc] = a0[c];
      if (th_r < 1.0 || th_a < 1.0) {   // rare: the cell is limited
        // store the scaled modes, and take the traces below from the stored
        // modes, so that a run resumed from the stored state (dg_set_state)
        // sees the same traces bit for bit
  #pragma unroll
        for (int c = 0; c < 4; ++c) {
          const double th = c == 0 ? th_r : th_a;
  #pragma unroll
          for (int l = 1; l < NB; ++l) {
            hi[c][l] = th < 1.0 ? Real(th * double(hi[c][l])) : hi[c][l];
            out.hi[(c * (NB - 1) + (l - 1)) * nt + Kc] = hi[c][l];
          }
        }
  #pragma unroll
        for (int i = 0; i < 3; ++i)
  #pragma unroll
          for (int nu = 0; nu < NQ; ++nu) {
            const double xi = edge_xi(i, gauss_s(NQ, nu)), eta = edge_eta(i, gauss_s(NQ, nu));
  #pragma unroll
            for (int c = 0; c < 4; ++c) {
              double s = 0.0;
  #pragma unroll
              for (int l = 1; l < NB; ++l) s = cfma(psi(l, xi, eta), double(hi[c][l]), s);
              dev[i * NQ + nu][c] = s;
            }
          }
        th_r = th_a = 1.0;
      } else {
  #pragma unroll
        for (int c = 0; c < 4; ++c)
  #pragma unroll
          for (int l = 1; l < NB; ++l) out.hi[(c * (NB - 1) + (l - 1)) * nt + Kc] = hi[c][l];
      }
      // traces, F.n and wave speed of the limited state at the edge Gauss points,
      // with the reciprocal densities of all points from one division
      const Real gm1 = phys_gm1<Real>(ph);
      double rho_t[NE], ri_t[NE];
  #pragma unroll
      for (int p = 0; p < NE; ++p) rho_t[p] = a0[0] + dev[p][0];   // theta is folded into dev above
      batch_reciprocal<NE>(rho_t, ri_t);
  #pragma unroll
      for (int i = 0; i < 3; ++i) {
  #pragma unroll
        for (int nu = 0; nu < NQ; ++nu) {
          Real u[4], f[4];
  #pragma unroll
          for (int c = 0; c < 4; ++c) u[c] = Real(a0[c] + dev[i * NQ + nu][c]);
          amax = max_nn(amax, double(flux_speed_ri(u, ri_t[i * NQ + nu], nxs[i], nys[i], gm1, gamma, f)));
          Real o8[8];
  #pragma unroll
          for (int q = 0; q < 4; ++q) { o8[q] = u[q]; o8[4 + q] = f[q]; }
          vstore<8>(tr + ((Kc * 3 + i) * NQ + nu) * 8, o8);
          if (cns[i] <= -2) {   // constant exterior states (walls mirror the trace: same speed)
            double px = 0.0, py = 0.0;
            if (cns[i] == -7) {
              const double s = gauss_s(NQ, nu);
              const double xa = m.vxy[(2 * ((i + 1) % 3)) * nt + Kc], ya = m.vxy[(2 * ((i + 1) % 3) + 1) * nt + Kc];
              const double xb = m.vxy[(2 * ((i + 2) % 3)) * nt + Kc], yb = m.vxy[(2 * ((i + 2) % 3) + 1) * nt + Kc];
              px = fma(xb - xa, s, xa);
              py = fma(yb - ya, s, ya);
            }
            Real up[4], ab[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) ab[c] = Real(a0[c]);
            ghost_state(-cns[i], u, ab, nxs[i], nys[i], px, py, t_out, ph, up);
            amax = max_nn(amax, double(wave_speed(up, nxs[i], nys[i], gamma)));
          }
        }
      }
    }
  }
  double av[1] = {amax};
  block_reduce<1>(av, part_alpha + tile, OpMaxNN());
  __syncthreads();
  long long cv[2] = {cnt[0], cnt[1]};
  block_reduce<2>(cv, part_cnt + 2 * tile, OpSum());
  __syncthreads();
}

// OE statistics of the tile's cells and the jump data of the edges it owns
template <int K, typename Real>
__global__ void __launch_bounds__(TPB, sizeof(Real) == 4 ? STATS_MINB_F : STATS_MINB_D)
    k_stats(MeshDev m, Phys ph, StateDev<Real> uh, double *part_dev, const Real *__restrict__ vdi,
            const Real *__restrict__ hsi, Real *__restrict__ ej, const Scalars *sc, double c_out) {
  if (!sc->active) return;
  stats_tile<K, Real>(m, uh, part_dev, sc, blockIdx.x);
  edge_tile<K, Real>(m, ph, uh.avg, vdi, hsi, ej, sc, c_out, blockIdx.x);
}

// RIOE damping, BP limiter, traces and wave speeds of the stage result
template <int K, typename Real>
__global__ void __launch_bounds__(TPB, sizeof(Real) == 4 ? OEBP_MINB_F : OEBP_MINB_D)
    k_oe_bp(MeshDev m, Phys ph, StateDev<Real> uh, StateDev<Real> out, const Real *__restrict__ ej,
            Real *__restrict__ tr, double *part_alpha, long long *part_cnt, const Scalars *sc, int do_oe,
            int do_bp, double c_out, int end_of_step) {
  if (!sc->active) return;
  oe_bp_tile<K, Real>(m, ph, uh, out, ej, tr, part_alpha, part_cnt, sc, do_oe, do_bp, c_out, end_of_step, blockIdx.x);
}

}  // namespace dg

#include "dg_stage_mixed.cuh"

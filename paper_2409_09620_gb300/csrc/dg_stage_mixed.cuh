// dg_stage_mixed.cuh -- stage kernels of the mixed-precision form (FP32 modes
// and flux arithmetic, FP64 cell averages and limiter decisions) without
// exchange buffers.
//
// Each pass reads the cells' modal states and geometry and nothing else: a
// cell evaluates its neighbours' polynomials itself from their modes (read
// through L2), so no trace, vertex or edge record is written by one pass and
// read back by the next.  The HBM traffic per cell and stage is the method's
// own: the flux pass reads v (and u_n) and writes u_h, the statistics pass
// reads u_h, the OE + limiter pass reads u_h and writes u_sigma, plus the
// geometry each needs.
//
// Conservation of the FP64 averages needs the two cells of an edge to form
// exactly opposite flux sums.  Both evaluate the same two traces with the
// same code (edge_dev below, the same FP32 constants in the same order), and every
// operation of the edge flux is an explicit fmaf or a non-contractible
// __fadd_rn / __fmul_rn, so no compiler choice of fused products can differ
// between the unrolled copies of the edge loop in which the two cells meet
// the edge.
#pragma once
#include <type_traits>
#include <utility>

namespace dg {

// f(std::integral_constant<int, 0>{}), ..., f(std::integral_constant<int, N - 1>{}):
// a loop whose index is a compile-time constant in the body
template <typename F, int... Is>
__device__ __forceinline__ void static_for_impl(F &&f, std::integer_sequence<int, Is...>) {
  (f(std::integral_constant<int, Is>{}), ...);
}
template <int N, typename F>
__device__ __forceinline__ void static_for(F &&f) {
  static_for_impl(f, std::make_integer_sequence<int, N>{});
}

// Basis values at the edge Gauss points and at the vertices, as FP32
// compile-time constants chosen by a local edge or vertex index.  With an
// index known at compile time the choice folds away; with a run-time index
// (a neighbour's local edge) it is a select, so the threads of a warp never
// diverge.  Both give the same constants in the same explicit fmaf order, so
// a cell's own trace and its neighbour's evaluation of it agree bit for bit.
template <int K, int NU, int L>
__device__ __forceinline__ float psi_at_edge(int e) {
  constexpr int NQ = Deg<K>::NQ;
  constexpr float p0 = float(psi(L, edge_xi(0, gauss_s(NQ, NU)), edge_eta(0, gauss_s(NQ, NU))));
  constexpr float p1 = float(psi(L, edge_xi(1, gauss_s(NQ, NU)), edge_eta(1, gauss_s(NQ, NU))));
  constexpr float p2 = float(psi(L, edge_xi(2, gauss_s(NQ, NU)), edge_eta(2, gauss_s(NQ, NU))));
  return e == 0 ? p0 : (e == 1 ? p1 : p2);
}
// D = 0: value, 1: d/dxi, 2: d/deta of Psi_L at local vertex v
template <int L, int D>
__device__ __forceinline__ float psi_at_vertex(int v) {
  constexpr float p0 = float(D == 0 ? psi(L, 0.0, 0.0) : D == 1 ? psi_x(L, 0.0, 0.0) : psi_y(L, 0.0, 0.0));
  constexpr float p1 = float(D == 0 ? psi(L, 1.0, 0.0) : D == 1 ? psi_x(L, 1.0, 0.0) : psi_y(L, 1.0, 0.0));
  constexpr float p2 = float(D == 0 ? psi(L, 0.0, 1.0) : D == 1 ? psi_x(L, 0.0, 1.0) : psi_y(L, 0.0, 1.0));
  return v == 0 ? p0 : (v == 1 ? p1 : p2);
}

// deviation from the average of a cell's polynomial at Gauss point NU of local
// edge e: sum_{l >= 1} psi_l(x) hi[c][l]
template <int K, int NU>
__device__ __forceinline__ void edge_dev(int e, const float hi[4][Deg<K>::NB], float d[4]) {
  constexpr int NB = Deg<K>::NB;
  float ps[NB];
  static_for<NB - 1>([&](auto lc) {
    constexpr int l = decltype(lc)::value + 1;
    ps[l] = psi_at_edge<K, NU, l>(e);
  });
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    float s = 0.0f;
#pragma unroll
    for (int l = 1; l < NB; ++l) s = fmaf(ps[l], hi[c][l], s);
    d[c] = s;
  }
}

// value and reference gradient of a cell polynomial at local vertex v
template <int K>
__device__ __forceinline__ void vertex_eval(int v, const float a[4], const float hi[4][Deg<K>::NB], float val[4],
                                            float gx[4], float ge[4]) {
  constexpr int NB = Deg<K>::NB;
  float pv[NB], px[NB], py[NB];
  static_for<NB - 1>([&](auto lc) {
    constexpr int l = decltype(lc)::value + 1;
    pv[l] = psi_at_vertex<l, 0>(v);
    px[l] = psi_at_vertex<l, 1>(v);
    py[l] = psi_at_vertex<l, 2>(v);
  });
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    float s = a[c], x = 0.0f, y = 0.0f;
#pragma unroll
    for (int l = 1; l < NB; ++l) {
      s = fmaf(pv[l], hi[c][l], s);
      x = fmaf(px[l], hi[c][l], x);
      y = fmaf(py[l], hi[c][l], y);
    }
    val[c] = s;
    gx[c] = x;
    ge[c] = y;
  }
}

// value, physical gradient (x, y per component) and 1/rho and sound speed at
// a vertex; jinv = (dxi/dx, dxi/dy, deta/dx, deta/dy)
template <int K>
__device__ __forceinline__ void vertex_phys(const float val[4], const float gx[4], const float ge[4], float jx,
                                            float jy, float ex, float ey, float gamma, float gm1, float grd[8],
                                            float &ri, float &cs) {
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    grd[2 * c] = fdot2(gx[c], jx, ge[c], ex);
    grd[2 * c + 1] = fdot2(gx[c], jy, ge[c], ey);
  }
  ri = 0.0f;
  cs = INFINITY;
  if (val[0] > 0.0f) {
    ri = 1.0f / val[0];
    float p = gm1 * fmaf(-0.5f * fdot2(val[1], val[1], val[2], val[2]), ri, val[3]);
    p = p > 0.0f ? p : 0.0f;
    cs = sqrtf(gamma * p * ri);
  }
}

// physical Hessian (xx, xy, yy per component) of a P2 polynomial
__device__ __forceinline__ void hessian_p2(const float hi[4][6], float jx, float jy, float ex, float ey,
                                           float ho[12]) {
  const float gxx0 = jx * jx, gxe0 = 2.0f * jx * ex, gee0 = ex * ex;
  const float gxx1 = jx * jy, gxe1 = fdot2(jx, ey, jy, ex), gee1 = ex * ey;
  const float gxx2 = jy * jy, gxe2 = 2.0f * jy * ey, gee2 = ey * ey;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    float hxx = 0.0f, hxe = 0.0f, hee = 0.0f;
#pragma unroll
    for (int l = 3; l < 6; ++l) {
      hxx = cfma(psi_2(l, 0), hi[c][l], hxx);
      hxe = cfma(psi_2(l, 1), hi[c][l], hxe);
      hee = cfma(psi_2(l, 2), hi[c][l], hee);
    }
    ho[3 * c + 0] = fma(hxx, gxx0, fdot2(hxe, gxe0, hee, gee0));
    ho[3 * c + 1] = fma(hxx, gxx1, fdot2(hxe, gxe1, hee, gee1));
    ho[3 * c + 2] = fma(hxx, gxx2, fdot2(hxe, gxe2, hee, gee2));
  }
}

// a cell's modal state: FP64 averages (and their FP32 roundings) and FP32 modes
template <int K>
__device__ __forceinline__ void load_mixed(const StateDev<float> &s, int64_t nt, int64_t K_, double a[4],
                                           float af[4], float hi[4][Deg<K>::NB]) {
  load_state<float, Deg<K>::NB>(s, nt, K_, a, hi);
#pragma unroll
  for (int c = 0; c < 4; ++c) af[c] = float(a[c]);
}

// F(u) . d with every product and sum rounded on its own (no contraction;
// the reciprocal is the same instruction sequence wherever it is used)
__device__ __forceinline__ void flux_dir_nc(const float u[4], float dx, float dy, float gm1, float f[4]) {
  const float ri = 1.0f / u[0];
  const float q = fmaf(u[1], u[1], __fmul_rn(u[2], u[2]));
  const float p = __fmul_rn(gm1, __fsub_rn(u[3], __fmul_rn(__fmul_rn(0.5f, q), ri)));
  const float md = fmaf(u[1], dx, __fmul_rn(u[2], dy));
  const float vd = __fmul_rn(md, ri);
  f[0] = md;
  f[1] = fmaf(u[1], vd, __fmul_rn(p, dx));
  f[2] = fmaf(u[2], vd, __fmul_rn(p, dy));
  f[3] = __fmul_rn(__fadd_rn(u[3], p), vd);
}

// ==========================================================================
// K1 (mixed): u_h = a u_n + b (v + dt L(v))
// ==========================================================================
template <int K>
__device__ __forceinline__ void rk_tile_mixed(const MeshDev &m, const Phys &ph, StateDev<float> v, StateDev<float> un,
                                              StateDev<float> uh, double *part_sum, const Scalars *sc, double a,
                                              double b, double c_in, int64_t tile) {
  constexpr int NB = Deg<K>::NB, NQ = Deg<K>::NQ, NV = Deg<K>::NV;
  const int64_t nt = m.nt;
  const int64_t Kc = tile * TPB + threadIdx.x;
  double mass[4] = {0.0, 0.0, 0.0, 0.0};
  if (Kc < nt) {
    const double dt = sc->dt;
    const float alpha = float(sc->alpha), gm1 = ph.gm1_f;
    const double area = m.area[Kc];
    const float jx = m.jinv_f[Kc], jy = m.jinv_f[nt + Kc], ex = m.jinv_f[2 * nt + Kc], ey = m.jinv_f[3 * nt + Kc];
    double v0[4];
    float v0r[4], cv[4][NB];
    load_mixed<K>(v, nt, Kc, v0, v0r, cv);
    int32_t cns[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) cns[i] = m.conn[i * nt + Kc];

    // ---- volume term: |K| sum_mu w_mu F(u(x_mu)) . grad Psi_l ---------------
    float acc[4][NB];
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
      for (int l = 0; l < NB; ++l) acc[c][l] = 0.0f;
#pragma unroll
    for (int mu = 0; mu < NV; ++mu) {
      const double xi = vol_xi(NV, mu), eta = vol_eta(NV, mu), w = vol_w(NV, mu);
      float u[4], g1[4], g2[4];
      eval_fixed<float, NB>(v0r, cv, xi, eta, u);
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
      for (int l = 1; l < NB; ++l) acc[c][l] *= float(area);

    // ---- edge term -------------------------------------------------------------
    float s_hi[4] = {0.0f, 0.0f, 0.0f, 0.0f}, s_lo[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    static_for<3>([&](auto ic) {
      constexpr int i = decltype(ic)::value;
      const int32_t cn = cns[i];
      const float nx = m.nrm_f[(2 * i) * nt + Kc], ny = m.nrm_f[(2 * i + 1) * nt + Kc];
      const float li = m.len_f[i * nt + Kc];
      float tv0[NQ][4], nbr[4], nbh[4][NB];
      if (cn >= 0) {
        double na[4];
        load_mixed<K>(v, nt, cn >> 2, na, nbr, nbh);
      }
      static_for<NQ>([&](auto nc) {
        constexpr int nu = decltype(nc)::value;
        float um[4], up[4], fm[4], fp[4], d[4];
        // own trace at point nu of edge i; the neighbour's at its reversed point
        edge_dev<K, nu>(i, cv, d);
#pragma unroll
        for (int q = 0; q < 4; ++q) um[q] = __fadd_rn(v0r[q], d[q]);
        flux_dir_nc(um, nx, ny, gm1, fm);
        if (cn >= 0) {
          edge_dev<K, NQ - 1 - nu>(cn & 3, nbh, d);
#pragma unroll
          for (int q = 0; q < 4; ++q) up[q] = __fadd_rn(nbr[q], d[q]);
          flux_dir_nc(up, nx, ny, gm1, fp);   // = -F(u+).n of the neighbour, n+ = -n exactly
        } else {
          double px = 0.0, py = 0.0, t_in = 0.0;
          if (cn == -7) {   // the time-dependent exterior state needs the point and the stage time
            constexpr double sg = gauss_s(NQ, nu);
            const double xa = m.vxy[(2 * ((i + 1) % 3)) * nt + Kc], ya = m.vxy[(2 * ((i + 1) % 3) + 1) * nt + Kc];
            const double xb = m.vxy[(2 * ((i + 2) % 3)) * nt + Kc], yb = m.vxy[(2 * ((i + 2) % 3) + 1) * nt + Kc];
            px = fma(xb - xa, sg, xa);
            py = fma(yb - ya, sg, ya);
            t_in = fma(c_in, sc->dt, sc->t);
          }
          ghost_state(-cn, um, v0r, nx, ny, px, py, t_in, ph, up);
          flux_dir_nc(up, nx, ny, gm1, fp);
        }
        // l_i w_nu / 2: the 1/2 of the LF flux rides on the weight
        constexpr float hw = float(0.5 * gauss_w(NQ, nu));
        const float lw = __fmul_rn(li, hw);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const float fh = __fsub_rn(__fadd_rn(fm[c], fp[c]), __fmul_rn(alpha, __fsub_rn(up[c], um[c])));
          const float tv = __fmul_rn(lw, fh);
          tv0[nu][c] = tv;
          static_for<NB - 1>([&](auto lc) {
            constexpr int l = decltype(lc)::value + 1;
            constexpr double pe = -psi(l, edge_xi(i, gauss_s(NQ, nu)), edge_eta(i, gauss_s(NQ, nu)));
            acc[c][l] = cfma(pe, tv, acc[c][l]);
          });
        }
      });
      // the edge's mode-0 contribution summed in an order symmetric under the
      // neighbour's reversed point order (the neighbour's sum is the exact
      // negation), then added to an unevaluated FP32 pair (TwoSum)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const float se = NQ == 3 ? __fadd_rn(__fadd_rn(tv0[0][c], tv0[2][c]), tv0[1][c])
                                 : __fadd_rn(tv0[0][c], tv0[NQ - 1][c]);
        const float x = -se, sum = __fadd_rn(s_hi[c], x), bv = __fsub_rn(sum, s_hi[c]);
        const float err = __fadd_rn(__fsub_rn(s_hi[c], __fsub_rn(sum, bv)), __fsub_rn(x, bv));
        s_hi[c] = sum;
        s_lo[c] = __fadd_rn(s_lo[c], err);
      }
    });

    // ---- mass inverse and SSP-RK combination -----------------------------------
    const double dta = dt * m.iarea[Kc];
    const float ar = float(a), br = float(b), dtar = float(dta);
    const bool first = a == 0.0 && b == 1.0;
    double un0[4] = {0.0, 0.0, 0.0, 0.0};
    float cu[4][NB];
    if (!first) load_state<float, NB>(un, nt, Kc, un0, cu);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const double acc0 = double(s_hi[c]) + double(s_lo[c]);
      const double h0 = first ? fma(dta, acc0, v0[c]) : fdot2(a, un0[c], b, fma(dta, acc0, v0[c]));
      uh.avg[c * nt + Kc] = h0;
      mass[c] = area * h0;
#pragma unroll
      for (int l = 1; l < NB; ++l) {
        const float s = dtar * float(inv_mass_c(l));
        cv[c][l] = first ? fma(s, acc[c][l], cv[c][l]) : fdot2(ar, cu[c][l], br, fma(s, acc[c][l], cv[c][l]));
      }
    }
    store_modes_mixed<NB>(uh, Kc, cv);
  }
  block_reduce<4>(mass, part_sum + 4 * tile, OpSum());
}

// ==========================================================================
// K3 (mixed): RIOE from the cells' own and neighbouring polynomials, BP
// limiter, wave speeds of the stored result at the edge Gauss points
// ==========================================================================
// values per vertex kept by oe_bp_tile_mixed for edge_jumps_mixed: value 4,
// physical gradient 8, 1/rho, sound speed
constexpr int VTX_REC = 14;

// beta and the jump sums sqrt(2 J) of edge i (eqs. OEScalar:Coef2 with the
// trapezoidal rule, RIOESys:Coef1/Coef2) seen from this cell: vertex values
// and gradients at both endpoints, the (constant) Hessian jump once
template <int K>
__device__ __forceinline__ void edge_jumps_mixed(int I, const MeshDev &m, const Phys &ph, const StateDev<float> &uh,
                                                 int64_t Kc, const float a0f[4], const float (*sv)[TPB],
                                                 const float hme[12], int32_t cn, float nx, float ny, double t_out,
                                                 int cw, float &beta, float Jq[4][K + 1]) {
  constexpr int NB = Deg<K>::NB;
  const int64_t nt = m.nt;
  const float gamma = ph.gamma_f, gm1 = ph.gm1_f;
  // the neighbour's state and inverse Jacobian
  float nbf[4], nbh[4][NB];
  float njx = 0.0f, njy = 0.0f, nex = 0.0f, ney = 0.0f;
  int jn = 0;
  if (cn >= 0) {
    const int64_t nb = cn >> 2;
    jn = cn & 3;
    double na[4];
    load_mixed<K>(uh, nt, nb, na, nbf, nbh);
    njx = m.jinv_f[nb]; njy = m.jinv_f[nt + nb]; nex = m.jinv_f[2 * nt + nb]; ney = m.jinv_f[3 * nt + nb];
  }
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int j = 0; j <= K; ++j) Jq[q][j] = 0.0f;
  const int v0 = I == 2 ? 0 : I + 1;                 // v_c = (I + 1) mod 3, then v_d = (I + 2) mod 3
  const int v1 = I == 0 ? 2 : I - 1;
  if constexpr (K == 2) {
    // the Hessians of P2 polynomials (and of every exterior state) are
    // constant: their jump counts at both endpoints, formed once
    float jh[12];
    if (cn >= 0) {
      float hn[12];
      hessian_p2(nbh, njx, njy, nex, ney, hn);
#pragma unroll
      for (int q = 0; q < 12; ++q) jh[q] = hme[q] - hn[q];
    } else {
      float vz[4] = {0.0f, 0.0f, 0.0f, 0.0f}, gz[8] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
      float xv[4], xg[8], xh[12];
      double px = 0.0, py = 0.0;
      if (cn == -7) { px = m.vxy[(2 * v0) * nt + Kc]; py = m.vxy[(2 * v0 + 1) * nt + Kc]; }
      vz[0] = 1.0f;   // an admissible dummy state: only the exterior Hessian is used here
      ghost_vertex(-cn, vz, gz, hme, a0f, nx, ny, px, py, t_out, ph, xv, xg, xh);
#pragma unroll
      for (int q = 0; q < 12; ++q) jh[q] = hme[q] - xh[q];
    }
    if (!cw) {   // momentum rows to (m_n, m_t)
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        const float t0 = jh[3 + r], t1 = jh[6 + r];
        jh[3 + r] = fdot2(t0, nx, t1, ny);
        jh[6 + r] = fdot2(t1, nx, -t0, ny);
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float f = fma(jh[3 * q], jh[3 * q], fma(jh[3 * q + 1] + jh[3 * q + 1], jh[3 * q + 1],
                                                      jh[3 * q + 2] * jh[3 * q + 2]));
      Jq[q][K] = f + f;
    }
  }
  beta = 0.0f;
#pragma unroll
  for (int ev = 0; ev < 2; ++ev) {
    const int ov = ev == 0 ? v0 : v1;
    // this cell's value, physical gradient, 1/rho and sound speed at the vertex
    float val[4], grd[8];
#pragma unroll
    for (int q = 0; q < 4; ++q) val[q] = sv[VTX_REC * ov + q][threadIdx.x];
#pragma unroll
    for (int q = 0; q < 8; ++q) grd[q] = sv[VTX_REC * ov + 4 + q][threadIdx.x];
    const float ri = sv[VTX_REC * ov + 12][threadIdx.x], cs = sv[VTX_REC * ov + 13][threadIdx.x];
    const float r_own = fma(fabsf(fdot2(val[1], nx, val[2], ny)), ri, cs);
    float xv[4], xg[8], r_oth;
    if (cn >= 0) {
      const int xvtx = (jn + 2 - ev) % 3;            // the neighbour's copy of this vertex
      float xgx[4], xge[4], xri, xcs;
      vertex_eval<K>(xvtx, nbf, nbh, xv, xgx, xge);
      vertex_phys<K>(xv, xgx, xge, njx, njy, nex, ney, gamma, gm1, xg, xri, xcs);
      r_oth = fma(fabsf(fdot2(xv[1], nx, xv[2], ny)), xri, xcs);
    } else {
      double px = 0.0, py = 0.0;
      if (cn == -7) { px = m.vxy[(2 * ov) * nt + Kc]; py = m.vxy[(2 * ov + 1) * nt + Kc]; }
      float xh[12];
      ghost_vertex(-cn, val, grd, hme, a0f, nx, ny, px, py, t_out, ph, xv, xg, xh);
      r_oth = cn == -1 ? r_own : wave_speed(xv, nx, ny, gamma);   // a mirror state has the same speed
    }
    beta = max_nn(beta, max_nn(r_own, r_oth));
    float jv[4], jg[4][2];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      jv[c] = val[c] - xv[c];
      jg[c][0] = grd[2 * c] - xg[2 * c];
      jg[c][1] = grd[2 * c + 1] - xg[2 * c + 1];
    }
    if (!cw) {   // rotate the momentum jumps to (m_n, m_t)
      float t0 = jv[1], t1 = jv[2];
      jv[1] = fdot2(t0, nx, t1, ny); jv[2] = fdot2(t1, nx, -t0, ny);
#pragma unroll
      for (int d = 0; d < 2; ++d) {
        t0 = jg[1][d]; t1 = jg[2][d];
        jg[1][d] = fdot2(t0, nx, t1, ny); jg[2][d] = fdot2(t1, nx, -t0, ny);
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      Jq[q][0] = fma(jv[q], jv[q], Jq[q][0]);
      Jq[q][1] = fma(jg[q][0], jg[q][0], fma(jg[q][1], jg[q][1], Jq[q][1]));
    }
  }
}

// ---------------------------------------------------------------------------
// FP64 theta of the mixed form (Sec. 4.4 Steps 1-2), one warp per cell
// ---------------------------------------------------------------------------
// The limiter point set of a P_K cell: the 3 (K + 1) edge Gauss points, then
// two extra points (the internal nodes of the optimal decomposition for P2,
// the vertices v1, v2 for P1; with the classical decomposition both extra
// rows are the weighted edge combination of zxs_extra_points).  LimTab holds,
// per point, psi_1 .. psi_{NB-1} there; the node rows come from the mesh.
template <int K>
struct LimTab {
  static constexpr int NQ = K + 1, NE = 3 * NQ, NP = NE + 2, NB = Deg<K>::NB;
  double v[NP][NB];
};
template <int K>
constexpr LimTab<K> make_lim_tab() {
  LimTab<K> t{};
  constexpr int NQ = LimTab<K>::NQ, NE = LimTab<K>::NE, NB = LimTab<K>::NB;
  for (int p = 0; p < NE; ++p) {
    const double sg = gauss_s(NQ, p % NQ);
    for (int l = 0; l < NB; ++l) t.v[p][l] = psi(l, edge_xi(p / NQ, sg), edge_eta(p / NQ, sg));
  }
  for (int l = 0; l < NB; ++l) {
    double acc = 0.0;   // classical extra row: P1 the first edge point, P2 -1/6 sum_p w_p psi(x_p)
    for (int p = 0; p < NE; ++p) acc += gauss_w(NQ, p % NQ) * t.v[p][l];
    const double v = K == 1 ? t.v[0][l] : (-1.0 / 6.0) * acc;
    t.v[NE][l] = v;
    t.v[NE + 1][l] = v;
  }
  return t;
}
static __device__ const LimTab<1> g_lim_tab1 = make_lim_tab<1>();
static __device__ const LimTab<2> g_lim_tab2 = make_lim_tab<2>();

// per-warp scratch of the cooperative limiter: the cell's averages, modes in
// FP64, the scaled modes (FP32 and back in FP64) and the scalars of its theta
template <int K>
struct LimScratch {
  static constexpr int NM = 4 * (Deg<K>::NB - 1);
  double a0[4], hd[NM], hsd[NM], sa[4];
  float hs[NM];
};

// Warp reductions over the limiter points (lanes beyond the set hold the
// identity): minimum on the integer units through order-preserving keys,
// maximum of non-negative values on their bit patterns.
__device__ __forceinline__ double warp_min_ord(double x) {
  long long k = ord_key(x);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) k = min(k, __shfl_xor_sync(0xffffffffu, k, o));
  return ord_val(k);
}
__device__ __forceinline__ double warp_max_nn(double x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x = max_nn(x, __shfl_xor_sync(0xffffffffu, x, o));
  return x;
}

// FP64 theta for the cells of this warp that failed the FP32 screen (flag).
// The warp takes them one at a time; lane p evaluates limiter point p and
// lane j scales mode j, so the serial FP64 work of a cell (well over a
// thousand FP64 instructions, which GB300's narrow FP64 pipe runs at about
// one warp instruction per 64 cycles per scheduler) shrinks to about a
// hundred and fifty warp instructions.  The targets cover the rounding of
// the FP32 store (2^-22 per unit of sum |mode|, |Psi| <= 4 on K); the stored
// FP32 modes are then verified in FP64 at every point of the set, and a cell
// that still fails keeps its average only.  On return a flagged lane's hi
// holds the stored modes; limited is set when theta < 1 or the cell fell back
// to its average.  Every lane of the warp calls this (the shuffles and
// warp barriers take all 32).
template <int K>
__device__ __forceinline__ void limit_fp64_warp(const MeshDev &m, const Phys &ph, bool flag, int64_t Kc,
                                                const double a0[4], float hi[4][Deg<K>::NB], StateDev<float> out,
                                                long long &limited) {
  constexpr int NB = Deg<K>::NB, NQ = K + 1, NE = 3 * NQ, NP = NE + 2, NM = 4 * (NB - 1);
  static_assert(NP <= 32 && NM <= 32, "one lane per point and per mode");
  const unsigned FULL = 0xffffffffu;
  unsigned todo = __ballot_sync(FULL, flag);
  if (todo == 0u) return;
  __shared__ LimScratch<K> scr_all[TPB / 32];
  LimScratch<K> &S = scr_all[threadIdx.x >> 5];
  const int lane = threadIdx.x & 31;
  const int64_t nt = m.nt;
  const double r22 = 2.384185791015625e-07;   // 2^-22
  // this lane's basis values at its point (edge rows; extra rows per cell below)
  double psv[NB];
  const bool on_pt = lane < NP;
  const int prow = on_pt ? lane : 0;
#pragma unroll
  for (int l = 1; l < NB; ++l) psv[l] = K == 1 ? g_lim_tab1.v[prow][l] : g_lim_tab2.v[prow][l];
  const bool node_row = on_pt && lane >= NE && !ph.decomp;
  while (todo) {
    const int src = __ffs(todo) - 1;
    todo &= todo - 1u;
    const int64_t Ks = __shfl_sync(FULL, Kc, src);
    if (lane == src) {
#pragma unroll
      for (int c = 0; c < 4; ++c) S.a0[c] = a0[c];
#pragma unroll
      for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int l = 1; l < NB; ++l) S.hs[c * (NB - 1) + l - 1] = hi[c][l];
    }
    __syncwarp();
    if (lane < NM) S.hd[lane] = double(S.hs[lane]);
    if (node_row) {   // the extra point of this cell: P2 internal node, P1 vertex
      const int e = lane - NE;
      if (K == 1) {
        const int vp = m.limv[e * nt + Ks];
#pragma unroll
        for (int l = 1; l < NB; ++l) psv[l] = psi(l, vert_xi(vp), vert_eta(vp));
      } else {
#pragma unroll
        for (int l = 1; l < NB; ++l) psv[l] = m.psi_node[(5 * e + l - 1) * nt + Ks];
      }
    }
    __syncwarp();
    if (lane < 4) {
      double sa = 0.0;
#pragma unroll
      for (int l = 1; l < NB; ++l) sa += fabs(S.hd[lane * (NB - 1) + l - 1]);
      S.sa[lane] = sa;
    }
    double A[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) A[c] = S.a0[c];
    // deviations of the unlimited polynomial at this lane's point
    double d[4] = {0.0, 0.0, 0.0, 0.0};
    if (on_pt) {
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        double acc = 0.0;
#pragma unroll
        for (int l = 1; l < NB; ++l) acc = fma(psv[l], S.hd[c * (NB - 1) + l - 1], acc);
        d[c] = acc;
      }
    }
    __syncwarp();
    double Sa[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) Sa[c] = S.sa[c];
    // Step 1: density
    const double rmin = warp_min_ord(on_pt ? A[0] + d[0] : INFINITY);
    const double eps1 = fmin(A[0], 1e-13);
    const double tgt1 = fmin(A[0], fma(2.0 * r22, Sa[0], eps1));
    const double th1 = rmin < tgt1 ? (A[0] - tgt1) / (A[0] - rmin) : 1.0;
    // Step 2: internal energy of the density-limited polynomial; the target
    // covers the FP32 store through the largest squared speed on the set
    const double w0 = fma(th1, d[0], A[0]), w1 = A[1] + d[1], w2 = A[2] + d[2], w3 = A[3] + d[3];
    const double q = fdot2(w1, w1, w2, w2);
    const double v2 = q / (w0 * w0);
    const double vmax2 = warp_max_nn(on_pt && v2 == v2 ? v2 : 0.0);   // a NaN is ignored, as by fmax
    const double Ebar = int_energy(A);
    const double RE = r22 * fma(sqrt(vmax2), Sa[1] + Sa[2], fma(vmax2 * th1, Sa[0], Sa[3]));
    const double eps2 = fmin(Ebar, 1e-13);
    const double tgt2 = fmin(Ebar, fma(2.0, RE, eps2));
    // E - |m|^2 / (2 rho) < tgt2 tested as rho E - |m|^2 / 2 < tgt2 rho (rho > 0):
    // the division only at points that violate the target
    double e_pt = INFINITY;
    if (on_pt && (!(w0 > 0.0) || fma(w3, w0, -0.5 * q) < tgt2 * w0)) e_pt = w3 - 0.5 * q / w0;
    const double emin = warp_min_ord(e_pt);
    const double th2 = emin < tgt2 ? (Ebar - tgt2) / (Ebar - emin) : 1.0;
    // the scaled modes, one per lane, stored in FP32 and read back in FP64
    if (lane < NM) {
      const double th = lane < NB - 1 ? th1 * th2 : th2;
      const float h = float(th * S.hd[lane]);
      S.hs[lane] = h;
      S.hsd[lane] = double(h);
    }
    __syncwarp();
    // verify the stored modes at every point of the set
    bool bad_pt = false;
    if (on_pt) {
      double v[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        double acc = 0.0;
#pragma unroll
        for (int l = 1; l < NB; ++l) acc = fma(psv[l], S.hsd[c * (NB - 1) + l - 1], acc);
        v[c] = A[c] + acc;
      }
      bad_pt = !(v[0] > 0.0) || !(fma(v[3], v[0], -0.5 * fdot2(v[1], v[1], v[2], v[2])) > 0.0);
    }
    const bool bad = __any_sync(FULL, bad_pt);
    if (lane == src) {
#pragma unroll
      for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int l = 1; l < NB; ++l) hi[c][l] = bad ? 0.0f : S.hs[c * (NB - 1) + l - 1];
      store_modes_mixed<NB>(out, Kc, hi);
      if (th1 < 1.0 || th2 < 1.0 || bad) limited = 1;
    }
    __syncwarp();
  }
}

// FP32 screen of the BP limiter (Sec. 4.4) in the mixed form.  Stores the
// averages, and the modes of every cell that passes; returns true for a cell
// whose theta must be taken in FP64 (limit_fp64_warp).  cnt[1] counts a cell
// average outside G (left unlimited).
template <int K>
__device__ __forceinline__ bool limit_screen_mixed(const MeshDev &m, const Phys &ph, const double a0[4],
                                                   const float a0f[4], const float hi[4][Deg<K>::NB],
                                                   StateDev<float> out, int64_t Kc, int do_bp, long long cnt[2]) {
  constexpr int NB = Deg<K>::NB, NQ = Deg<K>::NQ;
  const int64_t nt = m.nt;
  float px[2], py[2];
  if (K == 1) {
    const int v1 = m.limv[Kc], v2 = m.limv[nt + Kc];
    px[0] = float(vert_xi(v1)); py[0] = float(vert_eta(v1)); px[1] = float(vert_xi(v2)); py[1] = float(vert_eta(v2));
  } else {
    px[0] = m.node_f[Kc]; py[0] = m.node_f[nt + Kc]; px[1] = m.node_f[2 * nt + Kc]; py[1] = m.node_f[3 * nt + Kc];
  }
#pragma unroll
  for (int c = 0; c < 4; ++c) out.avg[c * nt + Kc] = a0[c];
  bool avg_ok;
  float eps1, eps2;
  {
    const float q2 = fdot2(a0f[1], a0f[1], a0f[2], a0f[2]), pe = a0f[3] * a0f[0];
    if (a0f[0] > 2e-13f && fmaf(-0.5f, q2, pe) > fdot2(2e-13f, a0f[0], 1e-5f, fmaf(0.5f, q2, fabsf(pe)))) {
      avg_ok = true;
      eps1 = eps2 = float(1e-13);
    } else {
      const double Ebar = int_energy(a0);
      avg_ok = (a0[0] > 0.0) && (Ebar > 0.0);
      eps1 = float(fmin(a0[0], 1e-13));
      eps2 = float(fmin(Ebar, 1e-13));
    }
  }
  bool lim64 = false;
  if (do_bp) {
    if (!avg_ok) {
      cnt[1] = 1;
    } else {
      // |Psi_l| <= 4 on K: every point's deviation is at most D in magnitude
      float D[4], S[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        float a = 0.0f;
#pragma unroll
        for (int l = 1; l < NB; ++l) a += fabsf(hi[c][l]);
        D[c] = 4.0f * a;
        S[c] = fabsf(a0f[c]) + D[c];
      }
      auto passes = [&](const float d[4]) -> bool {
        const float r = a0f[0] + d[0];
        if (!(r >= eps1 + 1e-5f * S[0])) return false;
        const float m1 = a0f[1] + d[1], m2 = a0f[2] + d[2], E = a0f[3] + d[3];
        const float ri = 1.0f / r;
        const float q = fdot2(m1, m1, m2, m2) * ri;
        const float v = sqrtf(q * ri);
        const float margin = fdot2(1e-5f, fmaf(v, S[1] + S[2], fmaf(v * v, S[0], S[3])), 1e-6f, fabsf(E) + q);
        return E - 0.5f * q >= eps2 + margin;
      };
      // A bound over the whole cell settles the usual (smooth) cell without
      // visiting its points: each point's density is at least r_lo, its
      // energy at least E_lo and its momentum norm at most M_hi.  If these
      // pass the point test with twice the largest margin any point could
      // need (the doubling covers the rounding of the bound), every point
      // passes it.  Either way a cell goes to the FP64 theta only if some
      // point might fail, and that leaves an admissible cell unchanged, so
      // the bound changes no result.
      bool ok = false;
      const float r_lo = a0f[0] - D[0];
      if (r_lo >= eps1 + 2e-5f * S[0]) {
        const float M_hi = sqrtf(fdot2(a0f[1], a0f[1], a0f[2], a0f[2])) + D[1] + D[2];
        const float E_lo = a0f[3] - D[3], E_hi = fabsf(a0f[3]) + D[3];
        const float v_hi = M_hi / r_lo, q_hi = M_hi * v_hi;
        const float margin = fdot2(1e-5f, fmaf(v_hi, S[1] + S[2], fmaf(v_hi * v_hi, S[0], S[3])), 1e-6f, E_hi + q_hi);
        ok = E_lo - 0.5f * q_hi >= eps2 + 2.0f * margin;
      }
      // otherwise the points one at a time (few live registers); the
      // classical decomposition's extra point needs the weighted edge sum
      if (!ok) {
        ok = true;
        float zs[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
        for (int e = 0; e < 3; ++e)
          static_for<NQ>([&](auto nc) {
            constexpr int nu = decltype(nc)::value;
            float d[4];
            edge_dev<K, nu>(e, hi, d);
            ok = passes(d) && ok;
#pragma unroll
            for (int c = 0; c < 4; ++c) zs[c] += float(gauss_w(NQ, nu)) * d[c];
          });
        if (ph.decomp) {
          float d[4];
#pragma unroll
          for (int c = 0; c < 4; ++c) d[c] = K == 1 ? 0.0f : float(-1.0 / 6.0) * zs[c];
          if (K == 1) edge_dev<K, 0>(0, hi, d);   // P1: the edge weights sum to one (see zxs_extra_points)
          ok = passes(d) && ok;
        } else {
#pragma unroll
          for (int p = 0; p < 2; ++p) {
            float d[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
              float sacc = 0.0f;
#pragma unroll
              for (int l = 1; l < NB; ++l) sacc = fmaf(psi_t<float>(l, px[p], py[p]), hi[c][l], sacc);
              d[c] = sacc;
            }
            ok = passes(d) && ok;
          }
        }
      }
      lim64 = !ok;
    }
  }
  if (!lim64) store_modes_mixed<NB>(out, Kc, hi);
  return lim64;
}

// wave speeds at the edge Gauss points of the stored state (and of the
// exterior states of constant-state boundaries), evaluated as the next flux
// pass evaluates its traces, into amax
template <int K>
__device__ __forceinline__ void alpha_mixed(const MeshDev &m, const Phys &ph, const float a0f[4],
                                            const float hi[4][Deg<K>::NB], const float nxs[3], const float nys[3],
                                            const int32_t cns[3], int64_t Kc, double t_out, double &amax) {
  constexpr int NQ = Deg<K>::NQ;
  const int64_t nt = m.nt;
  const float gamma = ph.gamma_f, gm1 = ph.gm1_f;
  float amax32 = 0.0f;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    static_for<NQ>([&](auto nc) {
      constexpr int nu = decltype(nc)::value;
      float u[4], d[4];
      edge_dev<K, nu>(i, hi, d);
#pragma unroll
      for (int c = 0; c < 4; ++c) u[c] = __fadd_rn(a0f[c], d[c]);
      // |v . n| + c (+inf for rho <= 0, pressure clamped at 0)
      float r = INFINITY;
      if (u[0] > 0.0f) {
        const float ri = 1.0f / u[0];
        float p = gm1 * fmaf(-0.5f * fdot2(u[1], u[1], u[2], u[2]), ri, u[3]);
        p = p > 0.0f ? p : 0.0f;
        r = fmaf(fabsf(fdot2(u[1], nxs[i], u[2], nys[i])), ri, sqrtf(gamma * p * ri));
      }
      amax32 = (r > amax32 || r != r) ? r : amax32;
      if (cns[i] <= -2) {   // constant exterior states (walls mirror the trace: same speed)
        double qx = 0.0, qy = 0.0;
        if (cns[i] == -7) {
          constexpr double sg = gauss_s(NQ, nu);
          const double xa = m.vxy[(2 * ((i + 1) % 3)) * nt + Kc], ya = m.vxy[(2 * ((i + 1) % 3) + 1) * nt + Kc];
          const double xb = m.vxy[(2 * ((i + 2) % 3)) * nt + Kc], yb = m.vxy[(2 * ((i + 2) % 3) + 1) * nt + Kc];
          qx = fma(xb - xa, sg, xa);
          qy = fma(yb - ya, sg, ya);
        }
        float up[4];
        ghost_state(-cns[i], u, a0f, nxs[i], nys[i], qx, qy, t_out, ph, up);
        const float rg = wave_speed(up, nxs[i], nys[i], gamma);
        amax32 = (rg > amax32 || rg != rg) ? rg : amax32;
      }
    });
  }
  amax = max_nn(amax, double(amax32));
}

template <int K>
__device__ __forceinline__ void oe_bp_tile_mixed(const MeshDev &m, const Phys &ph, StateDev<float> uh,
                                                 StateDev<float> out, double *part_alpha, long long *part_cnt,
                                                 const Scalars *sc, int do_oe, int do_bp, double c_out, int end_of_step,
                                                 int64_t tile) {
  constexpr int NB = Deg<K>::NB;
  const int64_t nt = m.nt;
  const int64_t Kc = tile * TPB + threadIdx.x;
  const bool live = Kc < nt;
  double amax = 0.0;
  long long cnt[2] = {0, 0};
  // OE exterior states at the time of the stage result; the next stage's
  // alpha there too, or at the end time after the last stage of a clamped step
  const double dt = sc->dt, t_out = fma(c_out, sc->dt, sc->t);
  const double t_alpha = end_of_step && sc->pad ? sc->t_end : t_out;
  double a0[4] = {0.0, 0.0, 0.0, 0.0};
  float a0f[4] = {0.0f, 0.0f, 0.0f, 0.0f}, hi[4][NB];
  float nxs[3], nys[3];
  int32_t cns[3];
  bool lim64 = false;
  if (live) {
    load_mixed<K>(uh, nt, Kc, a0, a0f, hi);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      nxs[i] = m.nrm_f[(2 * i) * nt + Kc];
      nys[i] = m.nrm_f[(2 * i + 1) * nt + Kc];
      cns[i] = m.conn[i * nt + Kc];
    }
    if (do_oe) {
      const int cw = ph.oe == 2;
      const float jx = m.jinv_f[Kc], jy = m.jinv_f[nt + Kc], ex = m.jinv_f[2 * nt + Kc], ey = m.jinv_f[3 * nt + Kc];
      const float dtf = float(dt);
      float iD[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) iD[q] = sc->invDf[q];
      float hme[12];
#pragma unroll
      for (int q = 0; q < 12; ++q) hme[q] = 0.0f;
      if constexpr (K == 2) hessian_p2(hi, jx, jy, ex, ey, hme);
      // the cell's own vertex data, formed once (each vertex serves two
      // edges) at compile-time vertex indices, in this thread's column of a
      // block-shared array (no exchange between threads, so no barrier)
      __shared__ float s_vtx[3 * VTX_REC][TPB];
      {
        const float gamma = ph.gamma_f, gm1 = ph.gm1_f;
        static_for<3>([&](auto vc) {
          constexpr int v = decltype(vc)::value;
          float val[4], gx[4], ge[4], grd[8], ri, cs;
          vertex_eval<K>(v, a0f, hi, val, gx, ge);
          vertex_phys<K>(val, gx, ge, jx, jy, ex, ey, gamma, gm1, grd, ri, cs);
#pragma unroll
          for (int q = 0; q < 4; ++q) s_vtx[VTX_REC * v + q][threadIdx.x] = val[q];
#pragma unroll
          for (int q = 0; q < 8; ++q) s_vtx[VTX_REC * v + 4 + q][threadIdx.x] = grd[q];
          s_vtx[VTX_REC * v + 12][threadIdx.x] = ri;
          s_vtx[VTX_REC * v + 13][threadIdx.x] = cs;
        });
      }
      // sigma_q^j = sum_i (beta_i / h_i) A^{k,j} h_i^j sqrt(J) / D_q (see oe_bp_tile)
      float sig[4][K + 1];
#pragma unroll
      for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int j = 0; j <= K; ++j) sig[c][j] = 0.0f;
      // one edge at a time in a loop that is not unrolled: the edge work is
      // the bulk of the kernel's code, and one copy of it keeps the
      // instruction cache warm
#pragma unroll 1
      for (int i = 0; i < 3; ++i) {
        float beta, Jq[4][K + 1];
        edge_jumps_mixed<K>(i, m, ph, uh, Kc, a0f, s_vtx, hme, m.conn[i * nt + Kc], m.nrm_f[(2 * i) * nt + Kc],
                            m.nrm_f[(2 * i + 1) * nt + Kc], t_out, cw, beta, Jq);
        float er[4][K + 1];
#pragma unroll
        for (int j = 0; j <= K; ++j) {
          er[0][j] = sqrtf(Jq[0][j]);
          er[3][j] = sqrtf(Jq[3][j]);
          if (cw) {
            er[1][j] = sqrtf(Jq[1][j]);
            er[2][j] = sqrtf(Jq[2][j]);
          } else {
            er[1][j] = sqrtf(max_nn(Jq[1][j], Jq[2][j]));
            er[2][j] = 0.0f;
          }
        }
        const float h = m.hgeo_f[i * nt + Kc], ih = m.hgeo_f[(3 + i) * nt + Kc];
        const float bh = beta * ih;
        const bool bh_finite = is_finite_bits(bh);
        float hj = 1.0f;
#pragma unroll
        for (int j = 0; j <= K; ++j) {
          const float F = bh * (float((2.0 * j + 1.0) / ((2.0 * K - 1.0) * (j == 2 ? 2.0 : 1.0)) *
                                      0.70710678118654752440) * hj);
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            if (c == 2 && !cw) continue;
            const float e = er[c][j];
            if (bh_finite || nonzero_bits(e)) sig[c][j] = fma(F, e, sig[c][j]);
          }
          hj *= h;
        }
      }
#pragma unroll
      for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int j = 0; j <= K; ++j) sig[c][j] = nonzero_bits(iD[c]) ? iD[c] * sig[c][j] : 0.0f;
      float fac[4][K + 1];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        if (c == 2 && !cw) {
#pragma unroll
          for (int md = 1; md <= K; ++md) fac[2][md] = fac[1][md];
          continue;
        }
        float sacc = sig[c][0];
#pragma unroll
        for (int md = 1; md <= K; ++md) {
          sacc += sig[c][md];
          fac[c][md] = exp_neg(dtf * sacc);
        }
      }
#pragma unroll
      for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int l = 1; l < NB; ++l) hi[c][l] *= fac[c][degree_of(l)];
    }
    lim64 = limit_screen_mixed<K>(m, ph, a0, a0f, hi, out, Kc, do_bp, cnt);
  }
  // the FP64 theta of the cells that failed the screen, by the whole warp
  limit_fp64_warp<K>(m, ph, lim64, Kc, a0, hi, out, cnt[0]);
  if (live) alpha_mixed<K>(m, ph, a0f, hi, nxs, nys, cns, Kc, t_alpha, amax);
  double av[1] = {amax};
  block_reduce<1>(av, part_alpha + tile, OpMaxNN());
  __syncthreads();
  long long cv[2] = {cnt[0], cnt[1]};
  block_reduce<2>(cv, part_cnt + 2 * tile, OpSum());
  __syncthreads();
}

}  // namespace dg

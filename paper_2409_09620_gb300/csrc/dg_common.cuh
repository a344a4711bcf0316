// dg_common.cuh -- device data layout, basis, quadrature and physics of the
// GB300 BP RI-OEDG solver (Ding, Cui & Wu, arXiv 2409.09620).
//
// Data layout in HBM (one mesh of nt cells):
//   state     avg[4][nt] (FP64 cell averages, mode 0)  +  hi[4][nb-1][nt] (modes 1..nb-1, Real)
//   geometry  area[nt], jinv[4][nt] (dxi/dx, dxi/dy, deta/dx, deta/dy), nrm[6][nt],
//             len[3][nt], hgeo[6][nt] (h_i, 1/h_i), vxy[6][nt], node[4][nt] (P2 internal
//             nodes, reference coords),
//             limv[2][nt] (P1 limiter vertices), conn[3][nt] (neighbour << 2 | its edge, or -tag)
//   exchange buffers (FP64 form only; the mixed form's passes read the
//   neighbours' modal states instead, see dg_stage_mixed.cuh):
//             tr[nt][3][Q][8]  traces of the stage input at edge Gauss points:
//                              u (4) and F(u).n_i (4), written by the cell that owns them
//             vd[nt][3][16]    value (4), physical gradient (8), 1/rho and sound speed
//                              of u_h at each vertex (2 padding values)
//             hs[nt][12]       physical Hessian (xx, xy, yy) of u_h per component (P2)
//             ej[ne][16]       per edge: beta and the square roots of the OE jump sums
// Every kernel is one thread per cell; reductions are per-block partials
// reduced in a fixed order, so results are bitwise reproducible.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "dg_math.h"

namespace dg {

constexpr int TPB = 128;                 // cells per block
constexpr int FIN_THREADS = 1024;        // threads (virtual lanes) of the finalize reductions

template <int K> struct Deg;
template <> struct Deg<1> { static constexpr int NB = 3, NQ = 2, NV = 3; };
template <> struct Deg<2> { static constexpr int NB = 6, NQ = 3, NV = 6; };

struct MeshDev {
  int64_t nt;
  const double *area, *jinv, *nrm, *len, *vxy, *node;
  const double *hgeo;   // [6][nt]: h_i = 2|K| / l_i (i = 0..2), then 1 / h_i
  const int8_t *limv;
  const int32_t *conn;
  // edges, each once, ordered by the owning cell (the lower cell id of an
  // interior edge; the cell of a boundary edge)
  int64_t ne;
  const int32_t *e_cell;   // [ne] owning cell
  const int8_t *e_loc;     // [ne] its local edge
  const int32_t *etile;    // [ntiles + 1] first edge owned by each tile of TPB cells
  const int32_t *cedge;    // [3][nt] edge index of (cell, local edge)
  // FP32 copies of the geometry the mixed-precision kernels read (the same
  // rounded values, without a conversion per read), and 1/|K| in FP64
  const float *jinv_f, *nrm_f, *len_f, *hgeo_f;
  const double *iarea;
  const float *node_f;     // [4][nt] FP32 copy of node (P2 internal limiter nodes)
  const double *psi_node;  // [2][5][nt] P2 basis psi_1..psi_5 at the two internal nodes
};

// geometry in the working precision of a kernel
template <typename Real> struct Geo;
template <> struct Geo<double> {
  static __device__ __forceinline__ const double *jinv(const MeshDev &m) { return m.jinv; }
  static __device__ __forceinline__ const double *nrm(const MeshDev &m) { return m.nrm; }
  static __device__ __forceinline__ const double *len(const MeshDev &m) { return m.len; }
  static __device__ __forceinline__ const double *hgeo(const MeshDev &m) { return m.hgeo; }
};
template <> struct Geo<float> {
  static __device__ __forceinline__ const float *jinv(const MeshDev &m) { return m.jinv_f; }
  static __device__ __forceinline__ const float *nrm(const MeshDev &m) { return m.nrm_f; }
  static __device__ __forceinline__ const float *len(const MeshDev &m) { return m.len_f; }
  static __device__ __forceinline__ const float *hgeo(const MeshDev &m) { return m.hgeo_f; }
};

// values per edge Gauss point in the trace buffer tr[nt][3][Q][TS]: u and
// F(u).n in the FP64 form (TS = 8); u only in the FP32 form (TS = 4), whose
// stage kernel recomputes F(u).n in FP32 on both sides of the edge.  The two
// cells of an edge have exactly opposite normals, so the recomputed fluxes
// are the negated values the other cell uses, bit for bit.
template <typename Real> struct TraceStride { static constexpr int value = sizeof(Real) == 4 ? 4 : 8; };
__host__ __device__ constexpr int trace_stride(int precision) { return precision == 0 ? 8 : 4; }
// the exchange buffers (traces, vertex records, Hessians, edge records) are
// used by the FP64 form only; the mixed form's passes read the states directly
__host__ __device__ constexpr bool uses_exchange(int precision) { return precision == 0; }
// per-edge OE record ej[ne][EJ_STRIDE]: beta, then sqrt(2 J) of the trapezoidal
// jump sums J for q = rho, (m_n|m_t max | m1), (m2), E and j = 0..k (13 used)
constexpr int EJ_STRIDE = 16;
__host__ __device__ constexpr int ej_row(int q, int j, int K) { return 1 + q * (K + 1) + j; }
// per-cell vertex record vd[nt][3][VD_STRIDE]: value (4), gradient (8), 1/rho, sound speed
constexpr int VD_STRIDE = 16;
constexpr int VD_CELL = 3 * VD_STRIDE;

// 16-byte vector loads and stores of N consecutive values (N a multiple of 16/sizeof(T))
template <typename T> struct Vec16;
template <> struct Vec16<float> {
  using type = float4;
  static constexpr int n = 4;
  static __device__ __forceinline__ void get(const float4 &v, float *o) { o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w; }
  static __device__ __forceinline__ float4 make(const float *i) { return make_float4(i[0], i[1], i[2], i[3]); }
};
template <> struct Vec16<double> {
  using type = double2;
  static constexpr int n = 2;
  static __device__ __forceinline__ void get(const double2 &v, double *o) { o[0] = v.x; o[1] = v.y; }
  static __device__ __forceinline__ double2 make(const double *i) { return make_double2(i[0], i[1]); }
};
template <int N, typename T>
__device__ __forceinline__ void vload(const T *__restrict__ p, T out[N]) {
  constexpr int L = Vec16<T>::n;
  const typename Vec16<T>::type *q = reinterpret_cast<const typename Vec16<T>::type *>(p);
#pragma unroll
  for (int k = 0; k < N / L; ++k) Vec16<T>::get(q[k], out + k * L);
}
template <int N, typename T>
__device__ __forceinline__ void vstore(T *__restrict__ p, const T in[N]) {
  constexpr int L = Vec16<T>::n;
  typename Vec16<T>::type *q = reinterpret_cast<typename Vec16<T>::type *>(p);
#pragma unroll
  for (int k = 0; k < N / L; ++k) q[k] = Vec16<T>::make(in + k * L);
}

template <typename Real> struct StateDev {
  double *avg;   // [4][nt]
  Real *hi;      // FP64 form: [4][nb-1][nt]; mixed form: [nt][4][nb-1] (one 16-byte aligned record per cell)
};

struct Phys {
  double gamma;
  double bc[4][4];
  double shock_x0, shock_cot, shock_vx;   // x_s(y, t) = x0 + y cot(angle) + t speed / sin(angle)
  int shock_pre, shock_post;
  int oe, bp, k, decomp;   // decomp: 0 optimal convex decomposition, 1 classical (ZXS)
  float gamma_f, gm1_f;    // FP32 roundings of gamma and gamma - 1 (mixed form)
};

// gamma and gamma - 1 in the working precision (no conversion in the kernels)
template <typename Real>
__device__ __forceinline__ Real phys_gamma(const Phys &ph) {
  if constexpr (sizeof(Real) == sizeof(float)) return ph.gamma_f; else return ph.gamma;
}
template <typename Real>
__device__ __forceinline__ Real phys_gm1(const Phys &ph) {
  if constexpr (sizeof(Real) == sizeof(float)) return ph.gm1_f; else return ph.gamma - 1.0;
}

// Device-resident scalars of one solver.
struct Scalars {
  double t, t_end, dt, alpha, cfl, min_ca;
  double mean[4], area_total, dev[5];
  double invD[4];   // 1 / normaliser of the damped quantities (rho, m_n|m1, m_t|m2, E); 0 if constant
  float invDf[4];   // their FP32 roundings (mixed form)
  long long steps, limited, nonphys, breaches;
  int active, pad;
};

// ------------------------------------------------------------------------
// Basis of eq. (basisfunc), modes 0..5, on the reference triangle
// (v1 -> (0,0), v2 -> (1,0), v3 -> (0,1)).  Written as constexpr functions so
// that evaluations at the fixed quadrature points fold to constants.
// ------------------------------------------------------------------------
__host__ __device__ constexpr double psi(int l, double x, double y) {
  return l == 0 ? 1.0
       : l == 1 ? 4.0 * x + 2.0 * y - 2.0
       : l == 2 ? 3.0 * y - 1.0
       : l == 3 ? 24.0 * x * x + 24.0 * x * y + 4.0 * y * y - 24.0 * x - 8.0 * y + 4.0
       : l == 4 ? 20.0 * x * y + 10.0 * y * y - 4.0 * x - 12.0 * y + 2.0
                : 10.0 * y * y - 8.0 * y + 1.0;
}
__host__ __device__ constexpr double psi_x(int l, double x, double y) {   // d/dxi
  return l == 0 ? 0.0 : l == 1 ? 4.0 : l == 2 ? 0.0 : l == 3 ? 48.0 * x + 24.0 * y - 24.0
       : l == 4 ? 20.0 * y - 4.0 : 0.0;
}
__host__ __device__ constexpr double psi_y(int l, double x, double y) {   // d/deta
  return l == 0 ? 0.0 : l == 1 ? 2.0 : l == 2 ? 3.0 : l == 3 ? 24.0 * x + 8.0 * y - 8.0
       : l == 4 ? 20.0 * x + 20.0 * y - 12.0 : 20.0 * y - 8.0;
}
// the same basis evaluated in the arithmetic of T at run-time points
template <typename T>
__device__ __forceinline__ T psi_t(int l, T x, T y) {
  // nested forms with explicit fmas (see fdot2)
  return l == 0 ? T(1)
       : l == 1 ? fma(T(4), x, fma(T(2), y, T(-2)))
       : l == 2 ? fma(T(3), y, T(-1))
       : l == 3 ? fma(x, fma(T(24), x, fma(T(24), y, T(-24))), fma(y, fma(T(4), y, T(-8)), T(4)))
       : l == 4 ? fma(x, fma(T(20), y, T(-4)), fma(y, fma(T(10), y, T(-12)), T(2)))
                : fma(y, fma(T(10), y, T(-8)), T(1));
}
// second reference derivatives: r = 0 (xi xi), 1 (xi eta), 2 (eta eta)
__host__ __device__ constexpr double psi_2(int l, int r) {
  return l == 3 ? (r == 0 ? 48.0 : r == 1 ? 24.0 : 8.0)
       : l == 4 ? (r == 0 ? 0.0 : 20.0)
       : l == 5 ? (r == 2 ? 20.0 : 0.0) : 0.0;
}
// mass a_K^(l) = c_l |K| of the orthogonal basis
__host__ __device__ constexpr double mass_c(int l) {
  return l == 0 ? 1.0 : l == 1 ? 2.0 / 3.0 : l == 2 ? 0.5 : l == 3 ? 16.0 / 15.0 : l == 4 ? 4.0 / 9.0 : 1.0 / 3.0;
}
// 1 / c_l (exact in binary)
__host__ __device__ constexpr double inv_mass_c(int l) {
  return l == 0 ? 1.0 : l == 1 ? 1.5 : l == 2 ? 2.0 : l == 3 ? 0.9375 : l == 4 ? 2.25 : 3.0;
}
__host__ __device__ constexpr int degree_of(int l) { return l == 0 ? 0 : (l <= 2 ? 1 : 2); }

// Gauss-Legendre nodes of Appendix B mapped to s in (0, 1), weights summing to 1.
__host__ __device__ constexpr double gauss_s(int Q, int nu) {
  return Q == 2 ? (nu == 0 ? 0.21132486540518713 : 0.78867513459481287)
                : (nu == 0 ? 0.11270166537925831 : nu == 1 ? 0.5 : 0.88729833462074169);
}
__host__ __device__ constexpr double gauss_w(int Q, int nu) {
  return Q == 2 ? 0.5 : (nu == 1 ? 8.0 / 18.0 : 5.0 / 18.0);
}
// edge i is opposite vertex i, run from vertex i+1 to vertex i+2 (counter-clockwise)
__host__ __device__ constexpr double edge_xi(int i, double s) { return i == 0 ? 1.0 - s : i == 1 ? 0.0 : s; }
__host__ __device__ constexpr double edge_eta(int i, double s) { return i == 0 ? s : i == 1 ? 1.0 - s : 0.0; }
__host__ __device__ constexpr double vert_xi(int v) { return v == 1 ? 1.0 : 0.0; }
__host__ __device__ constexpr double vert_eta(int v) { return v == 2 ? 1.0 : 0.0; }

// Volume rules of Appendix A (tab:2th for N = 3, tab:4th for N = 6); (xi, eta) = (b2, b3).
__host__ __device__ constexpr double vol_xi(int N, int mu) {
  return N == 3 ? (mu == 0 ? 1.0 / 6.0 : mu == 1 ? 2.0 / 3.0 : 1.0 / 6.0)
       : (mu == 0 ? 0.445948490915965 : mu == 1 ? 0.108103018168070 : mu == 2 ? 0.445948490915965
          : mu == 3 ? 0.091576213509771 : mu == 4 ? 0.816847572980458 : 0.091576213509771);
}
__host__ __device__ constexpr double vol_eta(int N, int mu) {
  return N == 3 ? (mu == 0 ? 2.0 / 3.0 : mu == 1 ? 1.0 / 6.0 : 1.0 / 6.0)
       : (mu == 0 ? 0.108103018168070 : mu == 1 ? 0.445948490915965 : mu == 2 ? 0.445948490915965
          : mu == 3 ? 0.816847572980458 : mu == 4 ? 0.091576213509771 : 0.091576213509771);
}
__host__ __device__ constexpr double vol_w(int N, int mu) {
  return N == 3 ? 1.0 / 3.0 : (mu < 3 ? 0.223381589678010 : 0.109951743655322);
}

// acc + c * x with a coefficient c known at compile time after unrolling:
// zero terms vanish and unit coefficients become additions.
template <typename T>
__device__ __forceinline__ T cfma(double c, T x, T acc) {
  if (c == 0.0) return acc;
  if (c == 1.0) return acc + x;
  if (c == -1.0) return acc - x;
  return fma(static_cast<T>(c), x, acc);
}

// ------------------------------------------------------------------------
// Euler physics (eq. euler, G:Euler)
// ------------------------------------------------------------------------
// a b + c d with the fused product fixed: c d rounds, a b fuses into the
// sum.  Left to the compiler, which product of a two-product sum is fused
// depends on the surrounding code, so the same source inlined into two
// kernels could round differently; every such sum on the shared stage paths
// is written with fdot2 (or an explicit fma) so that all kernels agree bit
// for bit.
template <typename T>
__device__ __forceinline__ T fdot2(T a, T b, T c, T d) { return fma(a, b, c * d); }

// F(u) . d for any direction d (not necessarily unit); returns pressure.
template <typename T>
__device__ __forceinline__ T flux_dir(const T u[4], T dx, T dy, T gm1, T f[4]) {
  const T ri = T(1) / u[0];
  const T p = gm1 * fma(T(-0.5) * fdot2(u[1], u[1], u[2], u[2]), ri, u[3]);
  const T md = fdot2(u[1], dx, u[2], dy);
  const T vd = md * ri;
  f[0] = md;
  f[1] = fma(u[1], vd, p * dx);
  f[2] = fma(u[2], vd, p * dy);
  f[3] = (u[3] + p) * vd;
  return p;
}

// F(u) . d1 and F(u) . d2 with one reciprocal of the density
template <typename T>
__device__ __forceinline__ void flux_dir2(const T u[4], T d1x, T d1y, T d2x, T d2y, T gm1, T f1[4], T f2[4]) {
  const T ri = T(1) / u[0];
  const T p = gm1 * fma(T(-0.5) * fdot2(u[1], u[1], u[2], u[2]), ri, u[3]);
  const T ep = u[3] + p;
  const T m1 = fdot2(u[1], d1x, u[2], d1y), v1 = m1 * ri;
  const T m2 = fdot2(u[1], d2x, u[2], d2y), v2 = m2 * ri;
  f1[0] = m1; f1[1] = fma(u[1], v1, p * d1x); f1[2] = fma(u[2], v1, p * d1y); f1[3] = ep * v1;
  f2[0] = m2; f2[1] = fma(u[1], v2, p * d2x); f2[2] = fma(u[2], v2, p * d2y); f2[3] = ep * v2;
}

// x > 0 on the integer units for doubles (differs from the comparison only
// for a NaN with a clear sign bit); a plain comparison for floats
__device__ __forceinline__ bool gt0(double x) { return __double_as_longlong(x) > 0; }
__device__ __forceinline__ bool gt0(float x) { return x > 0.0f; }
// exp(-x), x >= 0 (or NaN): small FP64 arguments, the usual case of the OE
// damping away from discontinuities, take a 7-FMA Taylor polynomial
// (dg_math.h); the rest the library exp; FP32 the fast intrinsic, whose
// error (a few ulp) is far below the mixed form's FP32 arithmetic error
__device__ __forceinline__ double exp_neg(double x) { return x <= EXP_NEG_SMALL_MAX ? exp_neg_small(x) : exp(-x); }
__device__ __forceinline__ float exp_neg(float x) { return __expf(-x); }

// x != 0 on the integer units (true for NaN, false for +0 and -0, as the comparison)
__device__ __forceinline__ bool nonzero_bits(double x) { return (__double_as_longlong(x) << 1) != 0; }
__device__ __forceinline__ bool nonzero_bits(float x) { return (__float_as_int(x) << 1) != 0; }

// F(u) . n and the spectral radius |v.n| + c (+inf for rho <= 0) with one reciprocal
template <typename T>
__device__ __forceinline__ T flux_speed_ri(const T u[4], T ri, T nx, T ny, T gm1, T gamma, T f[4]) {
  const T p = gm1 * fma(T(-0.5) * fdot2(u[1], u[1], u[2], u[2]), ri, u[3]);
  const T mn = fdot2(u[1], nx, u[2], ny);
  const T vn = mn * ri;
  f[0] = mn;
  f[1] = fma(u[1], vn, p * nx);
  f[2] = fma(u[2], vn, p * ny);
  f[3] = (u[3] + p) * vn;
  if (!gt0(u[0])) return T(INFINITY);
  const T pc = gt0(p) ? p : T(0);
  return fabs(vn) + sqrt(gamma * pc * ri);
}
template <typename T>
__device__ __forceinline__ T flux_speed(const T u[4], T nx, T ny, T gm1, T gamma, T f[4]) {
  return flux_speed_ri(u, T(1) / u[0], nx, ny, gm1, gamma, f);
}

// 1 / x[p] for n values from one division (Montgomery's batch inversion:
// prefix products, one reciprocal, back-substitution with two multiplies
// per value; each result within about 2n roundings of 1 / x[p]).  If a prefix product is not a normal number (a
// zero, a non-finite or an extreme value) every value is divided instead.
template <int n>
__device__ __forceinline__ void batch_reciprocal(const double x[n], double r[n]) {
  double c[n];
  c[0] = x[0];
  unsigned bad = 0;
#pragma unroll
  for (int p = 0; p < n; ++p) {
    if (p > 0) c[p] = c[p - 1] * x[p];
    const unsigned ex = unsigned(__double_as_longlong(c[p]) >> 52) & 0x7ffu;
    bad |= (ex == 0u) | (ex == 0x7ffu);
  }
  if (bad) {
#pragma unroll
    for (int p = 0; p < n; ++p) r[p] = 1.0 / x[p];
    return;
  }
  double inv = 1.0 / c[n - 1];
#pragma unroll
  for (int p = n - 1; p > 0; --p) {
    r[p] = inv * c[p - 1];
    inv = inv * x[p];
  }
  r[0] = inv;
}

// spectral radius |v.n| + c; +inf for rho <= 0, pressure clamped at 0
template <typename T>
__device__ __forceinline__ T wave_speed(const T u[4], T nx, T ny, T gamma) {
  if (!gt0(u[0])) return T(INFINITY);
  const T ri = T(1) / u[0];
  T p = (gamma - T(1)) * fma(T(-0.5) * fdot2(u[1], u[1], u[2], u[2]), ri, u[3]);
  p = gt0(p) ? p : T(0);
  return fma(fabs(fdot2(u[1], nx, u[2], ny)), ri, sqrt(gamma * p * ri));
}

__device__ __forceinline__ double int_energy(const double u[4]) {
  return u[3] - 0.5 * fdot2(u[1], u[1], u[2], u[2]) / u[0];
}

// exterior state of a boundary edge (tag > 0) at physical point (px, py),
// time t, from the interior trace um and the cell average avg
template <typename T>
__device__ __forceinline__ void ghost_state(int tag, const T um[4], const T avg[4], T nx, T ny, double px,
                                            double py, double t, const Phys &ph, T up[4]) {
  if (tag == 1) {                       // reflecting wall: m - 2 (m . n) n, the fused product fixed
    const T mn2 = T(-2) * fdot2(um[1], nx, um[2], ny);
    up[0] = um[0];
    up[1] = fma(mn2, nx, um[1]);
    up[2] = fma(mn2, ny, um[2]);
    up[3] = um[3];
  } else if (tag >= 3 && tag <= 6) {    // constant state
#pragma unroll
    for (int c = 0; c < 4; ++c) up[c] = T(ph.bc[tag - 3][c]);
  } else if (tag == 7) {                // moving shock
    const double xs = fma(py, ph.shock_cot, fma(t, ph.shock_vx, ph.shock_x0));
    const int s = px < xs ? ph.shock_post : ph.shock_pre;
#pragma unroll
    for (int c = 0; c < 4; ++c) up[c] = T(ph.bc[s][c]);
  } else {                              // transmissive: the cell average (a constant state)
#pragma unroll
    for (int c = 0; c < 4; ++c) up[c] = avg[c];
  }
}

// ------------------------------------------------------------------------
// Deterministic block reductions
// ------------------------------------------------------------------------
// Maximum of two non-negative doubles (or +inf, or NaN) on the integer units:
// for x, y >= +0 the IEEE bit patterns order like the numbers, and a NaN of
// either sign compares above every number, so it propagates.  A double
// comparison would occupy GB300's narrow FP64 pipe.
__device__ __forceinline__ double max_nn(double a, double b) {
  const unsigned long long x = (unsigned long long)__double_as_longlong(a);
  const unsigned long long y = (unsigned long long)__double_as_longlong(b);
  return __longlong_as_double((long long)(x > y ? x : y));
}
__device__ __forceinline__ float max_nn(float a, float b) { return (a > b || a != a) ? a : b; }

// x is neither infinite nor NaN, tested on the integer units
__device__ __forceinline__ bool is_finite_bits(double x) {
  return (__double_as_longlong(x) & 0x7ff0000000000000LL) != 0x7ff0000000000000LL;
}
__device__ __forceinline__ bool is_finite_bits(float x) {
  return (__float_as_int(x) & 0x7f800000) != 0x7f800000;
}

// Order-preserving integer key of a double (NaN aside): negative numbers get
// their magnitude bits flipped, so signed integer comparison orders the keys
// like the numbers (-0 sorts just below +0).  The map is its own inverse.
__device__ __forceinline__ long long ord_key(double x) {
  const long long b = __double_as_longlong(x);
  return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}
__device__ __forceinline__ double ord_val(long long k) {
  return __longlong_as_double(k ^ ((k >> 63) & 0x7fffffffffffffffLL));
}

struct OpSum {
  template <typename T> __device__ T operator()(T a, T b) const { return a + b; }
  template <typename T> __device__ static T ident() { return T(0); }
};
// NaN-propagating maximum of non-negative values
struct OpMaxNN {
  template <typename T> __device__ T operator()(T a, T b) const { return max_nn(a, b); }
  template <typename T> __device__ static T ident() { return T(0); }
};

constexpr int pow2_ceil(int n) { return n <= 1 ? 1 : 2 * pow2_ceil((n + 1) / 2); }

// Warp reduction of N values per lane by transposition: at each of the first
// log2(P) shuffle levels (P = N rounded up to a power of two) a lane keeps half
// of its values and adds the partner's copies of them, so the level costs half
// as many operations as the one before; the remaining levels are a butterfly on
// one value.  Component q ends on lanes q * 32 / P (and their butterfly
// partners).  The tree is fixed, so the result is reproducible.
template <int N, typename T, typename Op>
__device__ __forceinline__ T warp_reduce_transposed(const T v[N], Op op) {
  constexpr int P = pow2_ceil(N);
  static_assert(P <= 32, "too many values for one warp");
  const int lane = threadIdx.x & 31;
  T w[P];
#pragma unroll
  for (int q = 0; q < P; ++q) w[q] = q < N ? v[q] : Op::template ident<T>();
  int o = 16;
#pragma unroll
  for (int cnt = P; cnt > 1; cnt >>= 1, o >>= 1) {
    const int half = cnt >> 1;
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int j = 0; j < half; ++j) {
      const T send = up ? w[j] : w[j + half];
      const T keep = up ? w[j + half] : w[j];
      w[j] = op(keep, __shfl_xor_sync(0xffffffffu, send, o));
    }
  }
#pragma unroll
  for (; o > 0; o >>= 1) w[0] = op(w[0], __shfl_xor_sync(0xffffffffu, w[0], o));
  return w[0];
}

// Block reduction: transposed warp reduction, then the warps in order.  Ends
// with a barrier, so the block may call it again at once.
template <int N, typename T, typename U, typename Op>
__device__ __forceinline__ void block_reduce(const T v[N], U *out, Op op) {
  constexpr int P = pow2_ceil(N);
  __shared__ T red[TPB / 32][N > 0 ? N : 1];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const T r = warp_reduce_transposed<N, T, Op>(v, op);
  if (lane % (32 / P) == 0 && lane / (32 / P) < N) red[warp][lane / (32 / P)] = r;
  __syncthreads();
  if (threadIdx.x < N) {
    T s = red[0][threadIdx.x];
#pragma unroll
    for (int w = 1; w < TPB / 32; ++w) s = op(s, red[w][threadIdx.x]);
    out[threadIdx.x] = U(s);
  }
  __syncthreads();
}

// Fixed-order reduction of nblk partials of N values by one block: FIN_THREADS
// virtual lanes each reduce a strided subset, then a fixed tree.  The
// arithmetic does not depend on the block size, so a persistent kernel with
// TPB threads reproduces the FIN_THREADS-thread finalize kernels bitwise.  The
// strided loop loads four partials ahead of the operations, in the same order.
// Shared scratch of fin_reduce: one array per kernel, whatever the value type
// and count, so a kernel that reduces several kinds of partials stays within
// the static shared-memory limit.
__device__ __forceinline__ unsigned char *fin_scratch() {
  __shared__ __align__(16) unsigned char buf[FIN_THREADS * 5 * sizeof(double)];
  return buf;
}

template <int N, typename T, typename Op>
__device__ void fin_reduce(const T *part, int nblk, T init, Op op, T out[N]) {
  static_assert(N * sizeof(T) <= 5 * sizeof(double), "fin_scratch too small");
  T (*sh)[N] = reinterpret_cast<T (*)[N]>(fin_scratch());
  for (int vt = threadIdx.x; vt < FIN_THREADS; vt += blockDim.x) {
    T acc[N];
#pragma unroll
    for (int q = 0; q < N; ++q) acc[q] = init;
    int b = vt;
    for (; b + 3 * FIN_THREADS < nblk; b += 4 * FIN_THREADS) {
      T x[4][N];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int q = 0; q < N; ++q) x[u][q] = part[(int64_t)(b + u * FIN_THREADS) * N + q];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int q = 0; q < N; ++q) acc[q] = op(acc[q], x[u][q]);
    }
    for (; b < nblk; b += FIN_THREADS)
#pragma unroll
      for (int q = 0; q < N; ++q) acc[q] = op(acc[q], part[(int64_t)b * N + q]);
#pragma unroll
    for (int q = 0; q < N; ++q) sh[vt][q] = acc[q];
  }
  __syncthreads();
  for (int st = FIN_THREADS / 2; st > 0; st >>= 1) {
    for (int vt = threadIdx.x; vt < st; vt += blockDim.x)
#pragma unroll
      for (int q = 0; q < N; ++q) sh[vt][q] = op(sh[vt][q], sh[vt + st][q]);
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < N; ++q) out[q] = sh[0][q];
  __syncthreads();
}

// ------------------------------------------------------------------------
// Per-solve finalize steps (one block; thread 0 writes the scalars)
// ------------------------------------------------------------------------
// 1 / D_q of the damped quantities from sc->dev and sc->mean (eqs.
// OEScalar:Coef2, RIOESys:Coef1/Coef2 with the round-off guard of Sec. 2.3:
// a component whose deviation is below 1e-12 max(1, |mean|) is constant)
__device__ __forceinline__ void write_inv_normalisers(Scalars *sc, int cw) {
  const double eps = 1e-12;
  auto inv = [&](double D, double ref) { return D <= eps * fmax(1.0, ref) ? 0.0 : 1.0 / D; };
  sc->invD[0] = inv(sc->dev[0], fabs(sc->mean[0]));
  sc->invD[3] = inv(sc->dev[2], fabs(sc->mean[3]));
  if (cw) {
    sc->invD[1] = inv(sc->dev[3], fabs(sc->mean[1]));
    sc->invD[2] = inv(sc->dev[4], fabs(sc->mean[2]));
  } else {
    const double mnorm = sqrt(fdot2(sc->mean[1], sc->mean[1], sc->mean[2], sc->mean[2]));
    sc->invD[1] = sc->invD[2] = inv(sc->dev[1], mnorm);
  }
  for (int q = 0; q < 4; ++q) sc->invDf[q] = float(sc->invD[q]);
}

// ------------------------------------------------------------------------
// Finalisation inside the producing kernel, in a fixed order
// ------------------------------------------------------------------------
// The tiles of a reduction (TPB cells each, one partial per tile) form groups
// of TILE_GROUP consecutive tiles.  After writing its partial, a block takes a
// ticket for its group; the block that takes the group's last ticket reduces
// the group's partials with block_reduce and takes a ticket at the top level;
// the block that takes the last top-level ticket reduces the group results in
// chunks of TPB, in order, and writes the scalars.  The arithmetic depends only
// on the number of tiles, not on which block finishes when, so results are
// reproducible and the same in the per-solve kernels and the batch kernel.
// Every ticket counter is reset by the block that takes its last ticket, so it
// is zero again when the next launch (or batch phase) starts.
constexpr int TILE_GROUP = TPB;
__host__ __device__ __forceinline__ int64_t num_groups(int64_t ntiles) {
  return (ntiles + TILE_GROUP - 1) / TILE_GROUP;
}
// ticket counters of one reduction: one per group, then the top level
__host__ __device__ __forceinline__ int64_t ticket_slots(int64_t ntiles) { return num_groups(ntiles) + 1; }

// Called by every thread of the block once the block's results are written:
// true in the block that took the last of `total` tickets of *cnt.
// The block's writes are ordered before the ticket by the barrier and one
// device-scope fence of thread 0 (cumulative over what the barrier ordered);
// the last block fences again before its threads read the other blocks'
// results.
__device__ __forceinline__ bool take_ticket(unsigned *cnt, unsigned total) {
  __shared__ int s_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned t = atomicAdd(cnt, 1u);
    const int last = t + 1 == total;
    if (last) {
      atomicExch(cnt, 0u);               // every ticket is taken: reset for the next launch
      __threadfence();
    }
    s_last = last;
  }
  __syncthreads();
  const bool last = s_last != 0;
  __syncthreads();                       // s_last may be rewritten by the next call
  return last;
}

// partials of other blocks are read from L2 (L1 is not coherent across SMs)
__device__ __forceinline__ double ld_l2(const double *p) { return __ldcg(p); }
__device__ __forceinline__ long long ld_l2(const long long *p) { return __ldcg(p); }

// group g's partials -> grp[g]
template <int N, typename T, typename Op>
__device__ __forceinline__ void reduce_group(const T *part, int64_t g, int64_t ntiles, T *grp, Op op) {
  const int64_t t0 = g * TILE_GROUP;
  const int64_t n = ntiles - t0 < TILE_GROUP ? ntiles - t0 : TILE_GROUP;
  T v[N];
#pragma unroll
  for (int q = 0; q < N; ++q)
    v[q] = threadIdx.x < n ? ld_l2(part + (t0 + threadIdx.x) * N + q) : Op::template ident<T>();
  block_reduce<N>(v, grp + g * N, op);
}

// all group results, in chunks of TPB -> out[] in every thread
template <int N, typename T, typename Op>
__device__ __forceinline__ void reduce_top(const T *grp, int64_t ng, Op op, T out[N]) {
  __shared__ T res[N];
#pragma unroll
  for (int q = 0; q < N; ++q) out[q] = Op::template ident<T>();
  for (int64_t c0 = 0; c0 < ng; c0 += TPB) {
    T v[N];
#pragma unroll
    for (int q = 0; q < N; ++q)
      v[q] = c0 + threadIdx.x < ng ? ld_l2(grp + (c0 + threadIdx.x) * N + q) : Op::template ident<T>();
    block_reduce<N>(v, res, op);
#pragma unroll
    for (int q = 0; q < N; ++q) out[q] = op(out[q], res[q]);
    __syncthreads();
  }
}

// scratch of the in-kernel finalisation of one solve
struct FinBufs {
  double *grp_sum, *grp_dev, *grp_alpha;   // [ng][4], [ng][5], [ng]
  long long *grp_cnt;                      // [ng][2]
  unsigned *tick;                          // 3 reductions x ticket_slots(ntiles)
};

// Top level of each finalisation: the block that takes the last top-level
// ticket reduces the group results and writes the scalars.  The three kinds
// use consecutive ranges of ticket_slots(ntiles) counters.
__device__ __forceinline__ void finish_means_top(const FinBufs &f, int64_t ntiles, Scalars *sc) {
  const int64_t ng = num_groups(ntiles);
  if (!take_ticket(f.tick + ng, (unsigned)ng)) return;
  double r[4];
  reduce_top<4>(f.grp_sum, ng, OpSum(), r);
  if (threadIdx.x == 0)
    for (int c = 0; c < 4; ++c) sc->mean[c] = r[c] / sc->area_total;
}

__device__ __forceinline__ void finish_deviations_top(const FinBufs &f, int64_t ntiles, Scalars *sc, int cw) {
  const int64_t ng = num_groups(ntiles);
  if (!take_ticket(f.tick + ticket_slots(ntiles) + ng, (unsigned)ng)) return;
  double r[5];
  reduce_top<5>(f.grp_dev, ng, OpMaxNN(), r);
  if (threadIdx.x == 0) {
    for (int q = 0; q < 5; ++q) sc->dev[q] = r[q];
    write_inv_normalisers(sc, cw);
  }
}

// alpha of the next stage input, counters, and after the last stage t += dt
// (stage < 0: outside a step, alpha and counters only)
__device__ __forceinline__ void finish_alpha_top(const FinBufs &f, int64_t ntiles, Scalars *sc, int stage) {
  const int64_t ng = num_groups(ntiles);
  if (!take_ticket(f.tick + 2 * ticket_slots(ntiles) + ng, (unsigned)ng)) return;
  double a[1];
  long long c[2];
  reduce_top<1>(f.grp_alpha, ng, OpMaxNN(), a);
  reduce_top<2>(f.grp_cnt, ng, OpSum(), c);
  if (threadIdx.x == 0) {
    sc->alpha = a[0];
    sc->limited += c[0];
    sc->nonphys += c[1];
    if (stage == 0 || stage == 1) {
      if (a[0] * sc->dt > sc->min_ca * (1.0 + 1e-12)) sc->breaches += 1;
    } else if (stage == 2) {
      sc->t = sc->pad ? sc->t_end : sc->t + sc->dt;
      sc->steps += 1;
    }
  }
}

// Group level.  In the per-solve finalize kernels block g reduces group g
// directly; in the batch kernel the block that finishes a group's last tile
// does (after a group ticket), so both produce the same group results.
__device__ __forceinline__ bool group_ticket(const FinBufs &f, int kind, int64_t tile, int64_t ntiles) {
  const int64_t g = tile / TILE_GROUP;
  return take_ticket(f.tick + kind * ticket_slots(ntiles) + g,
                     (unsigned)min((int64_t)TILE_GROUP, ntiles - g * TILE_GROUP));
}

// in-kernel finalisation after tile `tile` wrote its partials (batch kernel)
__device__ __forceinline__ void finish_means(const double *part_sum, const FinBufs &f, int64_t tile, int64_t ntiles,
                                             Scalars *sc) {
  if (!group_ticket(f, 0, tile, ntiles)) return;
  reduce_group<4>(part_sum, tile / TILE_GROUP, ntiles, f.grp_sum, OpSum());
  finish_means_top(f, ntiles, sc);
}
__device__ __forceinline__ void finish_deviations(const double *part_dev, const FinBufs &f, int64_t tile,
                                                  int64_t ntiles, Scalars *sc, int cw) {
  if (!group_ticket(f, 1, tile, ntiles)) return;
  reduce_group<5>(part_dev, tile / TILE_GROUP, ntiles, f.grp_dev, OpMaxNN());
  finish_deviations_top(f, ntiles, sc, cw);
}
__device__ __forceinline__ void finish_alpha(const double *part_alpha, const long long *part_cnt, const FinBufs &f,
                                             int64_t tile, int64_t ntiles, Scalars *sc, int stage) {
  if (!group_ticket(f, 2, tile, ntiles)) return;
  reduce_group<1>(part_alpha, tile / TILE_GROUP, ntiles, f.grp_alpha, OpMaxNN());
  reduce_group<2>(part_cnt, tile / TILE_GROUP, ntiles, f.grp_cnt, OpSum());
  finish_alpha_top(f, ntiles, sc, stage);
}

// dt of the BP CFL condition (Sec. 5), clamped to t_end; inactive once t >= t_end
__device__ __forceinline__ void step_begin_thread(Scalars *sc) {
  if (sc->t < sc->t_end) {
    double dt = sc->cfl * sc->min_ca / sc->alpha;
    int clamped = 0;
    if (sc->t + dt >= sc->t_end) { dt = sc->t_end - sc->t; clamped = 1; }
    sc->dt = dt;
    sc->pad = clamped;
    sc->active = 1;
  } else {
    sc->dt = 0.0;
    sc->active = 0;
  }
}

// Deviation from the average of the extra limiter point(s) of the classical
// decomposition, from the deviations at the edge Gauss points (the first 3Q
// rows of d): P1 has no internal term (its edge weights sum to one), so the
// edge point 0 is repeated; P2 takes the weighted internal state u_* of
// Sec. 4.1 with edge weights 1/9: u_* - ubar = -(1/9) sum w_nu dev / (1 - 3/9).
template <int K, typename T, int ROWS>
__device__ __forceinline__ void zxs_extra_points(T d[ROWS][4]) {
  constexpr int NQ = K + 1, NE = 3 * NQ;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    T v;
    if (K == 1) {
      v = d[0][c];
    } else {
      T acc = T(0);
#pragma unroll
      for (int p = 0; p < NE; ++p) acc += T(gauss_w(NQ, p % NQ)) * d[p][c];
      v = T(-1.0 / 6.0) * acc;
    }
    d[NE][c] = v;
    d[NE + 1][c] = v;
  }
}

}  // namespace dg

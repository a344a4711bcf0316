// dg_api.cu -- host implementation of the C ABI declared in include/dg.h:
// mesh construction (adjacency on the host, geometry on the GPU), the solver
// (device buffers, one SSP-RK3 step captured as a CUDA graph) and the single
// stage operators.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/dg.h"
#include "dg_internal.h"
#include "dg_mesh_host.h"

using namespace dg;

namespace {

thread_local std::string g_err;

int32_t fail(int32_t code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

#define CUDA_TRY(expr)                                                                          \
  do {                                                                                          \
    cudaError_t e_ = (expr);                                                                    \
    if (e_ != cudaSuccess) return fail(DG_ECUDA, "%s: %s (%s:%d)", #expr, cudaGetErrorString(e_), \
                                       __FILE__, __LINE__);                                    \
  } while (0)

template <typename T>
cudaError_t dalloc(T **p, size_t n) {
  *p = nullptr;
  if (n == 0) n = 1;
  return cudaMalloc((void **)p, n * sizeof(T));
}

}  // namespace

struct dg_mesh {
  int64_t nv = 0, nt = 0;
  std::vector<int32_t> nbr, nbr_edge;   // host adjacency
  std::vector<double> quad_xy;          // lazily built 12-point rule points
  std::vector<double> vxy_host;         // [6][nt]
  std::vector<int8_t> bnd_tag;          // [3 nt] tag of each boundary edge (0 for interior edges)
  // device
  double *area = nullptr, *jinv = nullptr, *nrm = nullptr, *len = nullptr, *vxy = nullptr, *node = nullptr,
         *c_area = nullptr, *hgeo = nullptr;
  int8_t *limv = nullptr;
  int32_t *conn = nullptr;
  int64_t ne = 0;
  int32_t *e_cell = nullptr, *etile = nullptr, *cedge = nullptr;
  int8_t *e_loc = nullptr;
  float *jinv_f = nullptr, *nrm_f = nullptr, *len_f = nullptr, *hgeo_f = nullptr;
  double *iarea = nullptr;
  float *node_f = nullptr;
  double *psi_node = nullptr;
  double min_ca[4] = {0, 0, 0, 0};   // (P1 optimal, P1 ZXS, P2 optimal, P2 ZXS)
  double area_total = 0.0;
  int device = 0;                    // the CUDA device that holds the mesh's arrays
  ~dg_mesh() {
    cudaFree(area); cudaFree(jinv); cudaFree(nrm); cudaFree(len); cudaFree(vxy); cudaFree(node);
    cudaFree(c_area); cudaFree(limv); cudaFree(conn); cudaFree(hgeo);
    cudaFree(e_cell); cudaFree(e_loc); cudaFree(etile); cudaFree(cedge);
    cudaFree(jinv_f); cudaFree(nrm_f); cudaFree(len_f); cudaFree(hgeo_f); cudaFree(iarea); cudaFree(node_f);
    cudaFree(psi_node);
  }
};

struct dg_solver {
  const dg_mesh *mesh = nullptr;
  dg_config cfg{};
  int nb = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  StateBuf un{}, uh{}, us{};
  void *tr = nullptr, *vd = nullptr, *hs = nullptr, *ej = nullptr;
  double *part_sum = nullptr, *part_dev = nullptr, *part_alpha = nullptr;
  long long *part_cnt = nullptr;
  FinBufs fin{};
  Scalars *sc = nullptr;
  cudaGraphExec_t step_exec = nullptr;
  StageCtx ctx{};
  ~dg_solver() {
    if (step_exec) cudaGraphExecDestroy(step_exec);
    StateBuf *bufs[3] = {&un, &uh, &us};
    for (auto *b : bufs) { cudaFree(b->avg); cudaFree(b->hi); }
    cudaFree(tr); cudaFree(vd); cudaFree(hs); cudaFree(ej);
    cudaFree(part_sum); cudaFree(part_dev); cudaFree(part_alpha); cudaFree(part_cnt); cudaFree(sc);
    cudaFree(fin.grp_sum); cudaFree(fin.grp_dev); cudaFree(fin.grp_alpha); cudaFree(fin.grp_cnt); cudaFree(fin.tick);
    if (own_stream && stream) cudaStreamDestroy(stream);
  }
};

extern "C" const char *dg_last_error(void) { return g_err.c_str(); }

namespace dg {
void mesh_view(const dg_mesh *mesh, int64_t *nt, const double **area, double *area_total) {
  *nt = mesh->nt;
  *area = mesh->area;
  *area_total = mesh->area_total;
}
int32_t set_error(int32_t code, const char *msg) { return fail(code, "%s", msg); }
int mesh_device(const dg_mesh *mesh) { return mesh->device; }
}  // namespace dg

// ============================================================================
// Mesh
// ============================================================================
extern "C" int32_t dg_mesh_create(int64_t nv, const double *xy, int64_t nt, const int32_t *tri, const int32_t *canon,
                                  const int8_t *bc, dg_mesh **out) {
  if (!out) return fail(DG_EINVAL, "out is NULL");
  *out = nullptr;
  HostMesh hm;
  std::string msg;
  const int32_t rc = build_host_mesh(nv, xy, nt, tri, canon, bc, TPB, hm, msg);
  if (rc != DG_OK) return fail(rc, "%s", msg.c_str());
  auto m = new (std::nothrow) dg_mesh();
  if (!m) return fail(DG_ENOMEM, "host allocation failed");
  m->nv = nv;
  m->nt = nt;
  if (cudaGetDevice(&m->device) != cudaSuccess) { delete m; return fail(DG_ECUDA, "no CUDA device"); }
  m->nbr = std::move(hm.nbr);
  m->nbr_edge = std::move(hm.nbr_edge);
  m->bnd_tag = std::move(hm.bnd_tag);
  m->vxy_host = std::move(hm.vxy);
  const std::vector<int32_t> &conn = hm.conn, &e_cell = hm.e_cell, &etile = hm.etile, &cedge = hm.cedge;
  const std::vector<int8_t> &e_loc = hm.e_loc;
  const int64_t ntiles = num_blocks(nt);
  if ((int64_t)etile.size() != ntiles + 1) { delete m; return fail(DG_EINVAL, "tile count mismatch"); }
  m->ne = (int64_t)e_cell.size();
  double *part = nullptr, *mins = nullptr;
  cudaError_t e = cudaSuccess;
#define MTRY(x)                                                                                         \
  if ((e = (x)) != cudaSuccess) {                                                                       \
    cudaFree(part); cudaFree(mins); delete m;                                                           \
    return fail(e == cudaErrorMemoryAllocation ? DG_ENOMEM : DG_ECUDA, "%s: %s", #x, cudaGetErrorString(e)); \
  }
  MTRY(dalloc(&m->area, nt));
  MTRY(dalloc(&m->jinv, 4 * nt));
  MTRY(dalloc(&m->nrm, 6 * nt));
  MTRY(dalloc(&m->len, 3 * nt));
  MTRY(dalloc(&m->hgeo, 6 * nt));
  MTRY(dalloc(&m->vxy, 6 * nt));
  MTRY(dalloc(&m->node, 4 * nt));
  MTRY(dalloc(&m->c_area, 4 * nt));
  MTRY(dalloc(&m->limv, 2 * nt));
  MTRY(dalloc(&m->conn, 3 * nt));
  MTRY(dalloc(&m->jinv_f, 4 * nt));
  MTRY(dalloc(&m->nrm_f, 6 * nt));
  MTRY(dalloc(&m->len_f, 3 * nt));
  MTRY(dalloc(&m->hgeo_f, 6 * nt));
  MTRY(dalloc(&m->iarea, nt));
  MTRY(dalloc(&m->node_f, 4 * nt));
  MTRY(dalloc(&m->psi_node, 10 * nt));
  MTRY(dalloc(&m->e_cell, m->ne));
  MTRY(dalloc(&m->e_loc, m->ne));
  MTRY(dalloc(&m->etile, ntiles + 1));
  MTRY(dalloc(&m->cedge, 3 * nt));
  MTRY(cudaMemcpy(m->e_cell, e_cell.data(), sizeof(int32_t) * m->ne, cudaMemcpyHostToDevice));
  MTRY(cudaMemcpy(m->e_loc, e_loc.data(), m->ne, cudaMemcpyHostToDevice));
  MTRY(cudaMemcpy(m->etile, etile.data(), sizeof(int32_t) * (ntiles + 1), cudaMemcpyHostToDevice));
  MTRY(cudaMemcpy(m->cedge, cedge.data(), sizeof(int32_t) * 3 * nt, cudaMemcpyHostToDevice));
  MTRY(dalloc(&part, 4 * num_blocks(nt)));
  MTRY(dalloc(&mins, 4));
  MTRY(cudaMemcpy(m->vxy, m->vxy_host.data(), sizeof(double) * 6 * nt, cudaMemcpyHostToDevice));
  MTRY(cudaMemcpy(m->conn, conn.data(), sizeof(int32_t) * 3 * nt, cudaMemcpyHostToDevice));
  GeomPtrs g{m->area,   m->jinv,  m->nrm,   m->len,    m->hgeo, m->node, m->c_area,
             m->limv,   m->jinv_f, m->nrm_f, m->len_f, m->hgeo_f, m->iarea, m->node_f, m->psi_node};
  launch_geometry(nullptr, nt, m->vxy, g, part, mins);
  MTRY(cudaGetLastError());
  MTRY(cudaMemcpy(m->min_ca, mins, sizeof(double) * 4, cudaMemcpyDeviceToHost));
  std::vector<double> area((size_t)nt);
  MTRY(cudaMemcpy(area.data(), m->area, sizeof(double) * nt, cudaMemcpyDeviceToHost));
#undef MTRY
  cudaFree(part);
  cudaFree(mins);
  double s = 0.0;
  for (int64_t K = 0; K < nt; ++K) s += area[K];
  m->area_total = s;
  *out = m;
  return DG_OK;
}

extern "C" void dg_mesh_destroy(dg_mesh *mesh) { delete mesh; }

extern "C" int32_t dg_mesh_info(const dg_mesh *m, int32_t decomp, int64_t *nt, double *p1, double *p2) {
  if (!m) return fail(DG_EINVAL, "mesh is NULL");
  if (nt) *nt = m->nt;
  const int z = decomp == DG_DECOMP_ZXS ? 1 : 0;
  if (p1) *p1 = m->min_ca[0 + z];
  if (p2) *p2 = m->min_ca[2 + z];
  return DG_OK;
}

extern "C" int32_t dg_mesh_neighbors(const dg_mesh *m, int32_t *nbr, int32_t *nbr_edge) {
  if (!m || !nbr || !nbr_edge) return fail(DG_EINVAL, "NULL argument");
  std::memcpy(nbr, m->nbr.data(), sizeof(int32_t) * 3 * m->nt);
  std::memcpy(nbr_edge, m->nbr_edge.data(), sizeof(int32_t) * 3 * m->nt);
  return DG_OK;
}

extern "C" int32_t dg_mesh_geometry(const dg_mesh *m, int32_t k, int32_t decomp, double *area, double *len,
                                    double *normal, double *c_area, double *nodes, int8_t *limv) {
  if (!m || (k != 1 && k != 2)) return fail(DG_EINVAL, "bad mesh or degree");
  const int64_t nt = m->nt;
  std::vector<double> buf((size_t)(6 * nt));
  if (area) CUDA_TRY(cudaMemcpy(area, m->area, sizeof(double) * nt, cudaMemcpyDeviceToHost));
  if (len) {
    CUDA_TRY(cudaMemcpy(buf.data(), m->len, sizeof(double) * 3 * nt, cudaMemcpyDeviceToHost));
    for (int64_t K = 0; K < nt; ++K)
      for (int i = 0; i < 3; ++i) len[3 * K + i] = buf[(size_t)i * nt + K];
  }
  if (normal) {
    CUDA_TRY(cudaMemcpy(buf.data(), m->nrm, sizeof(double) * 6 * nt, cudaMemcpyDeviceToHost));
    for (int64_t K = 0; K < nt; ++K)
      for (int q = 0; q < 6; ++q) normal[6 * K + q] = buf[(size_t)q * nt + K];
  }
  if (c_area) {
    const int q = (k - 1) * 2 + (decomp == DG_DECOMP_ZXS ? 1 : 0);
    CUDA_TRY(cudaMemcpy(c_area, m->c_area + (size_t)q * nt, sizeof(double) * nt, cudaMemcpyDeviceToHost));
  }
  if (nodes) {
    CUDA_TRY(cudaMemcpy(buf.data(), m->node, sizeof(double) * 4 * nt, cudaMemcpyDeviceToHost));
    for (int64_t K = 0; K < nt; ++K)
      for (int q = 0; q < 4; ++q) nodes[4 * K + q] = buf[(size_t)q * nt + K];
  }
  if (limv) {
    std::vector<int8_t> lb((size_t)(2 * nt));
    CUDA_TRY(cudaMemcpy(lb.data(), m->limv, 2 * nt, cudaMemcpyDeviceToHost));
    for (int64_t K = 0; K < nt; ++K) { limv[2 * K] = lb[K]; limv[2 * K + 1] = lb[nt + K]; }
  }
  return DG_OK;
}

// 12-point rule of Appendix A (Table tab:6th): barycentric coordinates and weights
static const double Q12_B[12][3] = {
    {0.063089014491502, 0.063089014491502, 0.873821971016996}, {0.063089014491502, 0.873821971016996, 0.063089014491502},
    {0.873821971016996, 0.063089014491502, 0.063089014491502}, {0.249286745170910, 0.249286745170910, 0.501426509658180},
    {0.249286745170910, 0.501426509658180, 0.249286745170910}, {0.501426509658180, 0.249286745170910, 0.249286745170910},
    {0.053145049844817, 0.636502499121399, 0.310352451033784}, {0.636502499121399, 0.053145049844817, 0.310352451033784},
    {0.053145049844817, 0.310352451033784, 0.636502499121399}, {0.636502499121399, 0.310352451033784, 0.053145049844817},
    {0.310352451033784, 0.053145049844817, 0.636502499121399}, {0.310352451033784, 0.636502499121399, 0.053145049844817}};
static const double Q12_W[12] = {0.050844906370207, 0.050844906370207, 0.050844906370207, 0.116786275726379,
                                 0.116786275726379, 0.116786275726379, 0.082851075618374, 0.082851075618374,
                                 0.082851075618374, 0.082851075618374, 0.082851075618374, 0.082851075618374};

extern "C" int32_t dg_quad_points(const dg_mesh *m, double *xy) {
  if (!m || !xy) return fail(DG_EINVAL, "NULL argument");
  const int64_t nt = m->nt;
  for (int64_t K = 0; K < nt; ++K)
    for (int mu = 0; mu < 12; ++mu) {
      double x = 0.0, y = 0.0;
      for (int v = 0; v < 3; ++v) {
        x += Q12_B[mu][v] * m->vxy_host[(size_t)(2 * v) * nt + K];
        y += Q12_B[mu][v] * m->vxy_host[(size_t)(2 * v + 1) * nt + K];
      }
      xy[(K * 12 + mu) * 2] = x;
      xy[(K * 12 + mu) * 2 + 1] = y;
    }
  return DG_OK;
}

extern "C" int32_t dg_project(const dg_mesh *m, int32_t k, const double *vals, double *coeffs) {
  if (!m || !vals || !coeffs || (k != 1 && k != 2)) return fail(DG_EINVAL, "bad argument");
  const int nb = k == 1 ? 3 : 6;
  const int64_t nt = m->nt;
  for (int64_t K = 0; K < nt; ++K) {
    double acc[4][6] = {};
    for (int mu = 0; mu < 12; ++mu) {
      const double xi = Q12_B[mu][1], eta = Q12_B[mu][2];
      for (int l = 0; l < nb; ++l) {
        const double w = Q12_W[mu] * psi(l, xi, eta) / mass_c(l);
        for (int c = 0; c < 4; ++c) acc[c][l] += w * vals[(K * 12 + mu) * 4 + c];
      }
    }
    for (int c = 0; c < 4; ++c)
      for (int l = 0; l < nb; ++l) coeffs[((int64_t)c * nb + l) * nt + K] = acc[c][l];
  }
  return DG_OK;
}

// ============================================================================
// Solver
// ============================================================================
namespace {

size_t real_size(const dg_solver *s) { return s->cfg.precision == DG_PREC_MIXED ? sizeof(float) : sizeof(double); }

cudaError_t alloc_state(dg_solver *s, StateBuf *b) {
  const int64_t nt = s->mesh->nt;
  cudaError_t e = dalloc(&b->avg, 4 * nt);
  if (e != cudaSuccess) return e;
  return cudaMalloc(&b->hi, std::max<size_t>(1, real_size(s) * 4 * (s->nb - 1) * nt));
}

// host modal state [4][nb][nt] (double) -> device buffer
int32_t upload_state(dg_solver *s, const double *coeffs, const StateBuf &b) {
  const int64_t nt = s->mesh->nt;
  const int nb = s->nb;
  for (int c = 0; c < 4; ++c)
    CUDA_TRY(cudaMemcpyAsync(b.avg + c * nt, coeffs + (int64_t)c * nb * nt, sizeof(double) * nt,
                             cudaMemcpyHostToDevice, s->stream));
  if (s->cfg.precision == DG_PREC_MIXED) {
    std::vector<float> tmp((size_t)(4 * (nb - 1) * nt));
    for (int c = 0; c < 4; ++c)
      for (int l = 1; l < nb; ++l)
        for (int64_t K = 0; K < nt; ++K)
          tmp[(size_t)K * 4 * (nb - 1) + c * (nb - 1) + (l - 1)] = (float)coeffs[((int64_t)c * nb + l) * nt + K];
    CUDA_TRY(cudaMemcpyAsync(b.hi, tmp.data(), sizeof(float) * tmp.size(), cudaMemcpyHostToDevice, s->stream));
    CUDA_TRY(cudaStreamSynchronize(s->stream));
  } else {
    for (int c = 0; c < 4; ++c)
      CUDA_TRY(cudaMemcpyAsync((double *)b.hi + (int64_t)c * (nb - 1) * nt, coeffs + ((int64_t)c * nb + 1) * nt,
                               sizeof(double) * (nb - 1) * nt, cudaMemcpyHostToDevice, s->stream));
  }
  return DG_OK;
}

int32_t download_state(const dg_solver *s, const StateBuf &b, double *coeffs) {
  const int64_t nt = s->mesh->nt;
  const int nb = s->nb;
  for (int c = 0; c < 4; ++c)
    CUDA_TRY(cudaMemcpyAsync(coeffs + (int64_t)c * nb * nt, b.avg + c * nt, sizeof(double) * nt,
                             cudaMemcpyDeviceToHost, s->stream));
  if (s->cfg.precision == DG_PREC_MIXED) {
    std::vector<float> tmp((size_t)(4 * (nb - 1) * nt));
    CUDA_TRY(cudaMemcpyAsync(tmp.data(), b.hi, sizeof(float) * tmp.size(), cudaMemcpyDeviceToHost, s->stream));
    CUDA_TRY(cudaStreamSynchronize(s->stream));
    for (int c = 0; c < 4; ++c)
      for (int l = 1; l < nb; ++l)
        for (int64_t K = 0; K < nt; ++K)
          coeffs[((int64_t)c * nb + l) * nt + K] = tmp[(size_t)K * 4 * (nb - 1) + c * (nb - 1) + (l - 1)];
  } else {
    for (int c = 0; c < 4; ++c)
      CUDA_TRY(cudaMemcpyAsync(coeffs + ((int64_t)c * nb + 1) * nt, (double *)b.hi + (int64_t)c * (nb - 1) * nt,
                               sizeof(double) * (nb - 1) * nt, cudaMemcpyDeviceToHost, s->stream));
  }
  CUDA_TRY(cudaStreamSynchronize(s->stream));
  return DG_OK;
}

int32_t read_scalars(const dg_solver *s, Scalars *h) {
  CUDA_TRY(cudaMemcpyAsync(h, s->sc, sizeof(Scalars), cudaMemcpyDeviceToHost, s->stream));
  CUDA_TRY(cudaStreamSynchronize(s->stream));
  return DG_OK;
}

int32_t write_scalars(dg_solver *s, const Scalars *h) {
  CUDA_TRY(cudaMemcpyAsync(s->sc, h, sizeof(Scalars), cudaMemcpyHostToDevice, s->stream));
  CUDA_TRY(cudaStreamSynchronize(s->stream));
  return DG_OK;
}

const double RK_A[3] = {0.0, 0.75, 1.0 / 3.0}, RK_B[3] = {1.0, 0.25, 2.0 / 3.0};
const double C_IN[3] = {0.0, 1.0, 0.5}, C_OUT[3] = {1.0, 0.5, 1.0};

// one SSP-RK3 step of the BP RI-OEDG scheme (Sec. 4.5) on the solver's stream
void enqueue_step(dg_solver *s) {
  const StageCtx &c = s->ctx;
  const int oe = s->cfg.oe != DG_OE_OFF, bp = s->cfg.bp != DG_BP_OFF;
  launch_step_begin(c);
  for (int st = 0; st < 3; ++st) {
    const StateBuf &v = st == 0 ? s->un : s->us;
    launch_rk(c, v, s->un, s->uh, RK_A[st], RK_B[st], C_IN[st]);
    if (oe) launch_stats(c, s->uh, C_OUT[st]);
    launch_oe_bp(c, s->uh, st == 2 ? s->un : s->us, oe, bp, C_OUT[st], st);
  }
}

}  // namespace

extern "C" int32_t dg_init(const dg_mesh *mesh, const dg_config *cfg, const double *coeffs, void *cuda_stream,
                           dg_solver **out) {
  if (!out) return fail(DG_EINVAL, "out is NULL");
  *out = nullptr;
  if (!mesh || !cfg || !coeffs) return fail(DG_EINVAL, "NULL argument");
  if (cfg->k != 1 && cfg->k != 2) return fail(DG_EINVAL, "k must be 1 or 2 (got %d)", cfg->k);
  if (cfg->precision != DG_PREC_FP64 && cfg->precision != DG_PREC_MIXED) return fail(DG_EINVAL, "bad precision");
  if (cfg->oe < 0 || cfg->oe > 2 || cfg->bp < 0 || cfg->bp > 1 || cfg->decomp < 0 || cfg->decomp > 1)
    return fail(DG_EINVAL, "bad oe / bp / decomp");
  if (!(cfg->gamma > 1.0) || !(cfg->cfl > 0.0)) return fail(DG_EINVAL, "gamma must be > 1 and cfl > 0");
  if (cfg->shock_pre < 0 || cfg->shock_pre > 3 || cfg->shock_post < 0 || cfg->shock_post > 3)
    return fail(DG_EINVAL, "bad shock state index");
  auto s = new (std::nothrow) dg_solver();
  if (!s) return fail(DG_ENOMEM, "host allocation failed");
  s->mesh = mesh;
  s->cfg = *cfg;
  s->nb = cfg->k == 1 ? 3 : 6;
  const int64_t nt = mesh->nt;
  const int nq = cfg->k + 1;
  const size_t rs = real_size(s);
  const int64_t nblk = num_blocks(nt);
  int32_t rc = DG_OK;
  cudaError_t e = cudaSuccess;
#define STRY(x)                                                                                          \
  if ((e = (x)) != cudaSuccess) {                                                                        \
    rc = fail(e == cudaErrorMemoryAllocation ? DG_ENOMEM : DG_ECUDA, "%s: %s", #x, cudaGetErrorString(e)); \
    delete s;                                                                                            \
    return rc;                                                                                           \
  }
  if (cuda_stream) {
    s->stream = (cudaStream_t)cuda_stream;
  } else {
    STRY(cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking));
    s->own_stream = true;
  }
  STRY(alloc_state(s, &s->un));
  STRY(alloc_state(s, &s->uh));
  STRY(alloc_state(s, &s->us));
  const int64_t xc = uses_exchange(cfg->precision) ? nt : 1;   // exchange buffers: FP64 form only
  STRY(cudaMalloc(&s->tr, rs * xc * 3 * nq * trace_stride(cfg->precision)));
  STRY(cudaMalloc(&s->vd, rs * xc * VD_CELL));
  STRY(cudaMalloc(&s->hs, rs * xc * 12));
  STRY(cudaMalloc(&s->ej, rs * (uses_exchange(cfg->precision) ? std::max<int64_t>(mesh->ne, 1) : 1) * EJ_STRIDE));
  STRY(dalloc(&s->part_sum, 4 * nblk));
  STRY(dalloc(&s->part_dev, 5 * nblk));
  STRY(dalloc(&s->part_alpha, nblk));
  STRY(dalloc(&s->part_cnt, 2 * nblk));
  const int64_t ngrp = num_groups(nblk);
  STRY(dalloc(&s->fin.grp_sum, 4 * ngrp));
  STRY(dalloc(&s->fin.grp_dev, 5 * ngrp));
  STRY(dalloc(&s->fin.grp_alpha, ngrp));
  STRY(dalloc(&s->fin.grp_cnt, 2 * ngrp));
  STRY(dalloc(&s->fin.tick, 3 * ticket_slots(nblk)));
  STRY(cudaMemsetAsync(s->fin.tick, 0, 3 * ticket_slots(nblk) * sizeof(unsigned), s->stream));   // tickets start at zero
  STRY(dalloc(&s->sc, 1));
  // context of every stage launch
  StageCtx &c = s->ctx;
  c.stream = s->stream;
  c.k = cfg->k;
  c.prec = cfg->precision;
  c.mesh = MeshDev{nt,         mesh->area, mesh->jinv,   mesh->nrm,   mesh->len,   mesh->vxy,  mesh->node,
                   mesh->hgeo, mesh->limv, mesh->conn,   mesh->ne,    mesh->e_cell, mesh->e_loc, mesh->etile,
                   mesh->cedge, mesh->jinv_f, mesh->nrm_f, mesh->len_f, mesh->hgeo_f, mesh->iarea,
                   mesh->node_f, mesh->psi_node};
  Phys &ph = c.phys;
  std::memset(&ph, 0, sizeof(ph));
  ph.gamma = cfg->gamma;
  ph.gamma_f = float(cfg->gamma);
  ph.gm1_f = float(cfg->gamma - 1.0);
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) ph.bc[i][j] = cfg->bc_state[i][j];
  ph.shock_x0 = cfg->shock_x0;
  if (cfg->shock_angle != 0.0) {
    ph.shock_cot = std::cos(cfg->shock_angle) / std::sin(cfg->shock_angle);
    ph.shock_vx = cfg->shock_speed / std::sin(cfg->shock_angle);
  }
  ph.shock_pre = cfg->shock_pre;
  ph.shock_post = cfg->shock_post;
  ph.oe = cfg->oe;
  ph.bp = cfg->bp;
  ph.k = cfg->k;
  ph.decomp = cfg->decomp;
  c.tr = s->tr;
  c.vd = s->vd;
  c.hs = s->hs;
  c.ej = s->ej;
  c.part_sum = s->part_sum;
  c.part_dev = s->part_dev;
  c.part_alpha = s->part_alpha;
  c.part_cnt = s->part_cnt;
  c.fin = s->fin;
  c.sc = s->sc;
  // scalars
  Scalars h{};
  h.t = 0.0;
  h.t_end = INFINITY;
  h.cfl = cfg->cfl;
  h.min_ca = mesh->min_ca[(cfg->k - 1) * 2 + (cfg->decomp == DG_DECOMP_ZXS ? 1 : 0)];
  h.area_total = mesh->area_total;
  h.active = 1;
  if ((rc = write_scalars(s, &h)) != DG_OK) { delete s; return rc; }
  // initial data: BP limiter once, traces and alpha (stage index -1: no step logic)
  if ((rc = upload_state(s, coeffs, s->uh)) != DG_OK) { delete s; return rc; }
  launch_oe_bp(c, s->uh, s->un, 0, cfg->bp != DG_BP_OFF, 0.0, -1);
  STRY(cudaGetLastError());
  Scalars r{};
  if ((rc = read_scalars(s, &r)) != DG_OK) { delete s; return rc; }
  if (r.nonphys > 0) {
    rc = fail(DG_ENONPHYS, "%lld initial cell averages are outside the admissible set", r.nonphys);
    delete s;
    return rc;
  }
  // capture one time step as a CUDA graph (with stack room for its kernels)
  if ((rc = ensure_stack_limit(stage_kernels_local_bytes(cfg->k, cfg->precision))) != DG_OK) {
    delete s;
    return rc;
  }
  cudaGraph_t graph = nullptr;
  STRY(cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal));
  enqueue_step(s);
  e = cudaStreamEndCapture(s->stream, &graph);
  if (e == cudaSuccess) e = cudaGraphInstantiate(&s->step_exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  STRY(e);
#undef STRY
  *out = s;
  return DG_OK;
}

extern "C" void dg_solver_destroy(dg_solver *s) {
  if (s && s->stream) cudaStreamSynchronize(s->stream);
  delete s;
}

extern "C" void *dg_stream(const dg_solver *s) { return s ? (void *)s->stream : nullptr; }

static void fill_stats(const Scalars &a, const Scalars &b, dg_stats *st) {
  if (!st) return;
  st->steps = b.steps - a.steps;
  st->limited_cells = b.limited - a.limited;
  st->nonphysical = b.nonphys - a.nonphys;
  st->cfl_breaches = b.breaches - a.breaches;
  st->t = b.t;
  st->dt_last = b.dt;
  st->alpha = b.alpha;
}

extern "C" int32_t dg_advance(dg_solver *s, double t_end, int64_t max_steps, dg_stats *stats) {
  if (!s) return fail(DG_EINVAL, "solver is NULL");
  if (max_steps < 0) return fail(DG_EINVAL, "max_steps < 0");
  Scalars h{};
  int32_t rc = read_scalars(s, &h);
  if (rc != DG_OK) return rc;
  const Scalars start = h;
  h.t_end = t_end;
  if ((rc = write_scalars(s, &h)) != DG_OK) return rc;
  int64_t done = 0;
  // launch in chunks; steps past t_end are no-ops on the device
  while (done < max_steps && h.t < t_end) {
    const int64_t chunk = std::min<int64_t>(max_steps - done, 32);
    for (int64_t i = 0; i < chunk; ++i) CUDA_TRY(cudaGraphLaunch(s->step_exec, s->stream));
    done += chunk;
    if ((rc = read_scalars(s, &h)) != DG_OK) return rc;
    if (!std::isfinite(h.alpha) || h.alpha <= 0.0) break;
  }
  fill_stats(start, h, stats);
  if (h.nonphys > start.nonphys)
    return fail(DG_ENONPHYS, "%lld cell averages left the admissible set", h.nonphys - start.nonphys);
  if (!std::isfinite(h.alpha)) return fail(DG_ENONPHYS, "the maximum wave speed is not finite");
  return DG_OK;
}

extern "C" int32_t dg_advance_async(dg_solver *s, int64_t n) {
  if (!s || n < 0) return fail(DG_EINVAL, "bad argument");
  for (int64_t i = 0; i < n; ++i) CUDA_TRY(cudaGraphLaunch(s->step_exec, s->stream));
  return DG_OK;
}

extern "C" int32_t dg_sync(dg_solver *s, dg_stats *stats) {
  if (!s) return fail(DG_EINVAL, "solver is NULL");
  CUDA_TRY(cudaStreamSynchronize(s->stream));
  if (stats) {
    Scalars h{};
    int32_t rc = read_scalars(s, &h);
    if (rc != DG_OK) return rc;
    Scalars z{};
    fill_stats(z, h, stats);
  }
  return DG_OK;
}

extern "C" int32_t dg_get_state(const dg_solver *s, double *coeffs, size_t len, double *t) {
  if (!s || !coeffs) return fail(DG_EINVAL, "NULL argument");
  if (len < (size_t)(4 * s->nb * s->mesh->nt)) return fail(DG_EINVAL, "output too small");
  int32_t rc = download_state(s, s->un, coeffs);
  if (rc != DG_OK) return rc;
  if (t) {
    Scalars h{};
    if ((rc = read_scalars(s, &h)) != DG_OK) return rc;
    *t = h.t;
  }
  return DG_OK;
}

extern "C" int32_t dg_set_state(dg_solver *s, const double *coeffs, double t) {
  if (!s || !coeffs) return fail(DG_EINVAL, "NULL argument");
  Scalars h{};
  int32_t rc = read_scalars(s, &h);
  if (rc != DG_OK) return rc;
  h.t = t;
  h.dt = 0.0;
  h.active = 1;
  if ((rc = write_scalars(s, &h)) != DG_OK) return rc;
  if ((rc = upload_state(s, coeffs, s->uh)) != DG_OK) return rc;
  launch_oe_bp(s->ctx, s->uh, s->un, 0, 0, 0.0, -1);   // traces and alpha only
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaStreamSynchronize(s->stream));
  return DG_OK;
}

// Instrumented steps: the kernels of enqueue_step launched one by one with a
// CUDA event pair around each launch, on the solver's stream.
extern "C" int32_t dg_profile_steps(dg_solver *s, int64_t n, double *ms, int64_t *launches) {
  if (!s || n < 0 || !ms || !launches) return fail(DG_EINVAL, "bad argument");
  for (int q = 0; q < DG_NUM_KERNEL_KINDS; ++q) { ms[q] = 0.0; launches[q] = 0; }
  const StageCtx &c = s->ctx;
  const int oe = s->cfg.oe != DG_OE_OFF, bp = s->cfg.bp != DG_BP_OFF;
  constexpr int MAXL = 1 + 3 * 6;
  cudaEvent_t ev[2 * MAXL];
  for (int i = 0; i < 2 * MAXL; ++i) CUDA_TRY(cudaEventCreate(&ev[i]));
  int32_t rc = DG_OK;
  for (int64_t step = 0; step < n && rc == DG_OK; ++step) {
    int kind[MAXL], nl = 0;
    auto rec = [&](int kd, auto &&fn) {
      cudaEventRecord(ev[2 * nl], s->stream);
      fn();
      cudaEventRecord(ev[2 * nl + 1], s->stream);
      kind[nl++] = kd;
    };
    rec(0, [&] { launch_step_begin(c); });
    for (int st = 0; st < 3; ++st) {
      const StateBuf &v = st == 0 ? s->un : s->us;
      rec(1, [&] { launch_rk_only(c, v, s->un, s->uh, RK_A[st], RK_B[st], C_IN[st]); });
      rec(2, [&] { launch_fin_mean(c); });
      if (oe) {
        rec(3, [&] { launch_stats_only(c, s->uh, C_OUT[st]); });
        rec(4, [&] { launch_fin_dev(c); });
      }
      rec(5, [&] { launch_oe_bp_only(c, s->uh, st == 2 ? s->un : s->us, oe, bp, C_OUT[st], st == 2); });
      rec(6, [&] { launch_fin_alpha(c, st); });
    }
    cudaError_t e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) { rc = fail(DG_ECUDA, "profiled step: %s", cudaGetErrorString(e)); break; }
    for (int i = 0; i < nl; ++i) {
      float t = 0.0f;
      cudaEventElapsedTime(&t, ev[2 * i], ev[2 * i + 1]);
      ms[kind[i]] += t;
      launches[kind[i]] += 1;
    }
  }
  for (int i = 0; i < 2 * MAXL; ++i) cudaEventDestroy(ev[i]);
  return rc;
}

// ============================================================================
// Single operators (host buffers).  They reuse the solver's buffers: the
// solver state is undefined afterwards until dg_set_state.
// ============================================================================
static int32_t op_prepare(dg_solver *s, double t, double dt, double alpha, Scalars *h) {
  int32_t rc = read_scalars(s, h);
  if (rc != DG_OK) return rc;
  h->t = t;
  h->dt = dt;
  h->alpha = alpha;
  h->active = 1;
  return write_scalars(s, h);
}

extern "C" int32_t dg_op_rk_stage(dg_solver *s, const double *un, const double *v, double a, double b, double dt,
                                  double alpha, double t, double *uh) {
  if (!s || !un || !v || !uh) return fail(DG_EINVAL, "NULL argument");
  Scalars h{};
  int32_t rc;
  if ((rc = op_prepare(s, t, dt, alpha, &h)) != DG_OK) return rc;
  if ((rc = upload_state(s, v, s->us)) != DG_OK) return rc;
  if ((rc = upload_state(s, un, s->un)) != DG_OK) return rc;
  launch_oe_bp(s->ctx, s->us, s->uh, 0, 0, 0.0, -1);   // traces of v; uh = v
  if ((rc = write_scalars(s, &h)) != DG_OK) return rc;  // restore alpha, dt
  launch_rk(s->ctx, s->uh, s->un, s->us, a, b, 0.0);
  CUDA_TRY(cudaGetLastError());
  return download_state(s, s->us, uh);
}

extern "C" int32_t dg_op_stats(dg_solver *s, const double *u, double *stats) {
  if (!s || !u || !stats) return fail(DG_EINVAL, "NULL argument");
  Scalars h{};
  int32_t rc;
  if ((rc = op_prepare(s, 0.0, 0.0, 0.0, &h)) != DG_OK) return rc;
  if ((rc = upload_state(s, u, s->us)) != DG_OK) return rc;
  launch_oe_bp(s->ctx, s->us, s->un, 0, 0, 0.0, -1);
  if ((rc = write_scalars(s, &h)) != DG_OK) return rc;
  launch_rk(s->ctx, s->un, s->un, s->uh, 1.0, 0.0, 0.0);   // uh = u, with |K| u^(0) block sums
  launch_stats(s->ctx, s->uh, 0.0);
  CUDA_TRY(cudaGetLastError());
  if ((rc = read_scalars(s, &h)) != DG_OK) return rc;
  for (int c = 0; c < 4; ++c) stats[c] = h.mean[c];
  stats[4] = h.dev[0];
  stats[5] = h.dev[1];
  stats[6] = h.dev[2];
  stats[7] = h.area_total;
  stats[8] = h.dev[3];
  stats[9] = h.dev[4];
  return DG_OK;
}

extern "C" int32_t dg_op_oe(dg_solver *s, const double *u, double dt, const double *stats, double t, double *out) {
  if (!s || !u || !stats || !out) return fail(DG_EINVAL, "NULL argument");
  Scalars h{};
  int32_t rc;
  if ((rc = op_prepare(s, t, dt, 0.0, &h)) != DG_OK) return rc;
  if ((rc = upload_state(s, u, s->us)) != DG_OK) return rc;
  launch_oe_bp(s->ctx, s->us, s->un, 0, 0, 0.0, -1);
  if ((rc = write_scalars(s, &h)) != DG_OK) return rc;
  launch_rk(s->ctx, s->un, s->un, s->uh, 1.0, 0.0, 0.0);   // vertex derivatives of u
  CUDA_TRY(cudaGetLastError());
  if ((rc = read_scalars(s, &h)) != DG_OK) return rc;
  h.t = t;
  h.dt = dt;
  if ((rc = write_scalars(s, &h)) != DG_OK) return rc;
  launch_stats(s->ctx, s->uh, 0.0);                         // jump data of every edge at time t
  CUDA_TRY(cudaGetLastError());
  if ((rc = read_scalars(s, &h)) != DG_OK) return rc;
  for (int c = 0; c < 4; ++c) h.mean[c] = stats[c];
  h.dev[0] = stats[4];
  h.dev[1] = stats[5];
  h.dev[2] = stats[6];
  h.dev[3] = stats[8];
  h.dev[4] = stats[9];
  h.t = t;
  h.dt = dt;
  if ((rc = write_scalars(s, &h)) != DG_OK) return rc;
  launch_set_inv_normalisers(s->ctx);
  launch_oe_bp(s->ctx, s->uh, s->us, 1, 0, 0.0, -1);
  CUDA_TRY(cudaGetLastError());
  return download_state(s, s->us, out);
}

extern "C" int32_t dg_op_limit(dg_solver *s, const double *u, double *out, int64_t *counters) {
  if (!s || !u || !out) return fail(DG_EINVAL, "NULL argument");
  Scalars h{};
  int32_t rc;
  if ((rc = op_prepare(s, 0.0, 0.0, 0.0, &h)) != DG_OK) return rc;
  if ((rc = upload_state(s, u, s->uh)) != DG_OK) return rc;
  launch_oe_bp(s->ctx, s->uh, s->us, 0, 1, 0.0, -1);
  CUDA_TRY(cudaGetLastError());
  Scalars r{};
  if ((rc = read_scalars(s, &r)) != DG_OK) return rc;
  if (counters) {
    counters[0] += r.limited - h.limited;
    counters[1] += r.nonphys - h.nonphys;
  }
  return download_state(s, s->us, out);
}

extern "C" int32_t dg_op_alpha(dg_solver *s, const double *u, double t, double *alpha) {
  if (!s || !u || !alpha) return fail(DG_EINVAL, "NULL argument");
  Scalars h{};
  int32_t rc;
  if ((rc = op_prepare(s, t, 0.0, 0.0, &h)) != DG_OK) return rc;
  if ((rc = upload_state(s, u, s->uh)) != DG_OK) return rc;
  launch_oe_bp(s->ctx, s->uh, s->us, 0, 0, 0.0, -1);
  CUDA_TRY(cudaGetLastError());
  Scalars r{};
  if ((rc = read_scalars(s, &r)) != DG_OK) return rc;
  *alpha = r.alpha;
  return DG_OK;
}

// ============================================================================
// Accessors used by the batch module
// ============================================================================
namespace dg {
const StageCtx &solver_ctx(const dg_solver *s) { return s->ctx; }
void solver_states(const dg_solver *s, StateBuf *un, StateBuf *uh, StateBuf *us) {
  *un = s->un;
  *uh = s->uh;
  *us = s->us;
}
int solver_nb(const dg_solver *s) { return s->nb; }
int32_t solver_read_scalars(const dg_solver *s, Scalars *h) { return read_scalars(s, h); }
int32_t solver_write_scalars(dg_solver *s, const Scalars *h) { return write_scalars(s, h); }
int32_t solver_capture_step(dg_solver *s, cudaGraph_t *graph) {
  *graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return set_error(DG_ECUDA, cudaGetErrorString(e));
  enqueue_step(s);
  e = cudaStreamEndCapture(s->stream, graph);
  if (e != cudaSuccess || !*graph) {
    cudaGetLastError();
    return set_error(DG_ECUDA, "step capture failed");
  }
  return DG_OK;
}

int32_t ensure_stack_limit(size_t bytes) {
  size_t cur = 0;
  cudaError_t e = cudaDeviceGetLimit(&cur, cudaLimitStackSize);
  if (e == cudaSuccess && cur < bytes) e = cudaDeviceSetLimit(cudaLimitStackSize, bytes);
  if (e != cudaSuccess) return set_error(DG_ECUDA, cudaGetErrorString(e));
  return DG_OK;
}

MeshDev mesh_device_view(const dg_mesh *m) {
  return MeshDev{m->nt,   m->area,   m->jinv,  m->nrm,   m->len,    m->vxy,    m->node,  m->hgeo, m->limv,
                 m->conn, m->ne,     m->e_cell, m->e_loc, m->etile, m->cedge, m->jinv_f, m->nrm_f, m->len_f,
                 m->hgeo_f, m->iarea, m->node_f, m->psi_node};
}

// every boundary edge carries a tag the scalar solver handles (transmissive or
// constant state), or any tag for the Euler solver
bool mesh_boundary_tags_ok(const dg_mesh *m, int scalar) {
  if (!scalar) return true;
  for (int8_t t : m->bnd_tag)
    if (t != 0 && !(t == DG_BC_TRANSMISSIVE || (t >= DG_BC_DIRICHLET0 && t < DG_BC_DIRICHLET0 + 4))) return false;
  return true;
}
}  // namespace dg

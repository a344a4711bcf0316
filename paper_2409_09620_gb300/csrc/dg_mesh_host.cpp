// dg_mesh_host.cpp -- host half of dg_mesh_create (see dg_mesh_host.h).
#include "dg_mesh_host.h"

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <new>

#include "../../include/dg.h"

namespace dg {
namespace {

int32_t set_err(std::string &err, int32_t code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  err = buf;
  return code;
}

struct EdgeKey {
  int32_t lo, hi;
  int64_t cell;
  int32_t edge;
};

int32_t build(int64_t nv, const double *xy, int64_t nt, const int32_t *tri, const int32_t *canon, const int8_t *bc,
              int tile, HostMesh &hm, std::string &err) {
  if (nv <= 0 || nt <= 0 || !xy || !tri)
    return set_err(err, DG_EINVAL, "empty mesh or NULL arrays (nv=%lld nt=%lld)", (long long)nv, (long long)nt);
  if (nt >= (int64_t(1) << 29)) return set_err(err, DG_EINVAL, "too many cells (%lld)", (long long)nt);
  if (tile <= 0) return set_err(err, DG_EINVAL, "tile must be positive");
  auto canon_of = [&](int32_t v) { return canon ? canon[v] : v; };
  // validation: vertex ids, orientation
  for (int64_t e = 0; e < 3 * nt; ++e)
    if (tri[e] < 0 || tri[e] >= nv) return set_err(err, DG_EMESH, "vertex id out of range at %lld", (long long)e);
  if (canon)
    for (int64_t v = 0; v < nv; ++v)
      if (canon[v] < 0 || canon[v] >= nv)
        return set_err(err, DG_EMESH, "canon id out of range at %lld", (long long)v);
  for (int64_t K = 0; K < nt; ++K) {
    const double *a = xy + 2 * tri[3 * K], *b = xy + 2 * tri[3 * K + 1], *c = xy + 2 * tri[3 * K + 2];
    const double det = (b[0] - a[0]) * (c[1] - a[1]) - (c[0] - a[0]) * (b[1] - a[1]);
    if (!(det > 0.0))
      return set_err(err, DG_EMESH, "cell %lld is not counter-clockwise with positive area", (long long)K);
  }
  // adjacency: sort edges by canonical vertex pair
  std::vector<EdgeKey> keys((size_t)(3 * nt));
  for (int64_t K = 0; K < nt; ++K)
    for (int i = 0; i < 3; ++i) {
      int32_t a = canon_of(tri[3 * K + (i + 1) % 3]), b = canon_of(tri[3 * K + (i + 2) % 3]);
      if (a == b) return set_err(err, DG_EMESH, "degenerate edge in cell %lld", (long long)K);
      keys[3 * K + i] = {std::min(a, b), std::max(a, b), K, i};
    }
  std::sort(keys.begin(), keys.end(), [](const EdgeKey &x, const EdgeKey &y) {
    if (x.lo != y.lo) return x.lo < y.lo;
    if (x.hi != y.hi) return x.hi < y.hi;
    if (x.cell != y.cell) return x.cell < y.cell;
    return x.edge < y.edge;
  });
  hm.nbr.assign((size_t)(3 * nt), -1);
  hm.nbr_edge.assign((size_t)(3 * nt), -1);
  for (size_t e = 0; e < keys.size();) {
    size_t f = e + 1;
    while (f < keys.size() && keys[f].lo == keys[e].lo && keys[f].hi == keys[e].hi) ++f;
    if (f - e > 2) return set_err(err, DG_EMESH, "edge shared by more than two cells");
    if (f - e == 2) {
      const EdgeKey &p = keys[e], &q = keys[e + 1];
      // the two cells must traverse the shared edge in opposite directions
      int32_t pa = canon_of(tri[3 * p.cell + (p.edge + 1) % 3]);
      int32_t qa = canon_of(tri[3 * q.cell + (q.edge + 1) % 3]);
      if (pa == qa) return set_err(err, DG_EMESH, "edge traversed twice in the same direction");
      // both ends of an identified (periodic) edge move by the same translation;
      // for an ordinary interior edge both translations are zero
      const int32_t p0 = tri[3 * p.cell + (p.edge + 1) % 3], p1 = tri[3 * p.cell + (p.edge + 2) % 3];
      const int32_t q0 = tri[3 * q.cell + (q.edge + 1) % 3], q1 = tri[3 * q.cell + (q.edge + 2) % 3];
      const double sx = xy[2 * q1] - xy[2 * p0], sy = xy[2 * q1 + 1] - xy[2 * p0 + 1];
      const double tx = xy[2 * q0] - xy[2 * p1], ty = xy[2 * q0 + 1] - xy[2 * p1 + 1];
      const double scale = 1.0 + std::fabs(sx) + std::fabs(sy);
      if (!(std::fabs(sx - tx) <= 1e-9 * scale && std::fabs(sy - ty) <= 1e-9 * scale))
        return set_err(err, DG_EMESH, "the two copies of periodic edge %d of cell %lld are not translates",
                       p.edge, (long long)p.cell);
      hm.nbr[3 * p.cell + p.edge] = (int32_t)q.cell;
      hm.nbr_edge[3 * p.cell + p.edge] = q.edge;
      hm.nbr[3 * q.cell + q.edge] = (int32_t)p.cell;
      hm.nbr_edge[3 * q.cell + q.edge] = p.edge;
    } else {
      const int8_t tag = bc ? bc[3 * keys[e].cell + keys[e].edge] : 0;
      if (tag < DG_BC_REFLECT || tag > DG_BC_SHOCK)
        return set_err(err, DG_EMESH, "boundary edge %d of cell %lld has no valid tag", keys[e].edge,
                       (long long)keys[e].cell);
    }
    e = f;
  }
  hm.conn.assign((size_t)(3 * nt), 0);
  hm.bnd_tag.assign((size_t)(3 * nt), 0);
  for (int64_t K = 0; K < nt; ++K)
    for (int i = 0; i < 3; ++i) {
      const int32_t nbK = hm.nbr[3 * K + i];
      hm.conn[(size_t)i * nt + K] = nbK >= 0 ? ((nbK << 2) | hm.nbr_edge[3 * K + i]) : -(int32_t)bc[3 * K + i];
      if (nbK < 0) hm.bnd_tag[3 * K + i] = bc[3 * K + i];
    }
  // edge list: every edge once, owned by its lower cell id (or its only cell),
  // ordered by owner; tiles of `tile` cells own contiguous edge ranges
  const int64_t ntiles = (nt + tile - 1) / tile;
  hm.e_cell.clear();
  hm.e_loc.clear();
  hm.etile.assign((size_t)ntiles + 1, 0);
  hm.cedge.assign((size_t)(3 * nt), 0);
  for (int64_t K = 0; K < nt; ++K) {
    if (K % tile == 0) hm.etile[(size_t)(K / tile)] = (int32_t)hm.e_cell.size();
    for (int i = 0; i < 3; ++i) {
      const int32_t nbK = hm.nbr[3 * K + i];
      if (nbK < 0 || K < nbK) {
        hm.cedge[(size_t)i * nt + K] = (int32_t)hm.e_cell.size();
        hm.e_cell.push_back((int32_t)K);
        hm.e_loc.push_back((int8_t)i);
      }
    }
  }
  hm.etile[(size_t)ntiles] = (int32_t)hm.e_cell.size();
  for (int64_t K = 0; K < nt; ++K)
    for (int i = 0; i < 3; ++i) {
      const int32_t nbK = hm.nbr[3 * K + i];
      if (nbK >= 0 && nbK < K) hm.cedge[(size_t)i * nt + K] = hm.cedge[(size_t)hm.nbr_edge[3 * K + i] * nt + nbK];
    }
  hm.vxy.resize((size_t)(6 * nt));
  for (int64_t K = 0; K < nt; ++K)
    for (int v = 0; v < 3; ++v) {
      hm.vxy[(size_t)(2 * v) * nt + K] = xy[2 * tri[3 * K + v]];
      hm.vxy[(size_t)(2 * v + 1) * nt + K] = xy[2 * tri[3 * K + v] + 1];
    }
  return DG_OK;
}

}  // namespace

int32_t build_host_mesh(int64_t nv, const double *xy, int64_t nt, const int32_t *tri, const int32_t *canon,
                        const int8_t *bc, int tile, HostMesh &out, std::string &err) {
  try {
    return build(nv, xy, nt, tri, canon, bc, tile, out, err);
  } catch (const std::bad_alloc &) {
    return set_err(err, DG_ENOMEM, "host allocation failed");
  }
}

}  // namespace dg

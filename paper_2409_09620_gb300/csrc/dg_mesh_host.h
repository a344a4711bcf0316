// dg_mesh_host.h -- the host half of mesh construction: input validation,
// edge adjacency (periodic sides identified through the canonical vertex
// ids), the packed connectivity the stage kernels read and the edge list of
// the edge kernels.  Plain C++ with no CUDA header, so that it also builds and
// runs on a machine without a GPU.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace dg {

struct HostMesh {
  std::vector<int32_t> nbr, nbr_edge;   // [nt][3]: neighbour across edge i and its local edge; -1 on a boundary
  std::vector<int8_t> bnd_tag;          // [nt][3]: tag of a boundary edge, 0 on interior edges
  std::vector<int32_t> conn;            // [3][nt]: (neighbour << 2) | its local edge, or -tag on a boundary
  std::vector<int32_t> e_cell;          // [ne]: owner of each edge (its lower cell id, or its only cell)
  std::vector<int8_t> e_loc;            // [ne]: the owner's local index of the edge
  std::vector<int32_t> etile;           // [ntiles + 1]: first edge owned by each tile of `tile` cells, then ne
  std::vector<int32_t> cedge;           // [3][nt]: edge id of local edge i of cell K (both cells of an edge agree)
  std::vector<double> vxy;              // [6][nt]: x0, y0, x1, y1, x2, y2 of each cell's vertices
};

// Edge i of a cell is the one opposite its vertex i; cells are counter-
// clockwise.  Returns 0 or DG_EINVAL (empty mesh, NULL arrays, too many
// cells), DG_EMESH (vertex or canonical id out of range, area <= 0, an edge
// with coincident canonical ends, an edge shared by more than two cells or
// traversed twice in the same direction, the two copies of a periodic edge
// that are not translates of each other, a boundary edge without a valid tag)
// or DG_ENOMEM, with a message in `err`.  `tile` is the number of cells per
// tile of the edge list.
int32_t build_host_mesh(int64_t nv, const double *xy, int64_t nt, const int32_t *tri, const int32_t *canon,
                        const int8_t *bc, int tile, HostMesh &out, std::string &err);

}  // namespace dg

// mesh_host_driver.cpp -- runs the library's host mesh builder
// (paper_2409_09620_gb300/csrc/dg_mesh_host.cpp) on a mesh read from a file,
// for a CPU build under AddressSanitizer and UndefinedBehaviorSanitizer
// (tests/test_mesh_host.py).  Test infrastructure.
//
// Input (native byte order): int64 nv, nt, tile, has_canon, has_bc; double
// xy[2 nv]; int32 tri[3 nt]; int32 canon[nv] if has_canon; int8 bc[3 nt] if
// has_bc.  Output: int32 status, int64 message length, the message; then, on
// success, int32 nbr[3 nt], nbr_edge[3 nt], int8 bnd_tag[3 nt], int32
// conn[3 nt], int64 ne, int32 e_cell[ne], int8 e_loc[ne], int64 ntiles, int32
// etile[ntiles + 1], int32 cedge[3 nt], double vxy[6 nt].
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <string>
#include <vector>

#include "dg_mesh_host.h"

template <typename T>
static std::vector<T> read_vec(FILE *f, size_t n) {
  std::vector<T> v(n);
  if (n && fread(v.data(), sizeof(T), n, f) != n) {
    fprintf(stderr, "short read\n");
    exit(3);
  }
  return v;
}

template <typename T>
static void write_vec(FILE *f, const std::vector<T> &v) {
  if (!v.empty() && fwrite(v.data(), sizeof(T), v.size(), f) != v.size()) exit(4);
}

template <typename T>
static void write_one(FILE *f, T x) {
  if (fwrite(&x, sizeof(T), 1, f) != 1) exit(4);
}

int main(int argc, char **argv) {
  if (argc != 3) return 2;
  FILE *f = fopen(argv[1], "rb");
  FILE *out = fopen(argv[2], "wb");
  if (!f || !out) return 2;
  std::vector<int64_t> h = read_vec<int64_t>(f, 5);
  const int64_t nv = h[0], nt = h[1];
  const int tile = (int)h[2];
  std::vector<double> xy = read_vec<double>(f, (size_t)(nv > 0 ? 2 * nv : 0));
  std::vector<int32_t> tri = read_vec<int32_t>(f, (size_t)(nt > 0 ? 3 * nt : 0));
  std::vector<int32_t> canon = h[3] ? read_vec<int32_t>(f, (size_t)nv) : std::vector<int32_t>();
  std::vector<int8_t> bc = h[4] ? read_vec<int8_t>(f, (size_t)(3 * nt)) : std::vector<int8_t>();
  fclose(f);
  dg::HostMesh hm;
  std::string err;
  const int32_t rc = dg::build_host_mesh(nv, xy.empty() ? nullptr : xy.data(), nt,
                                         tri.empty() ? nullptr : tri.data(), h[3] ? canon.data() : nullptr,
                                         h[4] ? bc.data() : nullptr, tile, hm, err);
  write_one<int32_t>(out, rc);
  write_one<int64_t>(out, (int64_t)err.size());
  if (!err.empty() && fwrite(err.data(), 1, err.size(), out) != err.size()) return 4;
  if (rc == 0) {
    write_vec(out, hm.nbr);
    write_vec(out, hm.nbr_edge);
    write_vec(out, hm.bnd_tag);
    write_vec(out, hm.conn);
    write_one<int64_t>(out, (int64_t)hm.e_cell.size());
    write_vec(out, hm.e_cell);
    write_vec(out, hm.e_loc);
    write_one<int64_t>(out, (int64_t)hm.etile.size() - 1);
    write_vec(out, hm.etile);
    write_vec(out, hm.cedge);
    write_vec(out, hm.vxy);
  }
  return fclose(out) == 0 ? 0 : 4;
}

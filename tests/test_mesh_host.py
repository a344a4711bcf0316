"""The library's host mesh builder (``csrc/dg_mesh_host.cpp``, the host half
of ``dg_mesh_create``) on the CPU, built with AddressSanitizer and
UndefinedBehaviorSanitizer through a small driver (``tests/mesh_host_driver.cpp``).

* The adjacency (neighbour and its local edge across every edge) equals the
  oracle's, bit for bit, on periodic, wall, inflow/outflow, moving-shock and
  unstructured meshes.
* The packed connectivity decodes to that adjacency and to the boundary tags.
* The edge list holds every edge once, owned by its lower cell id (or its only
  cell), ordered by owner, with tile ranges and per-cell edge ids consistent
  on both sides of each edge, for the kernels' tile of 128 cells and for a
  ragged tile of 5.
* Rejected inputs return the documented status with a message, and the
  oracle rejects the same meshes.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_2409_09620_gb300 import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_2409_09620_gb300", "csrc")
DG_OK, DG_EINVAL, DG_EMESH = 0, -1, -2


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("no g++")
    d = tmp_path_factory.mktemp("meshhost")
    exe = str(d / "driver")
    cmd = ["g++", "-O1", "-g", "-std=c++17", "-fsanitize=address,undefined", "-fno-sanitize-recover=all",
           "-fno-omit-frame-pointer", "-Wall", "-I", CSRC, os.path.join(HERE, "mesh_host_driver.cpp"),
           os.path.join(CSRC, "dg_mesh_host.cpp"), "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0 and ("asan" in r.stderr or "ubsan" in r.stderr):
        pytest.skip("the sanitizer runtimes are not installed")
    assert r.returncode == 0, r.stderr
    return exe, d


def build_host(driver, name, xy, tri, canon=None, bc=None, tile=128):
    exe, d = driver
    xy = np.ascontiguousarray(xy, np.float64).reshape(-1, 2)
    tri = np.ascontiguousarray(tri, np.int32).reshape(-1, 3)
    nv, nt = xy.shape[0], tri.shape[0]
    fin, fout = str(d / f"{name}.in"), str(d / f"{name}.out")
    with open(fin, "wb") as f:
        f.write(np.array([nv, nt, tile, canon is not None, bc is not None], np.int64).tobytes())
        f.write(xy.tobytes())
        f.write(tri.tobytes())
        if canon is not None:
            f.write(np.ascontiguousarray(canon, np.int32).tobytes())
        if bc is not None:
            f.write(np.ascontiguousarray(bc, np.int8).tobytes())
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1:exitcode=23", UBSAN_OPTIONS="print_stacktrace=1")
    r = subprocess.run([exe, fin, fout], capture_output=True, text=True, env=env, timeout=120)
    assert r.returncode == 0 and "runtime error" not in r.stderr, r.stderr[-4000:]
    raw = open(fout, "rb").read()
    pos = 0

    def take(dtype, n):
        nonlocal pos
        a = np.frombuffer(raw, dtype, n, pos)
        pos += a.nbytes
        return a
    rc = int(take(np.int32, 1)[0])
    msg = take(np.uint8, int(take(np.int64, 1)[0])).tobytes().decode()
    if rc != DG_OK:
        return rc, msg, None
    out = {"nbr": take(np.int32, 3 * nt).reshape(nt, 3), "nbr_edge": take(np.int32, 3 * nt).reshape(nt, 3),
           "bnd_tag": take(np.int8, 3 * nt).reshape(nt, 3), "conn": take(np.int32, 3 * nt).reshape(3, nt)}
    ne = int(take(np.int64, 1)[0])
    out["e_cell"], out["e_loc"] = take(np.int32, ne), take(np.int8, ne)
    ntiles = int(take(np.int64, 1)[0])
    out["etile"] = take(np.int32, ntiles + 1)
    out["cedge"] = take(np.int32, 3 * nt).reshape(3, nt)
    out["vxy"] = take(np.float64, 6 * nt).reshape(6, nt)
    assert pos == len(raw)
    return rc, msg, out


MESHES = {
    "vortex_periodic": lambda: W.vortex_workload(n=9, k=1).mesh,
    "dmr": lambda: W.dmr_workload(nx=12, ny=4, k=2).mesh,
    "sedov_walls": lambda: W.sedov_workload(n=10, k=2).mesh,
    "riemann_transmissive": lambda: W.riemann4_workload(n=7, k=1).mesh,
    "ffs_unstructured": lambda: W.ffs_mesh(h=1.0 / 8),
    "wedge_unstructured": lambda: W.wedge_mesh(h=1.0 / 10),
}


@pytest.mark.parametrize("tile", [128, 5])
@pytest.mark.parametrize("name", sorted(MESHES))
def test_host_builder_matches_oracle_adjacency(oracle_mod, driver, name, tile):
    mesh = MESHES[name]()
    nt = mesh.tri.shape[0]
    rc, msg, h = build_host(driver, f"{name}_{tile}", mesh.xy, mesh.tri, mesh.canon, mesh.bc, tile)
    assert rc == DG_OK, msg
    om = oracle_mod.OracleMesh.from_mesh(mesh)
    nbr, ne = om.neighbors()
    assert np.array_equal(h["nbr"], nbr) and np.array_equal(h["nbr_edge"], ne)
    # packed connectivity and boundary tags
    K = np.arange(nt)
    for i in range(3):
        c = h["conn"][i]
        inner = nbr[:, i] >= 0
        assert np.array_equal(c[inner] >> 2, nbr[inner, i]) and np.array_equal(c[inner] & 3, ne[inner, i])
        assert np.array_equal(-c[~inner], mesh.bc[~inner, i].astype(np.int32))
        assert np.array_equal(h["bnd_tag"][~inner, i], mesh.bc[~inner, i])
        assert not h["bnd_tag"][inner, i].any()
    # edge list: each edge once, owned by its lower cell (or its only cell)
    n_int = int((nbr >= 0).sum()) // 2
    n_bnd = int((nbr < 0).sum())
    assert h["e_cell"].size == n_int + n_bnd
    assert np.all(np.diff(h["e_cell"]) >= 0)
    owner_nbr = nbr[h["e_cell"], h["e_loc"]]
    assert np.all((owner_nbr < 0) | (owner_nbr > h["e_cell"]))
    seen = np.zeros((nt, 3), int)
    seen[h["e_cell"], h["e_loc"]] += 1
    inner = owner_nbr >= 0
    seen[owner_nbr[inner], ne[h["e_cell"][inner], h["e_loc"][inner]]] += 1
    assert (seen == 1).all()
    # tiles own contiguous ranges; per-cell edge ids agree across each edge
    ntiles = (nt + tile - 1) // tile
    assert h["etile"].size == ntiles + 1 and h["etile"][-1] == h["e_cell"].size
    for t in range(ntiles):
        assert h["etile"][t] == np.searchsorted(h["e_cell"], t * tile)
    for i in range(3):
        e = h["cedge"][i]
        own = (h["e_cell"][e] == K) & (h["e_loc"][e] == i)
        other = ~own
        assert np.all(nbr[other, i] >= 0)
        assert np.all(h["e_cell"][e[other]] == nbr[other, i])
        assert np.all(h["e_loc"][e[other]] == ne[other, i])
    # vertex coordinates per cell
    for v in range(3):
        assert np.array_equal(h["vxy"][2 * v], mesh.xy[mesh.tri[:, v], 0])
        assert np.array_equal(h["vxy"][2 * v + 1], mesh.xy[mesh.tri[:, v], 1])


_STRIP_TRI = [[c, c + 1, c + 5] for c in range(3)] + [[c, c + 5, c + 4] for c in range(3)]
_STRIP_CANON = np.array([0, 1, 2, 0, 4, 5, 6, 4], np.int32)


def _strip(right_height):
    xy = np.array([[i, 0.0] for i in range(4)] + [[i, 1.0] for i in range(4)])
    xy[7, 1] = right_height
    return xy


def _bad_cases():
    """name -> (xy, tri, canon, bc, expected status, part of the message)"""
    sq = np.array([[0, 0], [1, 0], [1, 1], [0, 1], [-1, 0.5]], float)
    w = lambda n: np.full((n, 3), 1, np.int8)
    return {
        "clockwise": (sq, [[0, 2, 1]], None, w(1), DG_EMESH, "counter-clockwise"),
        "zero_area": (np.array([[0, 0], [1, 0], [2, 0]], float), [[0, 1, 2]], None, w(1), DG_EMESH,
                      "positive area"),
        "vertex_out_of_range": (sq, [[0, 1, 7]], None, w(1), DG_EMESH, "vertex id"),
        "negative_vertex": (sq, [[0, 1, -1]], None, w(1), DG_EMESH, "vertex id"),
        "untagged_boundary": (sq, [[0, 1, 2]], None, None, DG_EMESH, "no valid tag"),
        "tag_out_of_range": (sq, [[0, 1, 2]], None, np.full((1, 3), 9, np.int8), DG_EMESH, "no valid tag"),
        # the diagonal {0, 2} in three counter-clockwise cells
        "non_manifold": (sq, [[0, 1, 2], [0, 2, 3], [0, 2, 4]], None, w(3), DG_EMESH, "more than two"),
        "valid_pair": (sq, [[0, 1, 2], [0, 2, 3]], None, w(2), DG_OK, ""),
        "canon_out_of_range": (sq, [[0, 1, 2]], np.array([0, 1, 9, 3, 4], np.int32), w(1), DG_EMESH, "canon"),
        "canon_degenerate_edge": (sq, [[0, 1, 2]], np.array([0, 0, 2, 3, 4], np.int32), w(1), DG_EMESH,
                                  "degenerate edge"),
        "empty": (np.zeros((0, 2)), np.zeros((0, 3), np.int32), None, None, DG_EINVAL, "empty mesh"),
        # a 3 x 1 strip periodic in x; moving vertex 7 makes the right side
        # 1.2 long against the left side's 1
        "periodic_not_translates": (_strip(1.2), _STRIP_TRI, _STRIP_CANON, w(6), DG_EMESH, "not translates"),
        "periodic_translates": (_strip(1.0), _STRIP_TRI, _STRIP_CANON, w(6), DG_OK, ""),
    }


@pytest.mark.parametrize("case", sorted(_bad_cases()))
def test_host_builder_rejects_bad_meshes(oracle_mod, driver, case):
    xy, tri, canon, bc, want, text = _bad_cases()[case]
    rc, msg, _ = build_host(driver, f"bad_{case}", xy, tri, canon, bc)
    assert rc == want and text in msg, (rc, msg)
    if want == DG_EMESH:
        with pytest.raises(ValueError):
            oracle_mod.OracleMesh(np.asarray(xy, float), np.asarray(tri, np.int32), canon, bc)


def test_host_builder_rejects_edge_traversed_twice_in_one_direction(oracle_mod, driver):
    """Two counter-clockwise cells on the same side of their shared edge
    (overlapping) list it in the same direction: rejected by both."""
    xy = np.array([[0, 0], [1, 0], [0, 1], [0.2, 0.2]], float)
    tri = np.array([[0, 1, 2], [3, 1, 2]], np.int32)   # edge opposite vertex 0 / 3 goes 1 -> 2 in both
    bc = np.full((2, 3), 1, np.int8)
    rc, msg, _ = build_host(driver, "same_dir", xy, tri, None, bc)
    assert rc == DG_EMESH and "same direction" in msg
    with pytest.raises(ValueError):
        oracle_mod.OracleMesh(xy, tri, None, bc)

"""Lattice meshes of the non-rectangular domains of Sec. 5 (the tunnel with a
forward facing step and the tube over a 30-degree wedge) and the oracle on
them.

Pins: the mesh covers exactly the domain (area and boundary length per
boundary kind from the domain's shape), it is conforming (the oracle's
adjacency accepts it; every interior edge is shared by two cells), and the
inflow, outflow, wall and moving-shock conditions reproduce a uniform state
wherever the obstacle or the shock cannot reach within one step.  A longer
oracle run keeps density and pressure positive at every limiter point.
"""
import math

import numpy as np
import pytest

from paper_2409_09620_gb300 import workloads as W

S3 = math.sqrt(3.0)
FFS_AREA = 3.0 - 2.4 * 0.2
WEDGE_AREA = 2.8 * 2.0 - 0.5 * 2.7 * (2.7 / S3)
# boundary length per tag (inflow, outflow, walls, moving-shock exact solution)
FFS_LENGTHS = {W.BC_DIRICHLET0: 1.0, W.BC_TRANSMISSIVE: 0.8, W.BC_REFLECT: 0.6 + 0.2 + 2.4 + 3.0}
WEDGE_LENGTHS = {W.BC_DIRICHLET0: 2.0, W.BC_TRANSMISSIVE: 2.0 - 2.7 / S3, W.BC_SHOCK: 2.8 + 0.1,
                 W.BC_REFLECT: 2.0 * 2.7 / S3}


def _mesh(name, h):
    return W.ffs_mesh(h) if name == "ffs" else W.wedge_mesh(h)


def _cell_geometry(m):
    p = m.xy[m.tri]
    area = 0.5 * ((p[:, 1, 0] - p[:, 0, 0]) * (p[:, 2, 1] - p[:, 0, 1])
                  - (p[:, 2, 0] - p[:, 0, 0]) * (p[:, 1, 1] - p[:, 0, 1]))
    ang = []
    for i in range(3):
        u = p[:, (i + 1) % 3] - p[:, i]
        v = p[:, (i + 2) % 3] - p[:, i]
        c = (u * v).sum(1) / np.linalg.norm(u, axis=1) / np.linalg.norm(v, axis=1)
        ang.append(np.degrees(np.arccos(np.clip(c, -1.0, 1.0))))
    return area, np.min(ang, axis=0), p.mean(axis=1)


def _on_wall(name, pa, pb):
    """Both end points on a wall of the domain (reflecting boundary)."""
    if name == "ffs":
        segs = [lambda x, y: y == 0.0 and x <= 0.6, lambda x, y: x == 0.6 and y <= 0.2,
                lambda x, y: y == 0.2 and x >= 0.6, lambda x, y: y == 1.0]
        return any(s(*pa) and s(*pb) for s in segs)
    on_face = lambda x, y: abs(y - (x - 0.1) / S3) <= 1e-12
    return on_face(*pa) and on_face(*pb)


@pytest.mark.parametrize("name,h", [("ffs", 1 / 20), ("ffs", 1 / 37), ("wedge", 1 / 16), ("wedge", 1 / 29)])
def test_lattice_mesh_covers_the_domain(oracle_mod, name, h):
    m = _mesh(name, h)
    area, min_angle, _ = _cell_geometry(m)
    assert (area > 0).all()                              # counter-clockwise
    expect = FFS_AREA if name == "ffs" else WEDGE_AREA
    assert abs(area.sum() - expect) <= 1e-12 * expect
    assert min_angle.min() > 15.0 and np.median(min_angle) > 45.0   # near-equilateral lattice
    # edges: interior ones twice and untagged, boundary ones once and tagged
    a = m.tri[:, [1, 2, 0]].reshape(-1).astype(np.int64)
    b = m.tri[:, [2, 0, 1]].reshape(-1).astype(np.int64)
    key = np.minimum(a, b) * m.nv + np.maximum(a, b)
    _, inv, cnt = np.unique(key, return_inverse=True, return_counts=True)
    assert cnt.max() <= 2
    tags = m.bc.reshape(-1)
    once = cnt[inv] == 1
    assert (tags[once] != 0).all() and (tags[~once] == 0).all()
    # boundary length per tag, and every wall edge on a wall
    lengths = {}
    for e in np.nonzero(once)[0]:
        pa, pb = m.xy[a[e]], m.xy[b[e]]
        lengths[int(tags[e])] = lengths.get(int(tags[e]), 0.0) + float(np.hypot(*(pb - pa)))
        if tags[e] == W.BC_REFLECT:
            assert _on_wall(name, pa, pb)
    want = FFS_LENGTHS if name == "ffs" else WEDGE_LENGTHS
    assert set(lengths) == set(want)
    for t, L in want.items():
        assert abs(lengths[t] - L) <= 1e-12 * L
    oracle_mod.OracleMesh.from_mesh(m)                   # conforming adjacency


@pytest.mark.parametrize("k", [1, 2])
def test_ffs_free_stream_away_from_the_step(oracle_mod, k):
    """One step of the uniform Mach-3 state: the inflow state, the outflow
    copy and the walls parallel to the flow reproduce the free stream, so only
    cells within reach of the step's face change."""
    O = oracle_mod
    h = 1 / 20
    wl = W.ffs_workload(h=h, k=k)
    om = O.OracleMesh.from_mesh(wl.mesh)
    cf = O.config_for(wl)
    u0 = O.project_workload(om, wl)
    u, t, dt, cnt, rc = om.step(cf, u0, 0.0, 10.0)
    assert rc == 0 and t > 0
    _, _, cen = _cell_geometry(wl.mesh)
    # distance of the centroid to the step's face x = 0.6, 0 <= y <= 0.2
    d = np.hypot(np.maximum(0.6 - cen[:, 0], cen[:, 0] - 0.6), np.maximum(cen[:, 1] - 0.2, 0.0))
    far = d > 6 * h
    diff = np.abs(u - u0).max(axis=(0, 1))
    assert diff[far].max() <= 1e-13 * np.abs(u0).max()
    assert diff[~far].max() > 1e-3


@pytest.mark.parametrize("k", [1, 2])
def test_wedge_uniform_away_from_the_shock(oracle_mod, k):
    """One step of the moving Mach-10 shock: the inflow state, the exact
    solution on the top and on the bottom before the wedge, the outflow copy
    and the reflecting wedge keep both uniform states wherever the shock
    cannot reach."""
    O = oracle_mod
    h = 1 / 16
    wl = W.wedge_dmr_workload(h=h, k=k)
    om = O.OracleMesh.from_mesh(wl.mesh)
    cf = O.config_for(wl)
    u0 = O.project_workload(om, wl)
    u, t, dt, cnt, rc = om.step(cf, u0, 0.0, 10.0)
    assert rc == 0 and t > 0
    _, _, cen = _cell_geometry(wl.mesh)
    far = np.abs(cen[:, 0] - 0.1) > 6 * h + 10.0 * t
    diff = np.abs(u - u0).max(axis=(0, 1))
    assert diff[far].max() <= 1e-13 * np.abs(u0).max()
    assert diff[~far].max() > 1e-2


@pytest.mark.parametrize("name", ["ffs", "wedge"])
def test_positivity_on_lattice_meshes(oracle_mod, name):
    """40 P2 steps with the BP limiter: density and pressure stay positive at
    every point of the limiter set (Sec. 4.4)."""
    O = oracle_mod
    wl = W.ffs_workload(h=1 / 20, k=2) if name == "ffs" else W.wedge_dmr_workload(h=1 / 16, k=2)
    om = O.OracleMesh.from_mesh(wl.mesh)
    cf = O.config_for(wl)
    u, t, cnt, rc = om.advance(cf, O.project_workload(om, wl), 0.0, 10.0, max_steps=40)
    assert rc == 0 and cnt[3] == 40 and cnt[1] == 0
    assert np.isfinite(u).all()
    mins = om.point_minima(cf, u)
    assert (mins > 0).all()
    if name == "wedge":
        assert cnt[0] > 0          # the limiter acts behind the shock

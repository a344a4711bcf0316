"""The seeded synthetic inputs follow their stated recipes.

* Jittered grids: 2 nx ny counter-clockwise cells; boundary and fixed
  vertices stay on the grid; interior vertices move by at most 0.2 h per
  coordinate; the same seed gives the same mesh; both diagonals occur;
  periodic copies are exact translates; side tags sit on the right edges.
* Double Mach reflection: the post- and pre-shock states satisfy the
  Rankine-Hugoniot conditions across a shock of normal speed 10 with the
  post-shock velocity along the shock normal (60 degrees to the x-axis); the
  initial shock passes through (1/6, 0); the boundary tags match the
  problem.
* Sedov blast: the blast energy 0.244816 sits in the cells around the
  un-jittered origin; the gas elsewhere is at rest with p = 1e-10.
* Isentropic vortex: p / rho^gamma = 1 everywhere, and the state tends to
  the free stream away from the centre.
* Four-quadrant Riemann problem: one constant state per quadrant, drawn
  from the stated ranges.
"""
import math
import re

import numpy as np
import pytest

from paper_2409_09620_gb300 import workloads as W


def _area(mesh):
    a, b, c = (mesh.xy[mesh.tri[:, i]] for i in range(3))
    return 0.5 * ((b[:, 0] - a[:, 0]) * (c[:, 1] - a[:, 1]) - (c[:, 0] - a[:, 0]) * (b[:, 1] - a[:, 1]))


@pytest.mark.parametrize("periodic", [False, True])
def test_jittered_grid_recipe(periodic):
    nx, ny, box = 12, 7, (-1.0, 2.0, 0.5, 1.5)
    tags = None if periodic else {"left": 1, "right": 2, "bottom": 3, "top": 7}
    m = W.jittered_grid(nx, ny, box, seed=9, periodic=periodic, fixed_points=[(0.0, 1.0 + 1.0 / 14)],
                        side_tags=tags)
    assert m.tri.shape == (2 * nx * ny, 3) and (_area(m) > 0).all()
    hx, hy = (box[1] - box[0]) / nx, (box[3] - box[2]) / ny
    ii, jj = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), indexing="xy")
    grid = np.stack([box[0] + ii.ravel() * hx, box[2] + jj.ravel() * hy], axis=1)
    d = m.xy - grid
    assert (np.abs(d[:, 0]) <= 0.2 * hx + 1e-15).all() and (np.abs(d[:, 1]) <= 0.2 * hy + 1e-15).all()
    on_boundary = (ii.ravel() % nx == 0) | (jj.ravel() % ny == 0)
    assert (d[on_boundary] == 0).all()
    fixed = np.argmin(np.hypot(grid[:, 0] - 0.0, grid[:, 1] - (1.0 + 1.0 / 14)))
    assert (d[fixed] == 0).all() and (d[~on_boundary] != 0).any()
    # the same seed, the same mesh; another seed, another mesh
    m2 = W.jittered_grid(nx, ny, box, seed=9, periodic=periodic, fixed_points=[(0.0, 1.0 + 1.0 / 14)],
                         side_tags=tags)
    m3 = W.jittered_grid(nx, ny, box, seed=10, periodic=periodic, fixed_points=[(0.0, 1.0 + 1.0 / 14)],
                         side_tags=tags)
    assert np.array_equal(m.xy, m2.xy) and np.array_equal(m.tri, m2.tri)
    assert not np.array_equal(m.xy, m3.xy)
    # both diagonals: a square's two cells share either (v00, v11) or (v10, v01)
    first = m.tri[0::2]
    assert len({tuple(sorted(r)) for r in first[:, [0, 2]].tolist()}) > 1
    assert (first[:, 2] == first[:, 1] + nx + 1).any() and (first[:, 2] == first[:, 0] + nx + 1).any()
    if periodic:
        # vertex (i, j) and its canonical copy differ by whole periods
        c = m.canon
        shift = m.xy - m.xy[c]
        Lx, Ly = box[1] - box[0], box[3] - box[2]
        assert set(np.unique(shift[:, 0])) <= {0.0, Lx} and set(np.unique(shift[:, 1])) <= {0.0, Ly}
        assert (m.bc == 0).all()
    else:
        for e in range(3):
            a, b = m.tri[:, (e + 1) % 3], m.tri[:, (e + 2) % 3]
            on = {"left": (grid[a, 0] == box[0]) & (grid[b, 0] == box[0]),
                  "right": (grid[a, 0] == box[1]) & (grid[b, 0] == box[1]),
                  "bottom": (grid[a, 1] == box[2]) & (grid[b, 1] == box[2]),
                  "top": (grid[a, 1] == box[3]) & (grid[b, 1] == box[3])}
            any_side = np.zeros(m.tri.shape[0], bool)
            for side, sel in on.items():
                assert (m.bc[sel, e] == tags[side]).all()
                any_side |= sel
            assert (m.bc[~any_side, e] == 0).all()


def test_dmr_states_satisfy_rankine_hugoniot():
    """Across a shock moving with normal speed s = 10 along n: mass, normal
    and tangential momentum and energy fluxes in the shock frame agree."""
    post, pre = W.dmr_states()
    g = W.GAMMA
    n = np.array([math.sin(math.pi / 3), -math.cos(math.pi / 3)])   # normal of a 60-degree line
    s = 10.0

    def fluxes(u):
        rho, m, E = u[0], u[1:3], u[3]
        v = m / rho
        p = (g - 1.0) * (E - 0.5 * rho * v @ v)
        w = v @ n - s
        return np.array([rho * w, rho * w * (v @ n) + p, rho * w * (v @ np.array([-n[1], n[0]])),
                         (E + p) * w + p * s])

    assert np.allclose(fluxes(post), fluxes(pre), rtol=1e-13, atol=1e-12)
    # the printed primitive states
    v_post = post[1:3] / post[0]
    assert post[0] == 8.0 and abs(np.hypot(*v_post) - 8.25) < 1e-13 and abs(v_post @ n - 8.25) < 1e-13
    assert np.allclose(pre, [1.4, 0.0, 0.0, 1.0 / (g - 1.0)])


def test_dmr_workload_recipe():
    wl = W.dmr_workload(nx=24, ny=6, k=2)
    m = wl.mesh
    assert m.xy[:, 0].min() == 0.0 and m.xy[:, 0].max() == 4.0 and m.xy[:, 1].min() == 0.0 and m.xy[:, 1].max() == 1.0
    post, pre = W.dmr_states()
    assert np.array_equal(wl.bc_state[0], post) and np.array_equal(wl.bc_state[1], pre)
    assert wl.shock == (1.0 / 6.0, math.pi / 3.0, 10.0, 1, 0)
    # initial shock through (1/6, 0) at 60 degrees
    y = np.linspace(0.0, 1.0, 11)
    xs = 1.0 / 6.0 + y / math.sqrt(3.0)
    assert np.array_equal(wl.u0(xs - 1e-9, y), np.broadcast_to(post, (11, 4)))
    assert np.array_equal(wl.u0(xs + 1e-9, y), np.broadcast_to(pre, (11, 4)))
    # boundary tags by side
    for e in range(3):
        a, b = m.tri[:, (e + 1) % 3], m.tri[:, (e + 2) % 3]
        xa, ya, xb, yb = m.xy[a, 0], m.xy[a, 1], m.xy[b, 0], m.xy[b, 1]
        left = (xa == 0) & (xb == 0)
        right = (xa == 4) & (xb == 4)
        top = (ya == 1) & (yb == 1)
        bottom = (ya == 0) & (yb == 0)
        assert (m.bc[left, e] == W.BC_DIRICHLET0).all() and (m.bc[right, e] == W.BC_DIRICHLET0 + 1).all()
        assert (m.bc[top, e] == W.BC_SHOCK).all()
        xm = 0.5 * (xa + xb)
        assert (m.bc[bottom & (xm < 1.0 / 6.0), e] == W.BC_DIRICHLET0).all()
        assert (m.bc[bottom & (xm > 1.0 / 6.0), e] == W.BC_REFLECT).all()
    assert (W.dmr_workload(nx=24, ny=6, right=W.BC_TRANSMISSIVE).mesh.bc == W.BC_TRANSMISSIVE).any()


def test_sedov_energy_at_the_origin():
    wl = W.sedov_workload(n=10, k=2)
    m = wl.mesh
    origin = np.flatnonzero((m.xy[:, 0] == 0.0) & (m.xy[:, 1] == 0.0))
    assert origin.size == 1
    touch = np.any(m.tri == origin[0], axis=1)
    u = wl.cell_u0(np.arange(m.nt))
    area = _area(m)
    assert (u[:, 0] == 1.0).all() and (u[:, 1:3] == 0.0).all()
    assert abs((area[touch] * u[touch, 3]).sum() - 0.244816) < 1e-14
    assert np.allclose(u[~touch, 3], 1e-10 / (W.GAMMA - 1.0), rtol=1e-15)
    assert (m.bc[m.bc != 0] == W.BC_REFLECT).all() and abs(m.xy).max() == 1.1


def test_isentropic_vortex():
    rng = np.random.default_rng(0)
    x, y = rng.uniform(0, 1, 500), rng.uniform(0, 1, 500)
    u = W.vortex_state(x, y, 0.0, strength=5.0, radius=0.1)
    rho, vx, vy = u[..., 0], u[..., 1] / u[..., 0], u[..., 2] / u[..., 0]
    p = (W.GAMMA - 1.0) * (u[..., 3] - 0.5 * rho * (vx * vx + vy * vy))
    assert np.allclose(p / rho ** W.GAMMA, 1.0, rtol=1e-12)
    # far from the centre (0.5, 0.5): the free stream (1, 1, 1, 1)
    far = W.vortex_state(np.array([0.0]), np.array([0.0]), 0.0, strength=5.0, radius=0.05)
    assert np.allclose(far[0, :3], [1.0, 1.0, 1.0], atol=1e-9)
    # at the centre the temperature drop is (gamma - 1) eps^2 e / (8 gamma pi^2)
    c = W.vortex_state(np.array([0.5]), np.array([0.5]), 0.0, strength=5.0, radius=0.01)
    T = (W.GAMMA - 1.0) * (c[0, 3] - 0.5 * (c[0, 1] ** 2 + c[0, 2] ** 2) / c[0, 0]) / c[0, 0]
    assert abs(T - (1.0 - 0.4 * 25.0 * math.e / (8.0 * 1.4 * math.pi ** 2))) < 1e-12


def test_riemann4_quadrants():
    wl = W.riemann4_workload(n=8, k=1)
    g = np.linspace(0.05, 0.45, 5)
    for qx in (0, 1):
        for qy in (0, 1):
            xs, ys = np.meshgrid(g + 0.5 * qx, g + 0.5 * qy)
            s = wl.u0(xs.ravel(), ys.ravel())
            assert (s == s[0]).all()
            rho, v = s[0, 0], s[0, 1:3] / s[0, 0]
            p = (W.GAMMA - 1.0) * (s[0, 3] - 0.5 * rho * v @ v)
            assert 0.1 <= rho <= 2.0 and 0.01 <= p <= 2.0 + 1e-12 and (np.abs(v) <= 1.0 + 1e-12).all()
    assert (wl.mesh.bc[wl.mesh.bc != 0] == W.BC_TRANSMISSIVE).all()


def test_batch_and_serving_recipes():
    """Batch: 64 solves, P1/P2 mixed, cells log-uniform in [2k, 200k] (about
    2.8M expected; this seed gives 3.0M).  Serving: Poisson arrivals (times
    increasing), sizes in [1k, 100k], three kinds of data, end times in range."""
    ws = W.batch_workloads()
    cells = np.array([w.mesh.nt for w in ws])
    ks = {w.k for w in ws}
    assert len(ws) == 64 and ks == {1, 2}
    assert cells.min() >= 0.9 * 2000 and cells.max() <= 1.1 * 200000
    assert 2.9e6 < cells.sum() < 3.1e6
    assert all((w.mesh.bc[w.mesh.bc != 0] == W.BC_TRANSMISSIVE).all() for w in ws)
    reqs = W.serving_requests(n=24)
    at = np.array([a for _, _, a in reqs])
    assert (np.diff(at) > 0).all() and at[0] > 0
    assert all(0.005 <= te <= 0.02 for _, te, _ in reqs)
    sizes = np.array([w.mesh.nt for w, _, _ in reqs])
    assert sizes.min() >= 0.9 * 1000 and sizes.max() <= 1.1 * 100000
    kinds = {re.match(r"[a-z]+", w.name).group(0) for w, _, _ in reqs}
    assert kinds == {"vortex", "sedov", "riemann"}

"""GPU parity: each hot-path operator of the CUDA library, called through the
C ABI, against the CPU oracle on the same seeded inputs.

Tolerances: FP64 relative error <= 1e-12 after one operator / stage / step and
<= 1e-9 after 100 steps, relative to the largest oracle magnitude of the
density, the energy and the momentum vector (both momentum components share
one scale: the scheme is rotation invariant).  Integer work (adjacency, limiter vertex ids,
counters) is compared bit-exactly.
"""
import math

import numpy as np
import pytest

from paper_2409_09620_gb300 import workloads as W
from tests.helpers import rel_err

pytestmark = pytest.mark.gpu

TOL1 = 1e-12


@pytest.fixture(scope="module")
def N():
    from paper_2409_09620_gb300 import native
    native.lib()
    return native


def _dmr_small(k, nx=24, ny=8):
    return W.dmr_workload(nx=nx, ny=ny, k=k)


def _cases():
    # (name, workload factory): periodic, reflecting, transmissive, Dirichlet + moving shock
    return {
        "vortex": lambda k: W.vortex_workload(n=13, k=k),          # 338 cells: 3 blocks, ragged tail
        "sedov": lambda k: W.sedov_workload(n=14, k=k),
        "riemann": lambda k: W.riemann4_workload(n=11, k=k),
        "dmr": lambda k: _dmr_small(k),
    }


def _setup(oracle_mod, N, wl, precision=0, **kw):
    O = oracle_mod
    om = O.OracleMesh.from_mesh(wl.mesh)
    u0 = O.project_workload(om, wl)
    mesh = N.Mesh.from_mesh(wl.mesh)
    cfg = N.config_for(wl, precision=precision, **kw)
    solver = N.Solver(mesh, cfg, u0)
    return om, u0, mesh, solver


def _perturbed(u, seed, amp=0.02):
    rng = np.random.default_rng(seed)
    v = u.copy()
    scale = np.abs(u[:, :1, :])
    v[:, 1:, :] += amp * scale * rng.uniform(-1, 1, v[:, 1:, :].shape)
    return v


@pytest.mark.parametrize("k", [1, 2])
@pytest.mark.parametrize("case", ["vortex", "sedov", "dmr"])
def test_geometry_and_adjacency(oracle_mod, N, k, case):
    """Row a0: adjacency bit-exact; geometry and optimal decomposition vs the oracle."""
    O = oracle_mod
    wl = _cases()[case](k)
    om = O.OracleMesh.from_mesh(wl.mesh)
    mesh = N.Mesh.from_mesh(wl.mesh)
    nb_o, ne_o = om.neighbors()
    nb_g, ne_g = mesh.neighbors()
    assert np.array_equal(nb_o, nb_g) and np.array_equal(ne_o, ne_g)
    g = mesh.geometry(k)
    area, ln, nrm = om.geometry()
    np.testing.assert_allclose(g["area"], area, rtol=1e-14)
    np.testing.assert_allclose(g["len"], ln, rtol=1e-14)
    np.testing.assert_allclose(g["normal"], nrm, atol=1e-15)
    V = wl.mesh.xy[wl.mesh.tri]
    for K in range(0, wl.mesh.nt, 3):
        d = om.decomposition(k, K)
        np.testing.assert_allclose(g["c_area"][K], d["c_dcw"] * area[K], rtol=1e-13)
        if k == 1:
            assert list(g["limv"][K]) == list(d["limv"])
        else:
            for s in range(2):
                xi, eta = g["nodes"][K, s]
                p = V[K, 0] + xi * (V[K, 1] - V[K, 0]) + eta * (V[K, 2] - V[K, 0])
                np.testing.assert_allclose(p, d["nodes"][s], atol=1e-14)
    np.testing.assert_allclose(mesh.min_cfl_area(k), om.min_cfl_area(k, 0), rtol=1e-14)
    np.testing.assert_allclose(mesh.min_cfl_area(k, 1), om.min_cfl_area(k, 1), rtol=1e-14)


@pytest.mark.parametrize("k", [1, 2])
def test_projection(oracle_mod, N, k):
    wl = W.vortex_workload(n=9, k=k)
    om = oracle_mod.OracleMesh.from_mesh(wl.mesh)
    mesh = N.Mesh.from_mesh(wl.mesh)
    np.testing.assert_allclose(mesh.quad_points(), om.quad12_points(), atol=1e-15)
    assert rel_err(mesh.project(k, fn=wl.u0), om.project(k, fn=wl.u0)) < 1e-13


@pytest.mark.parametrize("k", [1, 2])
@pytest.mark.parametrize("case", ["vortex", "sedov", "riemann", "dmr"])
def test_rk_stage(oracle_mod, N, k, case):
    """Rows a1 + a2: volume quadrature, edge LF fluxes with neighbour traces or
    boundary ghosts, mass inverse and the RK combination."""
    O = oracle_mod
    wl = _cases()[case](k)
    om, u0, mesh, solver = _setup(O, N, wl)
    cf = O.config_for(wl)
    v = _perturbed(u0, 1)
    un = _perturbed(u0, 2)
    alpha = 1.3 * om.alpha(cf, v, 0.01)
    dt = 0.5 * om.min_cfl_area(k) / alpha
    for (a, b) in [(0.0, 1.0), (0.75, 0.25)]:
        got = solver.op_rk_stage(un, v, a, b, dt, alpha, t=0.01)
        exp = om.rk_stage(cf, un, v, a, b, dt, alpha, t=0.01)
        assert rel_err(got, exp) < TOL1
    # the spatial operator alone: L = (u_h - v) / dt at b = 1
    got = solver.op_rk_stage(un, v, 0.0, 1.0, 1.0, alpha, t=0.01)
    L = om.L(cf, v, alpha, t=0.01)
    assert rel_err(got - v, L) < 1e-11


@pytest.mark.parametrize("k", [1, 2])
@pytest.mark.parametrize("case", ["vortex", "sedov", "dmr"])
def test_oe_stats_and_damping(oracle_mod, N, k, case):
    """Rows a2b + a3: global OE statistics and the RIOE damping."""
    O = oracle_mod
    wl = _cases()[case](k)
    om, u0, mesh, solver = _setup(O, N, wl)
    cf = O.config_for(wl)
    u = _perturbed(u0, 3, amp=0.05)
    st_g = solver.op_stats(u)
    st_o = om.stats(cf, u)
    np.testing.assert_allclose(st_g[:4], st_o[:4], rtol=1e-13, atol=1e-15 * np.abs(st_o[:4]).max())
    np.testing.assert_allclose(st_g[4:], st_o[4:], rtol=1e-12)
    dt = 0.3 * om.min_cfl_area(k) / om.alpha(cf, u)
    got = solver.op_oe(u, dt, st_o, t=0.02)
    exp = om.oe(cf, u, dt, st_o, t=0.02)
    assert np.array_equal(got[:, 0], u[:, 0])
    assert rel_err(got, exp) < TOL1
    assert np.abs(got - u).max() > 0    # damping happened


@pytest.mark.parametrize("k", [1, 2])
def test_component_wise_oe(oracle_mod, N, k):
    O = oracle_mod
    wl = W.riemann4_workload(n=11, k=k)
    om, u0, mesh, solver = _setup(O, N, wl, oe=2)
    cf = O.config_for(wl, oe=2)
    u = _perturbed(u0, 4, amp=0.05)
    st = om.stats(cf, u)
    got = solver.op_oe(u, 0.01, st)
    assert rel_err(got, om.oe(cf, u, 0.01, st)) < TOL1


@pytest.mark.parametrize("k", [1, 2])
@pytest.mark.parametrize("case", ["vortex", "sedov", "riemann"])
def test_limiter(oracle_mod, N, k, case):
    """Row a4: BP limiter at the optimal-decomposition points; counters exact."""
    O = oracle_mod
    wl = _cases()[case](k)
    om, u0, mesh, solver = _setup(O, N, wl)
    cf = O.config_for(wl)
    u = _perturbed(u0, 5, amp=0.8 if k == 1 else 0.4)
    got, cg = solver.op_limit(u)
    exp, co = om.limit(cf, u)
    assert np.array_equal(cg, co) and co[0] > 0
    assert np.array_equal(got[:, 0], u[:, 0])
    assert rel_err(got, exp) < TOL1


@pytest.mark.parametrize("k", [1, 2])
@pytest.mark.parametrize("case", ["vortex", "sedov", "dmr"])
def test_alpha(oracle_mod, N, k, case):
    """Row a5: maximum wave speed at the edge Gauss points (ghosts included)."""
    O = oracle_mod
    wl = _cases()[case](k)
    om, u0, mesh, solver = _setup(O, N, wl)
    cf = O.config_for(wl)
    u = _perturbed(u0, 6, amp=0.01)
    for t in (0.0, 0.05):
        np.testing.assert_allclose(solver.op_alpha(u, t), om.alpha(cf, u, t), rtol=1e-13)


@pytest.mark.parametrize("k", [1, 2])
def test_alpha_extreme_densities(oracle_mod, N, k):
    """Cells whose states are scaled by 1e-160 and 1e+150 (velocity and sound
    speed unchanged): the product of a cell's trace densities leaves the
    normal range, so the kernel takes one division per point instead of the
    batch reciprocal.  alpha still matches the oracle."""
    O = oracle_mod
    wl = _cases()["riemann"](k)
    om, u0, mesh, solver = _setup(O, N, wl)
    cf = O.config_for(wl)
    u = _perturbed(u0, 8, amp=0.01)
    u[:, :, 3] *= 1e-160
    u[:, :, 40] *= 1e150
    np.testing.assert_allclose(solver.op_alpha(u, 0.0), om.alpha(cf, u, 0.0), rtol=1e-13)
    # the scaled cells in a slow quiescent gas (rho 1, p 0.01): they set alpha
    w = np.zeros_like(u)
    w[0, 0] = 1.0
    w[3, 0] = 0.01 / 0.4
    w[:, :, [3, 40]] = u[:, :, [3, 40]]
    a = solver.op_alpha(w, 0.0)
    np.testing.assert_allclose(a, om.alpha(cf, w, 0.0), rtol=1e-13)
    assert a > 0.5


@pytest.mark.parametrize("k", [1, 2])
@pytest.mark.parametrize("case", ["vortex", "sedov", "riemann", "dmr"])
def test_one_step(oracle_mod, N, k, case):
    """All rows: one SSP-RK3 step of the graph-captured solver vs the oracle."""
    O = oracle_mod
    wl = _cases()[case](k)
    om, u0, mesh, solver = _setup(O, N, wl)
    cf = O.config_for(wl)
    st, _ = solver.advance(10.0, max_steps=1)
    ug, tg = solver.get_state()
    uo, to, dto, cnt, rc = om.step(cf, u0, 0.0, 10.0)
    assert rc == 0 and st["steps"] == 1
    np.testing.assert_allclose(tg, to, rtol=1e-13)
    assert rel_err(ug, uo) < TOL1
    assert st["limited_cells"] == cnt[0] and st["cfl_breaches"] == cnt[2]


@pytest.mark.parametrize("k", [1, 2])
def test_hundred_steps_vortex(oracle_mod, N, k):
    """BP RI-OEDG on the isentropic vortex (32 x 32 jittered periodic grid, P1
    is the small configuration of the benchmark family): 100 steps <= 1e-9."""
    O = oracle_mod
    wl = W.vortex_workload(n=32 if k == 1 else 16, k=k)
    om, u0, mesh, solver = _setup(O, N, wl)
    cf = O.config_for(wl)
    solver.advance(10.0, max_steps=100)
    ug, tg = solver.get_state()
    uo, to, cnt, rc = om.advance(cf, u0, 0.0, 10.0, max_steps=100)
    np.testing.assert_allclose(tg, to, rtol=1e-12)
    assert rel_err(ug, uo) < 1e-9


def test_advance_to_end_time(oracle_mod, N):
    """dt clamped to t_end exactly; the whole config-1 run (vortex P1, t = 0.5)."""
    O = oracle_mod
    wl = W.vortex_workload(n=32, k=1)
    om, u0, mesh, solver = _setup(O, N, wl)
    st, _ = solver.advance(wl.t_end)
    ug, tg = solver.get_state()
    assert tg == wl.t_end
    uo, to, cnt, rc = om.advance(O.config_for(wl), u0, 0.0, wl.t_end)
    assert st["steps"] == cnt[3]
    assert rel_err(ug, uo) < 1e-9


def test_deterministic(oracle_mod, N):
    wl = W.sedov_workload(n=20, k=2)
    outs = []
    for _ in range(2):
        om, u0, mesh, solver = _setup(oracle_mod, N, wl)
        solver.advance(10.0, max_steps=5)
        outs.append(solver.get_state()[0])
    assert np.array_equal(outs[0], outs[1])


def test_errors(N):
    xy = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]])
    with pytest.raises(N.DGError) as e:
        N.Mesh(xy, np.zeros((0, 3), np.int32))
    assert e.value.code == N.DG_EINVAL
    with pytest.raises(N.DGError) as e:
        N.Mesh(xy, np.array([[0, 2, 1]], np.int32), None, np.ones((1, 3), np.int8))
    assert e.value.code == N.DG_EMESH
    mesh = N.Mesh(xy, np.array([[0, 1, 2]], np.int32), None, np.ones((1, 3), np.int8))
    u = np.zeros((4, 3, 1))
    u[0, 0] = -1.0
    u[3, 0] = 1.0
    with pytest.raises(N.DGError) as e:
        N.Solver(mesh, N.make_config(1), u)
    assert e.value.code == N.DG_ENONPHYS
    with pytest.raises(N.DGError) as e:
        N.Solver(mesh, N.make_config(3), np.zeros((4, 6, 1)))
    assert e.value.code == N.DG_EINVAL


@pytest.mark.parametrize("k", [1, 2])
@pytest.mark.parametrize("case", ["vortex", "sedov", "dmr"])
def test_classical_decomposition_step(oracle_mod, N, k, case):
    """Classical (Zhang-Xia-Shu) decomposition: its CFL number (Sec. 4.3
    remarks) and limiter point set (Sec. 4.4: edge Gauss points, plus the
    weighted internal state for P2), one step vs the oracle."""
    O = oracle_mod
    wl = _cases()[case](k)
    om, u0, mesh, solver = _setup(O, N, wl, decomp=1)
    cf = O.config_for(wl, decomp=1)
    st, _ = solver.advance(10.0, max_steps=1)
    ug, tg = solver.get_state()
    uo, to, dto, cnt, rc = om.step(cf, u0, 0.0, 10.0)
    assert rc == 0
    np.testing.assert_allclose(tg, to, rtol=1e-13)
    assert rel_err(ug, uo) < TOL1
    u = _perturbed(u0, 8, amp=0.8 if k == 1 else 0.4)
    got, cg = solver.op_limit(u)
    exp, co = om.limit(cf, u)
    assert np.array_equal(cg, co) and co[0] > 0
    assert rel_err(got, exp) < TOL1


@pytest.mark.parametrize("k,lo,hi", [(1, 2.0, 3.0), (2, 3.8038, 4.5)])
def test_bp_time_step_ratio(oracle_mod, N, k, lo, hi):
    """The optimal decomposition's BP time step over the classical one, for
    the same state (the paper's headline gain, Fig. 1744 ranges)."""
    wl = W.dmr_workload(nx=48, ny=12, k=k)
    om, u0, mesh, s_opt = _setup(oracle_mod, N, wl)
    s_zxs = N.Solver(mesh, N.config_for(wl, decomp=1), u0)
    a, _ = s_opt.advance(10.0, max_steps=1)
    b, _ = s_zxs.advance(10.0, max_steps=1)
    r = a["dt_last"] / b["dt_last"]
    assert lo - 1e-9 <= r <= hi + 1e-9
    np.testing.assert_allclose(r, mesh.min_cfl_area(k, 0) / mesh.min_cfl_area(k, 1), rtol=1e-12)


@pytest.mark.parametrize("precision", [0, 1])
def test_profiled_steps_match_graph(oracle_mod, N, precision):
    """dg_profile_steps launches the kernels of a step one by one with events
    around them; the state it leaves is bitwise the state of the same number
    of captured steps, and every kernel kind launches as often as a step has
    it.  20,000 cells make 157 tiles, so the finalize kernels run with two
    tile groups, one of them partial; equality after several steps also shows
    that every ticket counter is back at zero after each launch."""
    wl = W.sedov_workload(n=100, k=2)
    _, _, _, s1 = _setup(oracle_mod, N, wl, precision=precision)
    prof = s1.profile_steps(3)
    assert {k: v[1] for k, v in prof.items()} == {"step_begin": 3, "rk": 9, "fin_mean": 9, "stats": 9,
                                                  "fin_dev": 9, "oe_bp": 9, "fin_alpha": 9}
    assert all(v[0] > 0 for v in prof.values())
    _, _, _, s2 = _setup(oracle_mod, N, wl, precision=precision)
    s2.advance(1e30, max_steps=3)
    u1, t1 = s1.get_state()
    u2, t2 = s2.get_state()
    assert t1 == t2 and t1 > 0
    assert np.array_equal(u1, u2)

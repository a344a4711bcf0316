"""GPU parity on the non-rectangular lattice meshes of Sec. 5: the tunnel
with a forward facing step (inflow, outflow, walls meeting at a re-entrant
corner) and the tube over a 30-degree wedge (inflow, outflow, reflecting
slanted wall, the moving-shock exact solution on the top and on the bottom
before the wedge).  Same tolerances as the rectangular cases: FP64 relative
error <= 1e-12 after one step, <= 1e-9 after 20 steps; the wedge at the
paper's resolution (h = 1/320, 826,173 P2 cells) is compared cell by cell
after one step.
"""
import numpy as np
import pytest

from paper_2409_09620_gb300 import workloads as W
from tests.helpers import rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def N():
    from paper_2409_09620_gb300 import native
    native.lib()
    return native


def _case(name, k):
    return W.ffs_workload(h=1 / 20, k=k) if name == "ffs" else W.wedge_dmr_workload(h=1 / 16, k=k)


def _setup(O, N, wl, **kw):
    om = O.OracleMesh.from_mesh(wl.mesh)
    u0 = O.project_workload(om, wl)
    mesh = N.Mesh.from_mesh(wl.mesh)
    solver = N.Solver(mesh, N.config_for(wl, **kw), u0)
    return om, u0, mesh, solver


@pytest.mark.parametrize("k", [1, 2])
@pytest.mark.parametrize("name", ["ffs", "wedge"])
def test_lattice_mesh_one_and_twenty_steps(oracle_mod, N, name, k):
    O = oracle_mod
    wl = _case(name, k)
    om, u0, mesh, solver = _setup(O, N, wl)
    cf = O.config_for(wl)
    st, _ = solver.advance(10.0, max_steps=1)
    u1, t1 = solver.get_state()
    uo, to, dto, cnt, rc = om.step(cf, u0, 0.0, 10.0)
    assert rc == 0
    np.testing.assert_allclose(t1, to, rtol=1e-13)
    assert rel_err(u1, uo) < 1e-12
    assert st["limited_cells"] == cnt[0]
    solver.advance(10.0, max_steps=19)
    u20, t20 = solver.get_state()
    uo20, to20, cnt20, rc = om.advance(cf, u0, 0.0, 10.0, max_steps=20)
    np.testing.assert_allclose(t20, to20, rtol=1e-12)
    assert rel_err(u20, uo20) < 1e-9


@pytest.mark.parametrize("name", ["ffs", "wedge"])
def test_lattice_mesh_mixed_bounds(oracle_mod, N, name):
    """The mixed-precision form keeps density and pressure of its stored state
    positive at every limiter point through 20 P2 steps."""
    O = oracle_mod
    wl = _case(name, 2)
    om, u0, mesh, solver = _setup(O, N, wl, precision=N.PREC_MIXED)
    solver.advance(10.0, max_steps=20)
    u, _ = solver.get_state()
    mins = om.point_minima(O.config_for(wl), u)
    assert (mins > 0).all()


@pytest.mark.parametrize("k", [1, 2])
@pytest.mark.parametrize("name", ["ffs", "wedge"])
def test_lattice_mesh_time_step_ratio(oracle_mod, N, name, k):
    """Ratio of the BP time steps of the optimal and the classical convex
    decompositions on the same state: the mesh's min C|K| ratio, as the
    oracle computes it."""
    O = oracle_mod
    wl = _case(name, k)
    om, u0, mesh, s_opt = _setup(O, N, wl)
    s_zxs = N.Solver(mesh, N.config_for(wl, decomp=1), u0)
    a, _ = s_opt.advance(10.0, max_steps=1)
    b, _ = s_zxs.advance(10.0, max_steps=1)
    expect = om.min_cfl_area(k, 0) / om.min_cfl_area(k, 1)
    np.testing.assert_allclose(a["dt_last"] / b["dt_last"], expect, rtol=1e-12)


def test_wedge_paper_resolution_one_step(oracle_mod, N):
    O = oracle_mod
    wl = W.wedge_dmr_workload(k=2)
    assert wl.mesh.nt > 800000
    om, u0, mesh, solver = _setup(O, N, wl)
    st, _ = solver.advance(10.0, max_steps=1)
    ug, tg = solver.get_state()
    uo, to, dto, cnt, rc = om.step(O.config_for(wl), u0, 0.0, 10.0)
    assert rc == 0
    np.testing.assert_allclose(tg, to, rtol=1e-13)
    assert rel_err(ug, uo) < 1e-12
    assert st["limited_cells"] == cnt[0]

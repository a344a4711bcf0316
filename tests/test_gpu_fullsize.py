"""GPU parity at the benchmark's full sizes, in the configuration bench.py
times (the graph-captured SSP-RK3 step of the solver):

* the 60-degree double Mach reflection on 1440 x 360 squares (1,036,800 P2
  cells), FP64: one step, every cell compared with the oracle;
* the Sedov-type blast on 256 x 256 squares (131,072 P2 cells, reflecting
  walls, p = 1e-10): one step and ten steps;
* the mixed-precision form on the full DMR: positivity at every limiter
  point of every cell, and the density L1 difference from the oracle.
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


@pytest.fixture(scope="module")
def dmr(oracle_mod):
    wl = W.dmr_workload()
    om = oracle_mod.OracleMesh.from_mesh(wl.mesh)
    u0 = oracle_mod.project_workload(om, wl)
    return wl, om, u0


def test_full_dmr_one_step_fp64(oracle_mod, N, dmr):
    wl, om, u0 = dmr
    assert wl.mesh.nt == 1036800
    mesh = N.Mesh.from_mesh(wl.mesh)
    solver = N.Solver(mesh, N.config_for(wl), u0)
    st, _ = solver.advance(10.0, max_steps=1)
    ug, tg = solver.get_state()
    uo, to, dto, cnt, rc = om.step(oracle_mod.config_for(wl), u0, 0.0, 10.0)
    assert rc == 0
    np.testing.assert_allclose(tg, to, rtol=1e-13)
    assert rel_err(ug, uo) < 1e-12
    assert st["limited_cells"] == cnt[0]


def test_full_dmr_mixed_bounds_and_l1(oracle_mod, N, dmr):
    wl, om, u0 = dmr
    mesh = N.Mesh.from_mesh(wl.mesh)
    solver = N.Solver(mesh, N.config_for(wl, precision=N.PREC_MIXED), u0)
    solver.advance(10.0, max_steps=2)
    ug, _ = solver.get_state()
    cf = oracle_mod.config_for(wl)
    mins = om.point_minima(cf, ug)
    assert (mins[:, 0] > 0).all() and (mins[:, 1] > 0).all()
    uo, t, cnt, rc = om.advance(cf, u0, 0.0, 10.0, max_steps=2)
    area, _, _ = om.geometry()
    l1 = float((np.abs(ug[0, 0] - uo[0, 0]) * area).sum() / (np.abs(uo[0, 0]) * area).sum())
    assert l1 < 1e-6, l1


def test_full_sedov_steps(oracle_mod, N):
    O = oracle_mod
    wl = W.sedov_workload(n=256, k=2)
    assert wl.mesh.nt == 131072
    om = O.OracleMesh.from_mesh(wl.mesh)
    u0 = O.project_workload(om, wl)
    mesh = N.Mesh.from_mesh(wl.mesh)
    solver = N.Solver(mesh, N.config_for(wl), u0)
    cf = O.config_for(wl)
    solver.advance(10.0, max_steps=1)
    u1, t1, _, _, _ = om.step(cf, u0, 0.0, 10.0)
    assert rel_err(solver.get_state()[0], u1) < 1e-12
    solver.advance(10.0, max_steps=9)
    ug, tg = solver.get_state()
    uo, to, cnt, rc = om.advance(cf, u1, t1, 10.0, max_steps=9)
    np.testing.assert_allclose(tg, to, rtol=1e-12)
    assert rel_err(ug, uo) < 1e-9

"""GPU runs to an end time against the oracle (the fully discrete scheme of
Sec. 4.5 over many steps, with the step clamped to the end time).

The 60-degree double Mach reflection (P2, pre-shock state on the right side,
reading R22) on a 160 x 40 grid (12,800 cells) to t = 0.02, several hundred
steps with the shock, its reflection and the limiter active:
  * FP64: state within 1e-9 of the oracle (relative to the largest oracle
    magnitude per quantity), the same number of steps, t = t_end exactly,
    the same limited-cell count, no cell average outside G;
  * mixed form: density L1 difference from the oracle below 1e-5 (relative to
    the oracle's density L1 norm), no cell average outside G, and positive
    density and internal energy at every limiter point of the stored state
    (evaluated in FP64 by the oracle).
"""
import numpy as np
import pytest

from paper_2409_09620_gb300 import workloads as W
from tests.helpers import rel_err

pytestmark = pytest.mark.gpu

T_END = 0.02


@pytest.fixture(scope="module")
def N():
    from paper_2409_09620_gb300 import native
    native.lib()
    return native


@pytest.fixture(scope="module")
def dmr_oracle(oracle_mod):
    O = oracle_mod
    wl = W.dmr_workload(nx=160, ny=40, k=2)
    om = O.OracleMesh.from_mesh(wl.mesh)
    u0 = O.project_workload(om, wl)
    uo, to, cnt, rc = om.advance(O.config_for(wl), u0, 0.0, T_END)
    assert rc == 0 and to == T_END
    return wl, om, u0, uo, cnt


def test_dmr_fp64_to_end_time(N, dmr_oracle):
    wl, om, u0, uo, cnt = dmr_oracle
    mesh = N.Mesh.from_mesh(wl.mesh)
    solver = N.Solver(mesh, N.config_for(wl), u0)
    st, _ = solver.advance(T_END)
    ug, tg = solver.get_state()
    assert tg == T_END and st["steps"] == cnt[3]
    assert st["nonphysical"] == 0
    assert st["limited_cells"] == cnt[0] and cnt[0] > 0
    err = rel_err(ug, uo)
    print(f"DMR 160x40 P2 FP64 to t={T_END}: {st['steps']} steps, max rel err vs oracle {err:.2e}")
    assert err < 1e-9


def test_dmr_mixed_to_end_time(oracle_mod, N, dmr_oracle):
    wl, om, u0, uo, cnt = dmr_oracle
    mesh = N.Mesh.from_mesh(wl.mesh)
    solver = N.Solver(mesh, N.config_for(wl, precision=N.PREC_MIXED), u0)
    st, _ = solver.advance(T_END)
    ug, tg = solver.get_state()
    assert tg == T_END and st["nonphysical"] == 0
    area = mesh.geometry(2)["area"]
    l1 = float((np.abs(ug[0, 0] - uo[0, 0]) * area).sum() / (np.abs(uo[0, 0]) * area).sum())
    mins = om.point_minima(oracle_mod.config_for(wl), ug)
    print(f"DMR 160x40 P2 mixed to t={T_END}: {st['steps']} steps (oracle {cnt[3]}), density L1 vs oracle {l1:.2e}")
    assert l1 < 1e-5
    assert (mins[:, 0] > 0).all() and (mins[:, 1] > 0).all()


@pytest.mark.parametrize("precision", [0, 1])
def test_riemann_with_outflow_sides_to_end_time(oracle_mod, N, precision):
    """A four-quadrant Riemann problem (seeded states as in the serving mix)
    with transmissive sides, P2 on 32 x 32 squares, to t = 0.49: about a
    thousand steps with waves leaving through every side.  The exterior
    state of a transmissive edge is the cell average; the maximum wave speed
    stays at the size of the data's (it grew without bound when the
    interior trace was the exterior).  FP64: the state within 1e-9 of the
    oracle; both forms: no cell average outside G."""
    O = oracle_mod
    wl = W.riemann4_workload(n=32, k=2, seed=1104, t_end=0.49)
    om = O.OracleMesh.from_mesh(wl.mesh)
    u0 = O.project_workload(om, wl)
    mesh = N.Mesh.from_mesh(wl.mesh)
    solver = N.Solver(mesh, N.config_for(wl, precision=precision), u0)
    st, _ = solver.advance(wl.t_end)
    ug, tg = solver.get_state()
    assert tg == wl.t_end and st["nonphysical"] == 0
    assert st["alpha"] < 5.0
    if precision == 0:
        uo, to, cnt, rc = om.advance(O.config_for(wl), u0, 0.0, wl.t_end)
        assert rc == 0 and cnt[3] == st["steps"]
        err = rel_err(ug, uo)
        print(f"Riemann 32x32 P2 FP64 to t={wl.t_end}: {st['steps']} steps, max rel err vs oracle {err:.2e}")
        assert err < 1e-9

"""GPU parity of the scalar OEDG solver (Sec. 2; dg_scalar_*) against the
oracle: one step <= 1e-12 and 20 steps <= 1e-9 relative to the largest
oracle coefficient, for P1-P3, the linear and the Burgers flux, with and
without the OE, on periodic meshes and with inflow / outflow boundaries;
the whole smooth problems to their end times; the error norms the library
computes against the oracle's evaluation."""
import numpy as np
import pytest

from paper_2409_09620_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def N():
    from paper_2409_09620_gb300 import native
    native.lib()
    return native


def rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def _pair(O, N, wl, k, **kw):
    om = O.OracleMesh.from_mesh(wl.mesh)
    u0 = om.sc_project(k, wl.u0)
    cfo = O.make_sc_config(k, flux=wl.flux, bc_state=wl.bc_state, **kw)
    mesh = N.Mesh.from_mesh(wl.mesh)
    cfg = N.make_scalar_config(k, flux=wl.flux, bc_state=wl.bc_state, **kw)
    return om, u0, cfo, mesh, N.ScalarSolver(mesh, cfg, u0)


@pytest.mark.parametrize("k", [1, 2, 3])
@pytest.mark.parametrize("flux", [0, 1])
def test_scalar_one_and_twenty_steps(oracle_mod, N, k, flux):
    O = oracle_mod
    wl = (W.scalar_linear_workload if flux == 0 else W.scalar_burgers_workload)(level=2, k=k)   # 800 cells
    om, u0, cfo, mesh, s = _pair(O, N, wl, k)
    st = s.advance(10.0, max_steps=1)
    u1, t1 = s.get_state()
    uo, to, dto, rc = om.sc_step(cfo, u0, 0.0, 10.0)
    assert rc == 0 and st["steps"] == 1
    np.testing.assert_allclose(t1, to, rtol=1e-13)
    assert rel(u1, uo) < 1e-12
    s.advance(10.0, max_steps=19)
    u20, t20 = s.get_state()
    uo20, to20, n, rc = om.sc_advance(cfo, u0, 0.0, 10.0, max_steps=20)
    np.testing.assert_allclose(t20, to20, rtol=1e-12)
    assert rel(u20, uo20) < 1e-9


@pytest.mark.parametrize("k", [1, 2, 3])
def test_scalar_without_oe(oracle_mod, N, k):
    """Plain RKDG (OE off) on the Burgers problem."""
    O = oracle_mod
    wl = W.scalar_burgers_workload(level=1, k=k)
    om, u0, cfo, mesh, s = _pair(O, N, wl, k, oe=0)
    s.advance(10.0, max_steps=5)
    uo, _, _, _ = om.sc_advance(cfo, u0, 0.0, 10.0, max_steps=5)
    assert rel(s.get_state()[0], uo) < 1e-11


@pytest.mark.parametrize("k", [1, 2, 3])
def test_burgers_riemann_inflow_outflow(oracle_mod, N, k):
    """Burgers Riemann problem II: constant-state inflow on the left and
    bottom (two values), outflow on the right and top; shocks form at once,
    so the OE acts from the first step."""
    O = oracle_mod
    wl = W.burgers_riemann2_workload(n=16, k=k)
    om, u0, cfo, mesh, s = _pair(O, N, wl, k)
    s.advance(10.0, max_steps=1)
    uo1, _, _, _ = om.sc_step(cfo, u0, 0.0, 10.0)
    assert rel(s.get_state()[0], uo1) < 1e-12
    s.advance(10.0, max_steps=19)
    uo, _, _, _ = om.sc_advance(cfo, u0, 0.0, 10.0, max_steps=20)
    assert rel(s.get_state()[0], uo) < 1e-9


@pytest.mark.parametrize("k", [1, 2, 3])
def test_smooth_problem_to_end_time_and_errors(oracle_mod, N, k):
    """The smooth linear problem to t = 0.1: the last step lands on t_end,
    the step counts agree, and the library's L1 / L2 / Linf errors match the
    oracle state's errors computed on the host."""
    O = oracle_mod
    wl = W.scalar_linear_workload(level=1, k=k)
    om, u0, cfo, mesh, s = _pair(O, N, wl, k)
    st = s.advance(wl.t_end)
    ug, tg = s.get_state()
    uo, to, n, rc = om.sc_advance(cfo, u0, 0.0, wl.t_end)
    assert tg == wl.t_end and to == wl.t_end and st["steps"] == n
    assert rel(ug, uo) < 1e-10
    xy = mesh.quad_points()
    exact = wl.exact(xy[..., 0], xy[..., 1], wl.t_end)
    got = np.array(s.errors(exact))
    area, _, _ = om.geometry()
    w = np.array([0.050844906370207] * 3 + [0.116786275726379] * 3 + [0.082851075618374] * 6)
    vals = np.array([[om.sc_eval(k, uo, K, *xy[K, mu]) for mu in range(12)] for K in range(om.nt)])
    e = vals - exact
    want = np.array([(np.abs(e) * w).sum(1) @ area, np.sqrt(((e * e) * w).sum(1) @ area), np.abs(e).max()])
    np.testing.assert_allclose(got, want, rtol=1e-8)


def test_scalar_errors_rejected_configurations(N):
    wl = W.scalar_linear_workload(level=0, k=2)
    mesh = N.Mesh.from_mesh(wl.mesh)
    u0 = N.scalar_project(mesh, 2, wl.u0)
    for bad in (dict(k=4), dict(k=2, rk=4), dict(k=2, flux=5), dict(k=2, cfl=0.0)):
        kk = bad.pop("k")
        with pytest.raises(N.DGError):
            N.ScalarSolver(mesh, N.make_scalar_config(kk, **bad), u0 if kk == 2 else np.zeros((15, mesh.nt)))
    # Euler wall tags are not scalar boundaries
    dmr = W.dmr_workload(nx=8, ny=4, k=1)
    m2 = N.Mesh.from_mesh(dmr.mesh)
    with pytest.raises(N.DGError):
        N.ScalarSolver(m2, N.make_scalar_config(1), np.zeros((3, m2.nt)))


@pytest.mark.parametrize("k", [1, 2, 3])
def test_library_projection_matches_oracle(oracle_mod, N, k):
    wl = W.scalar_burgers_workload(level=1, k=k)
    om = oracle_mod.OracleMesh.from_mesh(wl.mesh)
    mesh = N.Mesh.from_mesh(wl.mesh)
    assert rel(N.scalar_project(mesh, k, wl.u0), om.sc_project(k, wl.u0)) < 1e-13

"""GPU parity on degenerate and boundary-sized meshes: one cell with walls on
every edge, two cells, an 18-cell periodic grid (a cell meets the same
neighbour across a periodic and an interior edge), 8 cells with walls, the
double Mach reflection on 8 cells (walls, inflow and pre-shock states, the
moving shock), exactly one tile of
128 cells, and one tile plus a ragged tail of 4.  One SSP-RK3 step <= 1e-12 and ten steps <= 1e-9
against the oracle in FP64 (counters bit-exact); the mixed form on the same
meshes keeps every cell average admissible."""
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


def _smooth(x, y):
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    rho = 1.0 + 0.3 * np.sin(2.0 * x + 1.0) * np.cos(3.0 * y)
    u = 0.4 + 0.2 * y
    v = -0.3 + 0.1 * x
    p = 1.0 + 0.5 * x * y
    return W.prim_to_cons(rho, u, v, p)


def _custom(name, xy, tri, bc, k):
    xy = np.asarray(xy, np.float64)
    mesh = W.Mesh(xy=xy, tri=np.asarray(tri, np.int32), canon=np.arange(len(xy), dtype=np.int32),
                  bc=np.asarray(bc, np.int8))
    return W.Workload(name=name, mesh=mesh, k=k, t_end=1.0, u0=_smooth)


def _case(name, k):
    if name == "one_cell":
        return _custom(name, [[0.0, 0.0], [1.0, 0.1], [0.3, 0.9]], [[0, 1, 2]], [[1, 1, 1]], k)
    if name == "two_cells":
        return _custom(name, [[0.0, 0.0], [1.0, 0.0], [1.0, 1.0], [0.0, 1.0]], [[0, 1, 2], [0, 2, 3]],
                       [[2, 0, 2], [2, 2, 0]], k)
    if name == "periodic_18":
        return W.vortex_workload(n=3, k=k, radius=0.3)
    if name == "sedov_8":
        return W.sedov_workload(n=2, k=k)
    if name == "dmr_8":
        return W.dmr_workload(nx=2, ny=2, k=k)
    if name == "one_tile":
        return W.riemann4_workload(n=8, k=k)          # 128 cells
    if name == "two_tiles_ragged":
        return W.dmr_workload(nx=33, ny=2, k=k)       # 132 cells
    raise KeyError(name)


CASES = ["one_cell", "two_cells", "periodic_18", "sedov_8", "dmr_8", "one_tile", "two_tiles_ragged"]


def _setup(O, N, wl, precision=0):
    om = O.OracleMesh.from_mesh(wl.mesh)
    u0 = O.project_workload(om, wl)
    mesh = N.Mesh.from_mesh(wl.mesh)
    return om, u0, mesh, N.Solver(mesh, N.config_for(wl, precision=precision), u0)


@pytest.mark.parametrize("k", [1, 2])
@pytest.mark.parametrize("case", CASES)
def test_degenerate_mesh_steps(oracle_mod, N, case, k):
    O = oracle_mod
    wl = _case(case, k)
    om, u0, mesh, solver = _setup(O, N, wl)
    assert mesh.nt == wl.mesh.nt
    cf = O.config_for(wl)
    st, _ = solver.advance(10.0, max_steps=1)
    ug, tg = solver.get_state()
    uo, to, dto, cnt, rc = om.step(cf, u0, 0.0, 10.0)
    assert rc == 0 and st["steps"] == 1
    np.testing.assert_allclose(tg, to, rtol=1e-13)
    assert rel_err(ug, uo) < 1e-12
    assert st["limited_cells"] == cnt[0] and st["cfl_breaches"] == cnt[2]
    solver.advance(10.0, max_steps=9)
    ug10, tg10 = solver.get_state()
    uo10, to10, cnt10, rc10 = om.advance(cf, u0, 0.0, 10.0, max_steps=10)
    assert rc10 == 0
    np.testing.assert_allclose(tg10, to10, rtol=1e-12)
    assert rel_err(ug10, uo10) < 1e-9


@pytest.mark.parametrize("k", [1, 2])
@pytest.mark.parametrize("case", CASES)
def test_degenerate_mesh_mixed(oracle_mod, N, case, k):
    O = oracle_mod
    wl = _case(case, k)
    om, u0, mesh, solver = _setup(O, N, wl, precision=1)
    st, _ = solver.advance(10.0, max_steps=10)
    assert st["steps"] == 10 and st["nonphysical"] == 0
    u, _ = solver.get_state()
    rho, m1, m2, E = u[0, 0], u[1, 0], u[2, 0], u[3, 0]
    assert np.all(rho > 0) and np.all(E - 0.5 * (m1 * m1 + m2 * m2) / rho > 0)
    s64 = _setup(O, N, wl)[3]
    s64.advance(10.0, max_steps=10)
    u64, _ = s64.get_state()
    assert rel_err(u[:, :1], u64[:, :1]) < 1e-4


def test_periodic_two_by_two_rejected(oracle_mod, N):
    """On a 2 x 2 periodic grid the identified boundary vertices make four
    edges share one pair of vertices: not a manifold mesh.  The library and
    the oracle both reject it."""
    wl = W.vortex_workload(n=2, k=1)
    with pytest.raises(N.DGError) as e:
        N.Mesh.from_mesh(wl.mesh)
    assert e.value.code == N.DG_EMESH
    with pytest.raises(ValueError):
        oracle_mod.OracleMesh.from_mesh(wl.mesh)


@pytest.mark.parametrize("form", [3, 1, 0])
@pytest.mark.parametrize("precision", [0, 1])
def test_degenerate_meshes_in_a_batch(oracle_mod, N, precision, form):
    """A batch of the tiny meshes (1, 2, 8 and 132 cells, P1 and P2) is
    bitwise the solves run alone, in every launch form, and matches the
    oracle."""
    from tests.test_gpu_batch import check_against_oracle
    wls = [_case("one_cell", 1), _case("two_cells", 2), _case("dmr_8", 2), _case("two_tiles_ragged", 1)]
    O = oracle_mod
    meshes = [N.Mesh.from_mesh(w.mesh) for w in wls]
    us = [O.project_workload(O.OracleMesh.from_mesh(w.mesh), w) for w in wls]
    cfgs = [N.config_for(w, precision=precision) for w in wls]
    batch = N.Batch(meshes, cfgs, us)
    batch.set_shape(128, 4, form)
    st = batch.advance(None, max_steps=6)
    assert all(s["steps"] == 6 for s in st)
    for i in range(len(wls)):
        solo = N.Solver(meshes[i], cfgs[i], us[i])
        solo.advance(1e30, max_steps=6)
        a, ta = batch.solver(i).get_state()
        b, tb = solo.get_state()
        assert ta == tb and np.array_equal(a, b), i
        check_against_oracle(O, wls[i], us[i], a, ta, 6, precision)

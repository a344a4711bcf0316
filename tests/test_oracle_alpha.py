"""Pins of the oracle's viscosity coefficient alpha and of its BP time step.

alpha is the largest spectral radius R(u, n) = |v . n| + c over every cell,
edge and edge Gauss point, for the interior trace and for the exterior state
of a boundary edge (eq. 1250, with reading R4: both traces at the edge Gauss
points).  The time step is dt = cfl min_K(C_K |K|) / alpha, clamped to the end
time (Sec. 5; reading R9).

The expected values below come from primitive variables chosen so that the
answer has a closed form: a uniform state on a jittered periodic mesh, and
cells whose state has a linear density at constant velocity and pressure
(all four conserved variables are then linear, so the P1 and P2 projections
are exact): a single cell under each kind of boundary, and a periodic mesh
whose cells each hold their own such state.  Normals and Gauss points are
computed here from the vertex coordinates and numpy's Gauss-Legendre nodes,
not by the oracle.

A last test compiles copies of the oracle with plausible mistakes planted in
alpha or dt (sound speed dropped, boundary exterior states left out, the
cell average instead of the edge points, a wrong edge normal, the classical
decomposition's CFL area) and checks that these pins catch every one.
"""
import math
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_2409_09620_gb300 import workloads as W
from tests.helpers import single_cell

GAMMA = 1.4
HERE = os.path.dirname(os.path.abspath(__file__))
ORACLE = os.path.join(os.path.dirname(HERE), "oracle")


def _cons(rho, vx, vy, p):
    return np.stack(np.broadcast_arrays(rho, rho * vx, rho * vy, p / (GAMMA - 1.0) + 0.5 * rho * (vx * vx + vy * vy)),
                    axis=-1)


def _spectral_radius(rho, vx, vy, p, n):
    """|v . n| + sqrt(gamma p / rho) from primitive variables."""
    return abs(vx * n[0] + vy * n[1]) + math.sqrt(GAMMA * p / rho)


def _outward_normals(V):
    """Unit outward normal of edge i (opposite vertex i, from v_{i+1} to v_{i+2}) of a CCW triangle."""
    out = []
    for i in range(3):
        a, b = V[(i + 1) % 3], V[(i + 2) % 3]
        d = b - a
        out.append(np.array([d[1], -d[0]]) / math.hypot(d[0], d[1]))
    return out


def _edge_points(V, i, Q):
    x, _ = np.polynomial.legendre.leggauss(Q)
    s = 0.5 * (1.0 + x)
    a, b = V[(i + 1) % 3], V[(i + 2) % 3]
    return [a + (b - a) * sv for sv in s]


# --------------------------------------------------------------------------
# checks, shared by the pins and by the planted-mistake test
# --------------------------------------------------------------------------
def check_alpha_uniform(O, k):
    """Uniform state on a jittered periodic mesh: alpha = max over all cells and
    edges of |v . n_i| + c, with the normals computed from the vertices."""
    mesh = W.jittered_grid(9, 7, seed=81, periodic=True)
    om = O.OracleMesh.from_mesh(mesh)
    rho, vx, vy, p = 1.3, 0.37, -0.61, 0.8
    nb = 3 if k == 1 else 6
    u = np.zeros((4, nb, mesh.nt))
    u[:, 0, :] = _cons(rho, vx, vy, p)[:, None]
    got = om.alpha(O.make_config(k), u, 0.0)
    best = 0.0
    for K in range(mesh.nt):
        V = mesh.xy[mesh.tri[K]]
        for n in _outward_normals(V):
            best = max(best, _spectral_radius(rho, vx, vy, p, n))
    speed = math.hypot(vx, vy) + math.sqrt(GAMMA * p / rho)
    assert speed - best > 1e-6 * speed, "no normal may be parallel to v for this pin to see the projection"
    assert abs(got - best) <= 4e-16 * best, (got, best)
    del om


def check_alpha_piecewise_linear(O, k):
    """Every cell of a jittered periodic mesh holds its own linear density at
    its own constant velocity and pressure (discontinuous across edges):
    alpha = max over cells K, edges i and the Gauss points of edge i of
    |v_K . n_i| + sqrt(gamma p_K / rho_K(x)).  The neighbour's trace at the same
    point is its own cell's term with the opposite normal, so it needs no
    separate entry."""
    mesh = W.jittered_grid(6, 5, seed=83, periodic=True)
    om = O.OracleMesh.from_mesh(mesh)
    rng = np.random.default_rng(84)
    nt = mesh.nt
    cen = mesh.xy[mesh.tri].mean(axis=1)
    r0 = rng.uniform(0.8, 1.6, nt)
    gr = rng.uniform(-2.0, 2.0, (nt, 2))
    vel = rng.uniform(-1.0, 1.0, (nt, 2))
    pr = rng.uniform(0.3, 2.0, nt)

    def rho_at(K, x, y):
        return r0[K] + gr[K, 0] * (x - cen[K, 0]) + gr[K, 1] * (y - cen[K, 1])

    cells = np.arange(nt)[:, None]
    u = om.project(k, fn=lambda x, y: _cons(rho_at(cells, x, y), vel[cells, 0], vel[cells, 1], pr[cells]))
    got = om.alpha(O.make_config(k), u, 0.0)
    best = 0.0
    for K in range(nt):
        V = mesh.xy[mesh.tri[K]]
        for i, n in enumerate(_outward_normals(V)):
            for P in _edge_points(V, i, k + 1):
                assert rho_at(K, *P) > 0.1
                best = max(best, _spectral_radius(rho_at(K, *P), vel[K, 0], vel[K, 1], pr[K], n))
    assert abs(got - best) <= 1e-14 * best, (got, best)
    del om


def _cell_case(tag):
    V = np.array([[0.05, -0.1], [1.1, 0.15], [0.3, 0.95]])
    # linear density at constant velocity and pressure
    g = (0.9, -0.7)
    rho = lambda x, y: 1.2 + g[0] * x + g[1] * y          # noqa: E731  (0.53 ... 2.12 on the cell)
    v0, p0 = (0.8, -0.45), 0.6
    bc_state = np.zeros((4, 4))
    bc_state[0] = _cons(0.4, -2.0, 1.5, 3.0)               # Dirichlet exterior, R up to 6.4
    bc_state[1] = _cons(0.7, 0.1, 0.0, 0.2)                # pre-shock: slower than the interior
    bc_state[2] = _cons(1.5, 1.9, -3.2, 9.0)               # post-shock: faster, direction-dependent
    shock = (0.2, math.radians(60.0), 2.5, 1, 2)           # x0, angle, speed, pre, post
    return V, rho, v0, p0, bc_state, shock


def _cell_expected(tag, k, t, with_ghost=True):
    V, rho, v0, p0, bc_state, shock = _cell_case(tag)
    best = 0.0
    for i, n in enumerate(_outward_normals(V)):
        for P in _edge_points(V, i, k + 1):
            best = max(best, _spectral_radius(rho(*P), v0[0], v0[1], p0, n))
            if not with_ghost:
                continue
            if tag == 3:
                s = bc_state[0]
            elif tag == 7:
                x0, ang, spd, pre, post = shock
                xs = x0 + P[1] / math.tan(ang) + spd * t / math.sin(ang)
                s = bc_state[post if P[0] < xs else pre]
            elif tag == 2:   # transmissive: the cell average (density at the centroid, same v and p)
                s = _cons(rho(*V.mean(axis=0)), v0[0], v0[1], p0)
            else:   # a mirror of the interior has the same spectral radius
                continue
            r = s[0]
            vx, vy = s[1] / r, s[2] / r
            pe = (GAMMA - 1.0) * (s[3] - 0.5 * r * (vx * vx + vy * vy))
            best = max(best, _spectral_radius(r, vx, vy, pe, n))
    return best


def check_alpha_single_cell(O, k, tag, t=0.05):
    V, rho, v0, p0, bc_state, shock = _cell_case(tag)
    Vv, tri, bc = single_cell(V, tag=tag)
    om = O.OracleMesh(Vv, tri, None, bc)
    u = om.project(k, fn=lambda x, y: _cons(rho(x, y), v0[0], v0[1], p0))
    cf = O.make_config(k, bc_state=bc_state, shock=shock)
    got = om.alpha(cf, u, t)
    exp = _cell_expected(tag, k, t)
    assert abs(got - exp) <= 1e-14 * exp, (tag, got, exp)
    del om


def check_step_dt(O, k, cfl=0.6):
    """One step of a uniform state: dt = cfl min_K(C_K |K|) / alpha, with alpha in
    closed form and C_K the decomposition's CFL number of each cell; a step
    that would pass t_end is clamped to it."""
    mesh = W.jittered_grid(9, 7, seed=82, periodic=True)
    om = O.OracleMesh.from_mesh(mesh)
    rho, vx, vy, p = 0.9, -0.3, 0.52, 1.7
    nb = 3 if k == 1 else 6
    u = np.zeros((4, nb, mesh.nt))
    u[:, 0, :] = _cons(rho, vx, vy, p)[:, None]
    alpha = 0.0
    min_ca = math.inf
    for K in range(mesh.nt):
        V = mesh.xy[mesh.tri[K]]
        for n in _outward_normals(V):
            alpha = max(alpha, _spectral_radius(rho, vx, vy, p, n))
        area = 0.5 * ((V[1, 0] - V[0, 0]) * (V[2, 1] - V[0, 1]) - (V[2, 0] - V[0, 0]) * (V[1, 1] - V[0, 1]))
        min_ca = min(min_ca, om.decomposition(k, K)["c_dcw"] * area)
    cf = O.make_config(k, cfl=cfl)
    _, t1, dt, _, rc = om.step(cf, u, 0.25, 1e9)
    exp = cfl * min_ca / alpha
    assert rc == 0
    assert abs(dt - exp) <= 1e-14 * exp, (dt, exp)
    assert t1 == 0.25 + dt
    # the last step ends exactly at t_end
    _, t2, dt2, _, rc = om.step(cf, u, 0.25, 0.25 + 0.5 * exp)
    assert rc == 0 and t2 == 0.25 + 0.5 * exp and dt2 == (0.25 + 0.5 * exp) - 0.25
    del om


# --------------------------------------------------------------------------
# the pins
# --------------------------------------------------------------------------
@pytest.mark.parametrize("k", [1, 2])
def test_alpha_uniform_state(oracle_mod, k):
    check_alpha_uniform(oracle_mod, k)


@pytest.mark.parametrize("k", [1, 2])
def test_alpha_piecewise_linear_cells(oracle_mod, k):
    check_alpha_piecewise_linear(oracle_mod, k)


@pytest.mark.parametrize("tag", [1, 2, 3, 7])
@pytest.mark.parametrize("k", [1, 2])
def test_alpha_single_cell(oracle_mod, k, tag):
    check_alpha_single_cell(oracle_mod, k, tag)


def test_alpha_single_cell_cases_discriminate():
    """The single-cell cases are built so that the exterior states and the
    shock's time both change the answer (otherwise the pins could not see
    those mistakes), and the edge points differ from the cell average."""
    for k in (1, 2):
        assert _cell_expected(3, k, 0.05) > 1.2 * _cell_expected(3, k, 0.05, with_ghost=False)
        assert _cell_expected(7, k, 0.05) > 1.05 * _cell_expected(7, k, 0.05, with_ghost=False)
        assert abs(_cell_expected(7, k, 0.05) - _cell_expected(7, k, 0.0)) > 1e-3
        V, rho, v0, p0, _, _ = _cell_case(2)
        c = V.mean(axis=0)
        at_avg = max(_spectral_radius(rho(*c), v0[0], v0[1], p0, n) for n in _outward_normals(V))
        assert _cell_expected(2, k, 0.0) > 1.05 * at_avg


@pytest.mark.parametrize("k", [1, 2])
def test_step_time_step(oracle_mod, k):
    check_step_dt(oracle_mod, k)


# --------------------------------------------------------------------------
# planted mistakes, compiled into copies of the oracle on the CPU
# --------------------------------------------------------------------------
MUTANTS = {
    "no_sound_speed": ("return fabs(u[1] * n[0] + u[2] * n[1]) / u[0] + sqrt(gamma * p / u[0]);",
                       "return fabs(u[1] * n[0] + u[2] * n[1]) / u[0];"),
    "no_exterior": ("      if (m->nbr[3 * K + i] < 0) {\n        double uex[4], ubar[4];",
                    "      if (0) {\n        double uex[4], ubar[4];"),
    "cell_average": ("      eval_at(m, cf->k, u, K, &g, x, y, uin);\n      double r = wave_speed",
                     "      eval_at(m, cf->k, u, K, &g, (g.v[0][0] + g.v[1][0] + g.v[2][0]) / 3.0,\n"
                     "              (g.v[0][1] + g.v[1][1] + g.v[2][1]) / 3.0, uin);\n      double r = wave_speed"),
    "wrong_normal": ("      double r = wave_speed(uin, g.n[i], cf->gamma);",
                     "      double r = wave_speed(uin, g.n[(i + 1) % 3], cf->gamma);"),
    "zxs_cfl_area": ("double min_ca = or_min_cfl_area(m, k, cf->decomp);",
                     "double min_ca = or_min_cfl_area(m, k, 1);"),
}


def _build_mutant(tmp, name):
    src = open(os.path.join(ORACLE, "oracle.c")).read()
    old, new = MUTANTS[name]
    assert src.count(old) == 1, f"mutation site of {name} not found once"
    d = tmp / name
    d.mkdir()
    for f in os.listdir(ORACLE):
        if f.endswith((".c", ".h")):
            shutil.copy(os.path.join(ORACLE, f), d / f)
    (d / "oracle.c").write_text(src.replace(old, new))
    so = str(d / "liboracle.so")
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-w",
                           "-o", so, str(d / "oracle.c"), str(d / "scalar.c"), "-lm"])
    return so


@pytest.mark.slow
def test_planted_mistakes_are_caught(oracle_mod, tmp_path, monkeypatch):
    if shutil.which("gcc") is None:
        pytest.skip("no gcc")
    O = oracle_mod
    real = O.lib()
    checks = [lambda: [check_alpha_uniform(O, k) for k in (1, 2)],
              lambda: [check_alpha_piecewise_linear(O, k) for k in (1, 2)],
              lambda: [check_alpha_single_cell(O, k, tag) for k in (1, 2) for tag in (1, 2, 3, 7)],
              lambda: [check_step_dt(O, k) for k in (1, 2)]]
    import ctypes
    for name in MUTANTS:
        so = _build_mutant(tmp_path, name)
        # same entry points and argument types, different library
        mut = ctypes.CDLL(so)
        for fn in ("or_mesh_create", "or_mesh_destroy", "or_alpha", "or_project", "or_quad12_points",
                   "or_step", "or_decomposition", "or_min_cfl_area"):
            f = getattr(mut, fn)
            f.argtypes = getattr(real, fn).argtypes
            f.restype = getattr(real, fn).restype
        monkeypatch.setattr(O, "_lib", mut)
        caught = 0
        for chk in checks:
            try:
                chk()
            except AssertionError:
                caught += 1
        monkeypatch.setattr(O, "_lib", real)
        assert caught >= 1, f"planted mistake {name} passed every alpha / dt pin"
    # and the real oracle passes all of them
    for chk in checks:
        chk()

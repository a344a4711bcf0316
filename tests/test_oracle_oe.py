"""Pins of the oracle's OE procedure (Sec. 2.3 and 3.2-3.3): damping
coefficients recomputed by hand from exact polynomial derivatives, the exact
solution of the damping ODE, and the invariance theorems."""
import math

import numpy as np
import pytest

from paper_2409_09620_gb300 import workloads as W
from tests.helpers import PhysPoly, rotate_mesh_state, tri_integral

G = 1.4


def wave_speed(u, n):
    rho, m1, m2, E = u
    p = max((G - 1) * (E - 0.5 * (m1 * m1 + m2 * m2) / rho), 0.0)
    return abs(m1 * n[0] + m2 * n[1]) / rho + math.sqrt(G * p / rho)


def _cell_polys(mesh, k, rng, amp=0.05):
    polys = []
    for K in range(mesh.nt):
        base = [1.2, 0.3, -0.2, 3.0]
        polys.append([PhysPoly.random(k, rng, amp * max(1.0, abs(b))) + PhysPoly({(0, 0): b}) for b in base])
    return polys


def _project_cellwise(om, k, polys):
    xy = om.quad12_points()
    vals = np.zeros((om.nt, 12, 4))
    for K in range(om.nt):
        for c in range(4):
            vals[K, :, c] = polys[K][c](xy[K, :, 0], xy[K, :, 1])
    return om.project_values(k, vals)


def _derivs(p, j, x, y):
    """d^alpha p at (x, y) for |alpha| = j, listed with alpha_1 = j, ..., 0."""
    return np.array([p.d(a, j - a)(x, y) for a in range(j, -1, -1)])


@pytest.mark.parametrize("k", [1, 2])
def test_sigma_by_hand(oracle_mod, k):
    """sigma^j = sum_i beta_i / h_i delta_i^j with delta from the trapezoidal
    rule of the jumps of all derivatives of order j (RIOE, eqs. oe:sysdelta2,
    RIOESys:CoefM/Coef1/Coef2), h_i = 2|K| / l_i, A^{k,j} = (2j+1)/((2k-1) j!)."""
    O = oracle_mod
    rng = np.random.default_rng(40 + k)
    mesh = W.jittered_grid(5, 4, (0, 1, 0, 1), seed=17,
                           side_tags={s: W.BC_TRANSMISSIVE for s in ("left", "right", "bottom", "top")})
    om = O.OracleMesh.from_mesh(mesh)
    polys = _cell_polys(mesh, k, rng)
    u = _project_cellwise(om, k, polys)
    cf = O.make_config(k, oe=1)
    st = om.stats(cf, u)
    _, sig = om.oe(cf, u, dt=0.01, stats=st, want_sigma=True)
    nbr, _ = om.neighbors()
    area, ln, nrm = om.geometry()
    D = {"rho": st[4], "m": st[5], "E": st[6]}
    for K in range(mesh.nt):
        V = mesh.xy[mesh.tri[K]]
        expect = np.zeros((4, 3))
        for i in range(3):
            n = nrm[K, i]
            h = 2 * area[K] / ln[K, i]
            N = nbr[K, i]
            # a transmissive edge's exterior is the constant cell average (exact integral / |K|)
            other = polys[N] if N >= 0 else [PhysPoly({(0, 0): tri_integral(pc, V) / area[K]}) for pc in polys[K]]
            J = np.zeros((4, 3))
            beta = 0.0
            for vv in ((i + 1) % 3, (i + 2) % 3):
                x, y = V[vv]
                uo = np.array([p(x, y) for p in polys[K]])
                un = np.array([p(x, y) for p in other])
                beta = max(beta, wave_speed(uo, n), wave_speed(un, n))
                for j in range(k + 1):
                    jump = [_derivs(polys[K][c], j, x, y) - _derivs(other[c], j, x, y) for c in range(4)]
                    mn = jump[1] * n[0] + jump[2] * n[1]
                    mt = -jump[1] * n[1] + jump[2] * n[0]
                    w = np.array([math.comb(j, j - a) for a in range(j + 1)])
                    for q, d in enumerate([jump[0], mn, mt, jump[3]]):
                        J[q, j] += 0.5 * (w * d * d).sum()
            for j in range(k + 1):
                A = (2 * j + 1) / ((2 * k - 1) * math.factorial(j))
                dl = [A * h ** j * math.sqrt(J[q, j]) / D[name] for q, name in enumerate(["rho", "m", "m", "E"])]
                dm = max(dl[1], dl[2])
                expect[:, j] += beta / h * np.array([dl[0], dm, dm, dl[3]])
        np.testing.assert_allclose(sig[:, :, K], expect, rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("k", [1, 2])
def test_damping_is_exact_ode_solution(oracle_mod, k):
    """eq. (OE:m0) and the solution of the damping equation (DGSystem:OE):
    mode 0 is kept bitwise; a mode of degree m is multiplied by
    exp(-dt sum_{j<=m} sigma^j)."""
    O = oracle_mod
    mesh = W.jittered_grid(6, 6, seed=18, periodic=True)
    om = O.OracleMesh.from_mesh(mesh)
    u = W.random_modal_state(mesh.nt, k, seed=19, amp=0.05)
    cf = O.make_config(k)
    _, sig0 = om.oe(cf, u, 1.0, want_sigma=True)          # sigma does not depend on dt
    dt = 3.0 / sig0.sum(1).max()                          # strongest damping exp(-3)
    out, sig = om.oe(cf, u, dt, want_sigma=True)
    assert np.array_equal(out[:, 0], u[:, 0])
    deg = [0, 1, 1, 2, 2, 2]
    for l in range(1, u.shape[1]):
        # integrate du/dtau = -sum_{j<=m} sigma^j u with RK4 on a fine pseudo-time grid
        lam = sig[:, : deg[l] + 1, :].sum(1)
        y = u[:, l, :].copy()
        nsub = 1000
        h = dt / nsub
        for _ in range(nsub):
            k1 = -lam * y; k2 = -lam * (y + h / 2 * k1); k3 = -lam * (y + h / 2 * k2); k4 = -lam * (y + h * k3)
            y = y + h / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
        np.testing.assert_allclose(out[:, l, :], y, rtol=1e-9, atol=1e-14)
    assert sig[:, 1:, :].max() > 0    # the test exercises real damping


@pytest.mark.parametrize("k", [1, 2])
def test_oe_identity_cases(oracle_mod, k):
    """Constant state (delta = 0, eq. OEScalar:Coef2) and a globally smooth
    polynomial (no jumps across interior edges) leave the state unchanged;
    on a mesh with transmissive sides this holds for the cells away from the
    boundary, whose exterior there is the cell average (so boundary cells
    with a non-constant polynomial are damped)."""
    O = oracle_mod
    wl = W.uniform_workload(n=6, k=k)
    om = O.OracleMesh.from_mesh(wl.mesh)
    u = om.project(k, fn=wl.u0)
    cf = O.make_config(k)
    assert np.array_equal(om.oe(cf, u, 0.1), u)
    rng = np.random.default_rng(22)
    mesh = W.jittered_grid(6, 5, seed=23, side_tags={s: W.BC_TRANSMISSIVE for s in ("left", "right", "bottom", "top")})
    om = O.OracleMesh.from_mesh(mesh)
    ps = [PhysPoly.random(k, rng, 0.1) + PhysPoly({(0, 0): b}) for b in (1.0, 0.2, 0.1, 2.5)]
    u = om.project(k, fn=lambda x, y: np.stack([p(x, y) for p in ps], -1))
    out = om.oe(cf, u, 0.1)
    nbr, _ = om.neighbors()
    inner = (nbr >= 0).all(1)
    assert inner.sum() > 0 and (~inner).sum() > 0
    assert np.abs(out[:, :, inner] - u[:, :, inner]).max() < 1e-13
    assert np.array_equal(out[:, 0], u[:, 0])
    assert np.abs(out[:, 1:, ~inner] - u[:, 1:, ~inner]).max() > 1e-6


@pytest.mark.parametrize("k", [1, 2])
def test_oe_scale_invariance(oracle_mod, k):
    """Sec. 2.4: F(a u) = a F(u) (velocities and sound speed are unchanged by
    scaling all conservative variables)."""
    O = oracle_mod
    mesh = W.jittered_grid(6, 6, seed=24, periodic=True)
    om = O.OracleMesh.from_mesh(mesh)
    u = W.random_modal_state(mesh.nt, k, seed=25, amp=0.2)
    cf = O.make_config(k)
    a = 3.7
    np.testing.assert_allclose(om.oe(cf, a * u, 0.02), a * om.oe(cf, u, 0.02), rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("k", [1, 2])
def test_rioe_rotation_invariance(oracle_mod, k):
    """Thm (Rotational Invariance): sigma of RIOE is unchanged by rotating mesh
    and state; the component-wise OE is not rotation invariant (Sec. 3.2)."""
    O = oracle_mod
    mesh = W.jittered_grid(7, 6, seed=26, periodic=True)
    om = O.OracleMesh.from_mesh(mesh)
    u = W.random_modal_state(mesh.nt, k, seed=27, amp=0.05)
    errs = {}
    for oe in (1, 2):
        cf = O.make_config(k, oe=oe)
        out, sig = om.oe(cf, u, 0.05, want_sigma=True)
        for phi in (math.pi / 2, math.pi / 4):
            xy, ur = rotate_mesh_state(mesh, u, phi)
            omr = O.OracleMesh(xy, mesh.tri, mesh.canon, mesh.bc)
            outr, sigr = omr.oe(cf, ur, 0.05, want_sigma=True)
            _, outrot = rotate_mesh_state(mesh, out, phi)
            errs[(oe, phi)] = (np.abs(sigr - sig).max() / np.abs(sig).max(),
                               np.abs(outr - outrot).max() / np.abs(out).max())
    assert errs[(1, math.pi / 2)][0] < 1e-13 and errs[(1, math.pi / 2)][1] < 1e-14
    assert errs[(1, math.pi / 4)][0] < 1e-13 and errs[(1, math.pi / 4)][1] < 1e-14
    assert errs[(2, math.pi / 4)][0] > 1e-3      # CW-OE breaks rotation invariance


def test_reflecting_wall_ghost_is_mirror(oracle_mod):
    """Reading of the OE at a reflecting wall: the exterior polynomial is the
    mirror image (rho, E even; m reflected).  Checked with sympy by building the
    mirrored polynomial explicitly on a single cell."""
    sp = pytest.importorskip("sympy")
    O = oracle_mod
    k = 2
    V = np.array([[0.1, 0.0], [1.0, 0.2], [0.3, 0.9]])
    om = O.OracleMesh(V, np.array([[0, 1, 2]], np.int32), None, np.full((1, 3), W.BC_REFLECT, np.int8))
    rng = np.random.default_rng(31)
    x, y = sp.symbols("x y")
    polys = [PhysPoly.random(k, rng, 0.1) + PhysPoly({(0, 0): b}) for b in (1.0, 0.3, -0.2, 2.5)]
    exprs = [sum(c * x ** a * y ** b for (a, b), c in p.c.items()) for p in polys]
    u = om.project(k, fn=lambda X, Y: np.stack([p(X, Y) for p in polys], -1))
    cf = O.make_config(k)
    st = np.array([1.0, 0.3, -0.2, 2.5, 0.7, 0.9, 1.1, 1.0, 0.5, 0.5])   # any positive normalisers
    _, sig = om.oe(cf, u, 0.01, stats=st, want_sigma=True)
    area, ln, nrm = om.geometry()
    expect = np.zeros((4, 3))
    for i in range(3):
        n = nrm[0, i]
        P = V[(i + 1) % 3]
        R = np.eye(2) - 2 * np.outer(n, n)
        # mirror map x -> P + R (x - P)
        xr = P[0] + R[0, 0] * (x - P[0]) + R[0, 1] * (y - P[1])
        yr = P[1] + R[1, 0] * (x - P[0]) + R[1, 1] * (y - P[1])
        mir = [e.subs({x: xr, y: yr}, simultaneous=True) for e in exprs]
        ghost = [mir[0], R[0, 0] * mir[1] + R[0, 1] * mir[2], R[1, 0] * mir[1] + R[1, 1] * mir[2], mir[3]]
        h = 2 * area[0] / ln[0, i]
        J = np.zeros((4, 3))
        beta = 0.0
        for vv in ((i + 1) % 3, (i + 2) % 3):
            pt = {x: V[vv, 0], y: V[vv, 1]}
            uo = np.array([float(e.subs(pt)) for e in exprs])
            ug = np.array([float(e.subs(pt)) for e in ghost])
            beta = max(beta, wave_speed(uo, n), wave_speed(ug, n))
            for j in range(k + 1):
                jump = []
                for c in range(4):
                    jump.append(np.array([float((sp.diff(exprs[c], x, a, y, j - a) - sp.diff(ghost[c], x, a, y, j - a)).subs(pt))
                                          for a in range(j, -1, -1)]))
                mn = jump[1] * n[0] + jump[2] * n[1]
                mt = -jump[1] * n[1] + jump[2] * n[0]
                w = np.array([math.comb(j, a) for a in range(j, -1, -1)])
                for q, d in enumerate([jump[0], mn, mt, jump[3]]):
                    J[q, j] += 0.5 * (w * d * d).sum()
        for j in range(k + 1):
            A = (2 * j + 1) / ((2 * k - 1) * math.factorial(j))
            dl = [A * h ** j * math.sqrt(J[q, j]) / D for q, D in enumerate([st[4], st[5], st[5], st[6]])]
            dm = max(dl[1], dl[2])
            expect[:, j] += beta / h * np.array([dl[0], dm, dm, dl[3]])
    np.testing.assert_allclose(sig[:, :, 0], expect, rtol=1e-10, atol=1e-12)

"""Pins of the oracle's DG operator L(u) (eq. DGSystem:Dis) and of its global
OE statistics, against closed forms and textbook special cases."""
import math
import os

import numpy as np
import pytest

from paper_2409_09620_gb300 import workloads as W
from tests.helpers import PhysPoly, rotate_mesh_state, seg_integral

G = 1.4


def euler_flux_n(u, n, g=G):
    """Textbook Euler flux F(u).n (test-side restatement for the FV special case)."""
    rho, m1, m2, E = u
    v1, v2 = m1 / rho, m2 / rho
    p = (g - 1) * (E - 0.5 * (m1 * v1 + m2 * v2))
    f1 = np.array([m1, m1 * v1 + p, m2 * v1, (E + p) * v1])
    f2 = np.array([m2, m1 * v2, m2 * v2 + p, (E + p) * v2])
    return f1 * n[0] + f2 * n[1]


@pytest.mark.parametrize("k", [1, 2])
@pytest.mark.parametrize("periodic", [True, False])
def test_free_stream(oracle_mod, k, periodic):
    """A constant state is a steady solution: L = 0 to round-off."""
    O = oracle_mod
    wl = W.uniform_workload(n=7, k=k, periodic=periodic)
    om = O.OracleMesh.from_mesh(wl.mesh)
    u = om.project(k, fn=wl.u0)
    cf = O.config_for(wl)
    alpha = om.alpha(cf, u)
    L = om.L(cf, u, alpha=alpha)
    area, ln, _ = om.geometry()
    scale = alpha * np.abs(u[:, 0]).max() * (ln.sum(1) / area).max()   # size of one edge-flux term
    assert np.abs(L).max() < 1e-14 * scale


@pytest.mark.parametrize("k", [1, 2])
def test_conservation_periodic(oracle_mod, k):
    """Edge fluxes cancel in pairs: sum_K |K| (L u)^(0) = 0 on a periodic mesh."""
    O = oracle_mod
    mesh = W.jittered_grid(9, 8, seed=21, periodic=True)
    om = O.OracleMesh.from_mesh(mesh)
    u = W.random_modal_state(mesh.nt, k, seed=5, amp=0.2)
    cf = O.make_config(k)
    L = om.L(cf, u, alpha=om.alpha(cf, u))
    area, _, _ = om.geometry()
    tot = (L[:, 0, :] * area).sum(1)
    scale = (np.abs(L[:, 0, :]) * area).sum(1)
    assert (np.abs(tot) <= 1e-14 * scale).all()


@pytest.mark.parametrize("k", [1, 2])
def test_polynomial_flux_is_exact(oracle_mod, k):
    """For a global state with constant velocity v and density / pressure in
    P^k, the Euler flux is itself in P^k, traces agree across edges and the
    quadratures are exact, so L(u) is the L2 projection of -div F(u) in every
    cell whose edges are all interior (a transmissive edge takes the cell
    average as exterior state, pinned separately below)."""
    O = oracle_mod
    rng = np.random.default_rng(30 + k)
    mesh = W.jittered_grid(6, 5, (-0.5, 1.0, 0.0, 1.2), seed=4,
                           side_tags={s: W.BC_TRANSMISSIVE for s in ("left", "right", "bottom", "top")})
    om = O.OracleMesh.from_mesh(mesh)
    v = np.array([0.7, -0.4])
    rho = PhysPoly.random(k, rng, 0.2) + PhysPoly({(0, 0): 1.5})
    p = PhysPoly.random(k, rng, 0.2) + PhysPoly({(0, 0): 2.0})

    def state(x, y):
        r, pp = rho(x, y), p(x, y)
        E = pp / (G - 1) + 0.5 * r * (v @ v)
        return np.stack([r, r * v[0], r * v[1], E], -1)

    def minus_div(x, y):
        vgr = v[0] * rho.d(1, 0)(x, y) + v[1] * rho.d(0, 1)(x, y)
        vgp = v[0] * p.d(1, 0)(x, y) + v[1] * p.d(0, 1)(x, y)
        return -np.stack([vgr, v[0] * vgr + p.d(1, 0)(x, y), v[1] * vgr + p.d(0, 1)(x, y),
                          G / (G - 1) * vgp + 0.5 * (v @ v) * vgr], -1)

    u = om.project(k, fn=state)
    cf = O.make_config(k)
    L = om.L(cf, u, alpha=3.0)
    expect = om.project(k, fn=minus_div)
    nbr, _ = om.neighbors()
    inner = (nbr >= 0).all(1)
    assert inner.sum() >= 12
    assert np.abs(L[:, :, inner] - expect[:, :, inner]).max() < 1e-11 * max(1.0, np.abs(expect).max())


@pytest.mark.parametrize("k", [1, 2])
def test_transmissive_exterior_is_the_cell_average(oracle_mod, k):
    """A single cell with transmissive edges: mode 0 of L is
    -1/|K| sum_i l_i sum_nu w_nu Fhat(u(x_nu), ubar, n_i), with the LF flux of
    eq. fluxLF, the exact cell average ubar as exterior state, Gauss points
    from numpy and the Euler flux restated here."""
    O = oracle_mod
    rng = np.random.default_rng(70 + k)
    V = np.array([[0.1, 0.0], [1.0, 0.2], [0.25, 0.9]])
    tri = np.array([[0, 1, 2]], np.int32)
    bc = np.full((1, 3), W.BC_TRANSMISSIVE, np.int8)
    om = O.OracleMesh(V, tri, None, bc)
    polys = [PhysPoly.random(k, rng, 0.1 * b) + PhysPoly({(0, 0): b}) for b in (1.3, 0.4, -0.3, 2.9)]
    u = om.project(k, fn=lambda x, y: np.stack([p(x, y) for p in polys], -1))
    from tests.helpers import tri_integral
    area = 0.5 * ((V[1, 0] - V[0, 0]) * (V[2, 1] - V[0, 1]) - (V[2, 0] - V[0, 0]) * (V[1, 1] - V[0, 1]))
    ubar = np.array([tri_integral(p, V) / area for p in polys])
    alpha = 2.7
    cf = O.make_config(k)
    L = om.L(cf, u, alpha=alpha)
    xg, wg = np.polynomial.legendre.leggauss(k + 1)
    acc = np.zeros(4)
    for i in range(3):
        a, b = V[(i + 1) % 3], V[(i + 2) % 3]
        d = b - a
        ln = math.hypot(*d)
        n = np.array([d[1], -d[0]]) / ln
        for s, w in zip(0.5 * (1 + xg), 0.5 * wg):
            P = a + s * d
            um = np.array([p(*P) for p in polys])
            fh = 0.5 * (euler_flux_n(um, n) + euler_flux_n(ubar, n) - alpha * (ubar - um))
            acc -= ln * w * fh
    np.testing.assert_allclose(L[:, 0, 0], acc / area, rtol=1e-11, atol=1e-13 * np.abs(acc / area).max())


def test_piecewise_constant_reduces_to_fv_lf(oracle_mod):
    """P^0 data: mode 0 of L is the first-order finite-volume LF scheme
    -1/|K| sum_i l_i Fhat(u_K, u_nbr, n_i); higher modes follow from the
    divergence theorem with constant traces."""
    O = oracle_mod
    for k in (1, 2):
        mesh = W.jittered_grid(6, 6, seed=9, periodic=True)
        om = O.OracleMesh.from_mesh(mesh)
        rng = np.random.default_rng(3)
        nb = 3 if k == 1 else 6
        u = np.zeros((4, nb, mesh.nt))
        prim = np.stack([rng.uniform(0.5, 2, mesh.nt), rng.uniform(-1, 1, mesh.nt),
                         rng.uniform(-1, 1, mesh.nt), rng.uniform(0.5, 2, mesh.nt)], 1)
        u[:, 0, :] = W.prim_to_cons(*prim.T).T
        alpha = 2.5
        cf = O.make_config(k)
        L = om.L(cf, u, alpha=alpha)
        nbr, ne = om.neighbors()
        area, ln, nrm = om.geometry()
        cm = O.mass_constants(k)
        for K in range(0, mesh.nt, 5):
            uK = u[:, 0, K]
            fv = np.zeros(4)
            modes = np.zeros((4, nb))
            V = mesh.xy[mesh.tri[K]]
            T = np.array([[V[1, 0] - V[0, 0], V[2, 0] - V[0, 0]], [V[1, 1] - V[0, 1], V[2, 1] - V[0, 1]]])
            Ti = np.linalg.inv(T)
            for i in range(3):
                uN = u[:, 0, nbr[K, i]]
                n = nrm[K, i]
                fh = 0.5 * (euler_flux_n(uK, n) + euler_flux_n(uN, n) - alpha * (uN - uK))
                fv -= ln[K, i] * fh
                A, B = V[(i + 1) % 3], V[(i + 2) % 3]
                for l in range(nb):
                    def psi(x, y, l=l):
                        ref = Ti @ np.stack([x - V[0, 0], y - V[0, 1]])
                        return np.array([O.basis(a, b)[0][l] for a, b in zip(ref[0], ref[1])])
                    modes[:, l] += (euler_flux_n(uK, n) - fh) * seg_integral(psi, A, B, n=4)
            np.testing.assert_allclose(L[:, 0, K], fv / area[K], rtol=1e-12, atol=1e-12)
            np.testing.assert_allclose(L[:, :, K], modes / (cm[None, :] * area[K]), rtol=1e-10, atol=1e-11)


@pytest.mark.parametrize("k", [1, 2])
@pytest.mark.parametrize("phi", [math.pi / 2, math.pi / 4])
def test_operator_rotation_invariant(oracle_mod, k, phi):
    """Thm (DG is RI): rotating mesh and state rotates L(u)."""
    O = oracle_mod
    mesh = W.jittered_grid(7, 6, seed=12, periodic=True)
    om = O.OracleMesh.from_mesh(mesh)
    u = W.random_modal_state(mesh.nt, k, seed=8, amp=0.1)
    cf = O.make_config(k)
    L = om.L(cf, u, alpha=om.alpha(cf, u))
    xy, ur = rotate_mesh_state(mesh, u, phi)
    omr = O.OracleMesh(xy, mesh.tri, mesh.canon, mesh.bc)
    Lr = omr.L(cf, ur, alpha=omr.alpha(cf, ur))
    _, Lrot = rotate_mesh_state(mesh, L, phi)
    assert np.abs(Lr - Lrot).max() < 1e-12 * np.abs(L).max()


def _volume_rules():
    rows = np.loadtxt(os.path.join(os.path.dirname(__file__), "golden", "volume_rules.txt"))
    return {3: rows[rows[:, 0] == 3][:, 1:], 6: rows[rows[:, 0] == 6][:, 1:]}


@pytest.mark.parametrize("k", [1, 2])
def test_global_statistics(oracle_mod, k):
    """eqs. (OEScalar:Coef2), (normOmg), (RIOESys:Coef1): domain mean from the
    cell averages, sup deviations at the printed volume-rule points."""
    O = oracle_mod
    mesh = W.jittered_grid(8, 7, (0, 2, 0, 1), seed=13,
                           side_tags={s: W.BC_REFLECT for s in ("left", "right", "bottom", "top")})
    om = O.OracleMesh.from_mesh(mesh)
    u = W.random_modal_state(mesh.nt, k, seed=14, amp=0.3)
    st = om.stats(O.make_config(k), u)
    area, _, _ = om.geometry()
    mean = (u[:, 0, :] * area).sum(1) / area.sum()
    np.testing.assert_allclose(st[:4], mean, rtol=1e-14)
    np.testing.assert_allclose(st[7], 2.0, rtol=1e-14)
    rule = _volume_rules()[3 if k == 1 else 6]
    D = np.zeros(5)
    for K in range(mesh.nt):
        V = mesh.xy[mesh.tri[K]]
        for b in rule[:, :3]:
            x, y = b @ V
            val = om.eval(k, u, K, x, y) - mean
            D = np.maximum(D, [abs(val[0]), math.hypot(val[1], val[2]), abs(val[3]), abs(val[1]), abs(val[2])])
    np.testing.assert_allclose(st[[4, 5, 6, 8, 9]], D, rtol=1e-13)

"""Pins of the oracle's simplified BP limiter (Sec. 4.4) with the optimal
decomposition's point sets (eqs. 1944, 1981)."""
import math

import numpy as np
import pytest

from paper_2409_09620_gb300 import workloads as W
from tests.helpers import PhysPoly, random_triangle

G = 1.4


def int_energy(u):
    return u[3] - 0.5 * (u[1] ** 2 + u[2] ** 2) / u[0]


@pytest.mark.parametrize("k", [1, 2])
def test_limiter_invariants(oracle_mod, k):
    """After limiting: rho >= eps1 and E - |m|^2/2rho >= eps2 at every point of
    the set, averages bitwise unchanged, admissible cells untouched, and one
    of the two constraints active in every limited cell (theta is maximal)."""
    O = oracle_mod
    mesh = W.jittered_grid(10, 9, seed=50, periodic=True)
    om = O.OracleMesh.from_mesh(mesh)
    u = W.random_modal_state(mesh.nt, k, seed=51, amp=0.6 if k == 1 else 0.35)
    cf = O.make_config(k)
    before = om.point_minima(cf, u)
    out, cnt = om.limit(cf, u)
    after = om.point_minima(cf, out)
    assert np.array_equal(out[:, 0], u[:, 0])
    rb = u[0, 0]
    eb = int_energy(u[:, 0])
    eps1 = np.minimum(rb, 1e-13)
    eps2 = np.minimum(eb, 1e-13)
    scale = np.abs(u).max()
    assert (after[:, 0] >= eps1 - 1e-14 * scale).all()
    assert (after[:, 1] >= eps2 - 1e-13 * scale).all()
    bad = (before[:, 0] < eps1) | (before[:, 1] < eps2)
    assert 0 < bad.sum() < mesh.nt          # the test exercises both branches
    assert cnt[0] == bad.sum() and cnt[1] == 0
    assert np.array_equal(out[..., ~bad], u[..., ~bad])
    # recover theta2 from the energy modes and theta1 from the density modes;
    # where theta1 < 1 the density constraint is active after Step 1
    th2 = np.ones(mesh.nt)
    th1 = np.ones(mesh.nt)
    for K in np.nonzero(bad)[0]:
        l = np.argmax(np.abs(u[3, 1:, K])) + 1
        th2[K] = out[3, l, K] / u[3, l, K]
        l = np.argmax(np.abs(u[0, 1:, K])) + 1
        th1[K] = out[0, l, K] / (u[0, l, K] * th2[K])
    assert (th1 <= 1 + 1e-14).all() and (th2 <= 1 + 1e-14).all() and (th1 >= 0).all() and (th2 >= 0).all()
    sel = th1 < 1 - 1e-12
    assert sel.any()
    step1_min = rb[sel] + th1[sel] * (before[sel, 0] - rb[sel])
    np.testing.assert_allclose(step1_min, eps1[sel], atol=1e-13 * scale)


def test_p1_theta_by_hand(oracle_mod):
    """Step 1 for P1 on one cell: rho_min over the 6 edge Gauss points and the
    vertices v1, v2 opposite the two longest edges; theta1 = (rho - eps)/(rho - rho_min)."""
    O = oracle_mod
    rng = np.random.default_rng(52)
    for _ in range(50):
        V = random_triangle(rng)
        om = O.OracleMesh(V, np.array([[0, 1, 2]], np.int32), None, np.full((1, 3), 1, np.int8))
        g = np.array([rng.uniform(-3, 3), rng.uniform(-3, 3)])
        cen = V.mean(0)
        rho = PhysPoly({(0, 0): 1.0 - g @ cen, (1, 0): g[0], (0, 1): g[1]})
        fn = lambda x, y: np.stack([rho(x, y), 0 * x, 0 * x, 50.0 + 0 * x], -1)
        u = om.project(1, fn=fn)
        out, _ = om.limit(O.make_config(1), u)
        ln = np.array([math.hypot(*(V[(i + 2) % 3] - V[(i + 1) % 3])) for i in range(3)])
        order = np.argsort(-ln, kind="stable")
        pts = [V[order[0]], V[order[1]]]
        gl, _ = np.polynomial.legendre.leggauss(2)
        for i in range(3):
            A, B = V[(i + 1) % 3], V[(i + 2) % 3]
            pts += [A + (B - A) * 0.5 * (1 + s) for s in gl]
        rmin = min(rho(*p) for p in pts)
        rbar = u[0, 0, 0]
        th = 1.0 if rmin >= 1e-13 else (rbar - 1e-13) / (rbar - rmin)
        np.testing.assert_allclose(out[0, 1:, 0], th * u[0, 1:, 0], rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(out[3, 1:, 0], u[3, 1:, 0], atol=1e-15)


def test_p2_internal_nodes_are_needed(oracle_mod):
    """Reading of eq. (1981) for P2: the paper's E_* (the decomposition formula
    applied to E values) over-estimates E at the weighted internal state, since
    E is concave.  States exist with E > 0 at every edge Gauss point and
    E_* > 0, yet E < 0 at an internal node; the limiter must act on them."""
    O = oracle_mod
    rng = np.random.default_rng(53)
    V = np.array([[0.0, 0.0], [1.0, 0.1], [0.35, 0.8]])
    om = O.OracleMesh(V, np.array([[0, 1, 2]], np.int32), None, np.full((1, 3), 1, np.int8))
    d = om.decomposition(2, 0)
    cf = O.make_config(2)
    found = 0
    gl, gw = np.polynomial.legendre.leggauss(3)
    for _ in range(4000):
        u = np.zeros((4, 6, 1))
        u[:, 0, 0] = [1.0, rng.uniform(-1, 1), rng.uniform(-1, 1), 1.5]
        u[:, 1:, 0] = rng.uniform(-0.4, 0.4, (4, 5))
        ev = lambda x, y: om.eval(2, u, 0, x, y)
        edge_vals = []
        for i in range(3):
            A, B = V[(i + 1) % 3], V[(i + 2) % 3]
            edge_vals.append([ev(*(A + (B - A) * 0.5 * (1 + s))) for s in gl])
        if min(min(v[0], int_energy(v)) for ev_i in edge_vals for v in ev_i) <= 1e-3:
            continue
        ubar = u[:, 0, 0]
        sw = d["w"].sum()
        e_star = (int_energy(ubar) - sum(d["w"][i] * sum(0.5 * gw[q] * int_energy(edge_vals[i][q]) for q in range(3))
                                        for i in range(3))) / (1 - sw)
        node_e = [int_energy(ev(*d["nodes"][s])) for s in range(2)]
        node_r = [ev(*d["nodes"][s])[0] for s in range(2)]
        if e_star > 0 and min(node_r) > 0 and min(node_e) < 0:
            found += 1
            out, cnt = om.limit(cf, u)
            assert cnt[0] == 1
            mins = om.point_minima(cf, out)[0]
            assert mins[1] >= -1e-14
            if found >= 5:
                break
    assert found >= 5

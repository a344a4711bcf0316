"""Pins of the oracle's mesh, basis and decomposition against closed forms,
brute-force integration and the values printed in the paper."""
import math
import os

import numpy as np
import pytest

from paper_2409_09620_gb300 import workloads as W
from tests.helpers import PhysPoly, random_triangle, seg_integral, single_cell, tri_integral

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _mesh1(O, V):
    xy, tri, bc = single_cell(V)
    return O.OracleMesh(xy, tri, None, bc)


def test_basis_orthogonal_and_mass(oracle_mod):
    """eq. (basisfunc): orthogonality on the reference triangle and a_K/|K|
    against exact monomial integrals int xi^a eta^b = a! b! / (a+b+2)!."""
    O = oracle_mod
    # expand each Psi into monomials by sampling the oracle at 6 points and solving
    pts = np.array([[0.1, 0.2], [0.7, 0.1], [0.2, 0.6], [0.3, 0.3], [0.05, 0.9], [0.5, 0.45]])
    mons = [(0, 0), (1, 0), (0, 1), (2, 0), (1, 1), (0, 2)]
    A = np.array([[x ** a * y ** b for (a, b) in mons] for x, y in pts])
    P = np.array([O.basis(x, y)[0] for x, y in pts])         # [pt, l]
    coef = np.linalg.solve(A, P)                                # [mon, l]

    def integ(a, b):
        return math.factorial(a) * math.factorial(b) / math.factorial(a + b + 2)

    G = np.zeros((6, 6))
    for i, (a1, b1) in enumerate(mons):
        for j, (a2, b2) in enumerate(mons):
            G += np.outer(coef[i], coef[j]) * integ(a1 + a2, b1 + b2)
    off = G - np.diag(np.diag(G))
    assert np.abs(off).max() < 1e-13
    # |K_ref| = 1/2, so a/|K| = 2 * G_ll
    np.testing.assert_allclose(2.0 * np.diag(G), [1, 2 / 3, 1 / 2, 16 / 15, 4 / 9, 1 / 3], rtol=1e-13)
    np.testing.assert_allclose(O.mass_constants(2), 2.0 * np.diag(G), rtol=1e-13)
    # reference derivatives are the derivatives of the expansion
    for x, y in pts:
        psi, d, d2 = O.basis(x, y)
        dx = coef[1] + 2 * coef[3] * x + coef[4] * y
        dy = coef[2] + coef[4] * x + 2 * coef[5] * y
        np.testing.assert_allclose(d[:, 0], dx, atol=1e-12)
        np.testing.assert_allclose(d[:, 1], dy, atol=1e-12)
        np.testing.assert_allclose(d2[:, 0], 2 * coef[3], atol=1e-12)
        np.testing.assert_allclose(d2[:, 1], coef[4], atol=1e-12)
        np.testing.assert_allclose(d2[:, 2], 2 * coef[5], atol=1e-12)


@pytest.mark.parametrize("k", [1, 2])
def test_projection_reproduces_polynomials(oracle_mod, k):
    """The L2 projection with the 12-point rule is exact on P^k, and the
    oracle's evaluation reproduces a physical polynomial at random points."""
    O = oracle_mod
    rng = np.random.default_rng(10 + k)
    mesh = W.jittered_grid(5, 4, (0.0, 2.0, -1.0, 0.5), seed=3, side_tags={})
    om = O.OracleMesh.from_mesh(mesh)
    polys = [PhysPoly.random(k, rng) for _ in range(4)]
    u = om.project(k, fn=lambda x, y: np.stack([p(x, y) for p in polys], axis=-1))
    for K in range(0, mesh.nt, 7):
        V = mesh.xy[mesh.tri[K]]
        for _ in range(3):
            b = rng.dirichlet([1, 1, 1])
            x, y = b @ V
            np.testing.assert_allclose(om.eval(k, u, K, x, y), [p(x, y) for p in polys], atol=1e-12)


def test_mesh_adjacency_and_geometry(oracle_mod):
    O = oracle_mod
    mesh = W.jittered_grid(6, 5, (0, 1, 0, 1), seed=7, periodic=True)
    om = O.OracleMesh.from_mesh(mesh)
    nbr, ne = om.neighbors()
    assert (nbr >= 0).all()
    K = np.arange(mesh.nt)[:, None].repeat(3, 1)
    assert (nbr[nbr, ne] == K).all()      # symmetric
    area, ln, nrm = om.geometry()
    np.testing.assert_allclose(area.sum(), 1.0, rtol=1e-13)
    # closed boundary: sum_i l_i n_i = 0 per cell; normals point away from the centroid
    np.testing.assert_allclose((ln[..., None] * nrm).sum(1), 0.0, atol=1e-14)
    cen = mesh.xy[mesh.tri].mean(1)
    for i in range(3):
        a = mesh.xy[mesh.tri[:, (i + 1) % 3]]
        b = mesh.xy[mesh.tri[:, (i + 2) % 3]]
        mid = 0.5 * (a + b)
        assert ((mid - cen) * nrm[:, i]).sum(1).min() > 0
        np.testing.assert_allclose(np.hypot(*(b - a).T), ln[:, i], rtol=1e-14)
    # opposite normals on a shared edge
    np.testing.assert_allclose(nrm[nbr, ne], -nrm, atol=1e-15)


def test_mesh_rejects_bad_input(oracle_mod):
    O = oracle_mod
    xy, tri, bc = single_cell([[0, 0], [0, 1], [1, 0]])      # clockwise
    with pytest.raises(ValueError):
        O.OracleMesh(xy, tri, None, bc)
    xy, tri, bc = single_cell([[0, 0], [1, 0], [0, 1]], tag=0)  # boundary edge without a tag
    with pytest.raises(ValueError):
        O.OracleMesh(xy, tri, None, bc)


def _check_decomposition(O, V, k, rng, ntrial=5):
    om = _mesh1(O, V)
    d = om.decomposition(k, 0)
    area = tri_integral(lambda x, y: 1.0 + 0 * x, V)
    w, om_, nodes = d["w"], d["omega"], d["nodes"]
    assert (w > 0).all()
    nn = d["n_nodes"]
    tot = w.sum() + om_[:nn].sum()
    np.testing.assert_allclose(tot, 1.0, atol=1e-14)
    for _ in range(ntrial):
        p = PhysPoly.random(k, rng)
        lhs = tri_integral(p, V) / area
        rhs = 0.0
        for i in range(3):
            A, B = V[(i + 1) % 3], V[(i + 2) % 3]
            li = math.hypot(*(B - A))
            rhs += w[i] / li * seg_integral(p, A, B)
        for s in range(nn):
            rhs += om_[s] * p(*nodes[s])
        assert abs(lhs - rhs) < 1e-13 * max(1.0, abs(lhs))
    # internal nodes inside K (strict convex combination of the vertices)
    T = np.array([[V[1, 0] - V[0, 0], V[2, 0] - V[0, 0]], [V[1, 1] - V[0, 1], V[2, 1] - V[0, 1]]])
    for s in range(nn):
        xi, eta = np.linalg.solve(T, nodes[s] - V[0])
        if k == 2:
            assert min(xi, eta, 1 - xi - eta) > 0
        else:   # the P1 node lies on e3 (between v1 and v2 of the sorted labelling)
            assert min(xi, eta, 1 - xi - eta) > -1e-14
    return d


@pytest.mark.parametrize("k", [1, 2])
def test_decomposition_exact_feasible(oracle_mod, k):
    """eqs. (1040) and (1139): exact on P^k, positive weights summing to one,
    internal nodes in K (Definition 4.1), on random triangles."""
    rng = np.random.default_rng(100 + k)
    for _ in range(300):
        V = random_triangle(rng)
        _check_decomposition(oracle_mod, V, k, rng, ntrial=2)


def test_p1_critical_polynomial(oracle_mod):
    """Proof of Thm 4.2: with p_* = 0 at v1, v2 and 1 at v3 (sorted labels),
    the optimal weights satisfy w1/2 + w2/2 = 1/3 and the node sits on e3."""
    rng = np.random.default_rng(5)
    for _ in range(200):
        V = random_triangle(rng)
        d = _mesh1(oracle_mod, V).decomposition(1, 0)
        ln = np.array([math.hypot(*(V[(i + 2) % 3] - V[(i + 1) % 3])) for i in range(3)])
        order = np.argsort(-ln, kind="stable")
        np.testing.assert_allclose(d["w"][order[0]] / 2 + d["w"][order[1]] / 2, 1 / 3, atol=1e-15)
        np.testing.assert_allclose(d["c_dcw"], 2 / (3 * (ln[order[0]] + ln[order[1]])), rtol=1e-14)
        assert list(d["limv"]) == list(order[:2])


def _table_cells():
    eq = np.array([[0.0, 0.0], [1.0, 0.0], [0.5, math.sqrt(3) / 2]])
    ri = np.array([[0.0, 0.0], [1.0, 0.0], [0.5, 0.5]])
    return {"equilateral": eq, "right_isosceles": ri}


def test_table_2019_golden(oracle_mod):
    """Table tab:2019 (Sec. 4.3): BP CFL numbers and internal node counts."""
    cells = _table_cells()
    rows = [l.split() for l in open(os.path.join(GOLDEN, "tab2019.txt")) if l.strip() and not l.startswith("#")]
    assert len(rows) == 4
    for name, k, cdcw, nnodes, czxs in rows:
        V = cells[name]
        d = _mesh1(oracle_mod, V).decomposition(int(k), 0)
        np.testing.assert_allclose(d["c_dcw"], float(cdcw), rtol=1e-14)
        np.testing.assert_allclose(d["c_zxs"], float(czxs), rtol=1e-14)
        # distinct internal nodes with positive weight
        pts = [tuple(np.round(d["nodes"][s], 12)) for s in range(d["n_nodes"]) if d["omega"][s] > 1e-14]
        assert len(set(pts)) == int(nnodes)
    # the printed four-digit decimals
    got = []
    for name in ("equilateral", "right_isosceles"):
        for k in (1, 2):
            d = _mesh1(oracle_mod, cells[name]).decomposition(k, 0)
            got += [round(d["c_dcw"], 4), round(d["c_zxs"], 4)]
    assert got == [0.3333, 0.1111, 0.1667, 0.0370, 0.3905, 0.1381, 0.2042, 0.0460]


def test_cfl_ratio_ranges(oracle_mod):
    """Fig. fig:1744: C_DCW/C_ZXS in [2, 3] (P1), [3.8038, 4.5] (P2);
    C_DCW/C_CS in [2, 2.6667] (P1), [1, 1.4202] (P2), with C_CS = 1/(6 l1)."""
    rng = np.random.default_rng(8)
    lo = {1: [9, 9], 2: [9, 9]}
    hi = {1: [0, 0], 2: [0, 0]}
    shapes = [(rng.uniform(0.5, 1.0), None) for _ in range(3000)]
    shapes += [(1.0 - 1e-4, 1e-3), (1.0, 1.0), (0.5 + 1e-6, 0.5 + 1e-6), (1.0, 2e-3)]
    for l2, l3 in shapes:
        if l3 is None:
            l3 = rng.uniform(max(1.0 - l2, 1e-3), l2)
        # triangle with edge lengths (1, l2, l3): v2=(0,0), v3=(1,0) on e1, v1 from l2, l3
        x = (l3 ** 2 - l2 ** 2 + 1.0) / 2.0
        y = math.sqrt(max(l3 ** 2 - x ** 2, 1e-300))
        V = np.array([[x, y], [0.0, 0.0], [1.0, 0.0]])
        if (V[1, 0] - V[0, 0]) * (V[2, 1] - V[0, 1]) - (V[2, 0] - V[0, 0]) * (V[1, 1] - V[0, 1]) < 0:
            V = V[[0, 2, 1]]
        om = _mesh1(oracle_mod, V)
        for k in (1, 2):
            d = om.decomposition(k, 0)
            r = [d["c_dcw"] / d["c_zxs"], d["c_dcw"] * 6.0]
            for j in range(2):
                lo[k][j] = min(lo[k][j], r[j])
                hi[k][j] = max(hi[k][j], r[j])
    assert 2.0 - 1e-12 <= lo[1][0] and hi[1][0] <= 3.0 + 1e-12
    assert 2.0 - 1e-12 <= lo[1][1] and hi[1][1] <= 8 / 3 + 1e-12
    assert 3.8038 - 1e-4 <= lo[2][0] and hi[2][0] <= 4.5 + 1e-12
    assert 1.0 - 1e-12 <= lo[2][1] and hi[2][1] <= 1.4202 + 1e-4
    # the sampled extremes approach the printed bounds
    assert hi[1][0] > 2.99 and lo[1][0] < 2.05 and hi[2][0] > 4.49 and lo[2][0] < 3.82
    assert hi[2][1] > 1.41


@pytest.mark.parametrize("k,lo,hi", [(1, 2.0, 3.0), (2, 3.8038, 4.5)])
def test_dt_ratio_on_jittered_mesh(oracle_mod, k, lo, hi):
    """Sec. 5 step sizes: min(C_DCW |K|) / min(C_ZXS |K|) on a jittered grid
    lies in the per-cell ratio range (the paper measures 2.85-2.87 and 4.487-4.490)."""
    mesh = W.jittered_grid(20, 20, seed=11, periodic=True)
    om = oracle_mod.OracleMesh.from_mesh(mesh)
    r = om.min_cfl_area(k, 0) / om.min_cfl_area(k, 1)
    assert lo - 1e-9 <= r <= hi + 1e-9

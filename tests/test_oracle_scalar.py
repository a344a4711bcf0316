"""Pins of the oracle's OEDG scheme for scalar conservation laws (Sec. 2):
the P3 basis against exact integrals and finite differences, physical
derivatives against exact polynomials, the DG operator against the exact
divergence where the quadratures are exact, the normaliser at the printed
12-point rule, sigma recomputed by hand, the exact damping, conservation, the
free stream and the design order on the paper's smooth problems."""
import math
import os

import numpy as np
import pytest

from paper_2409_09620_gb300 import workloads as W
from tests.helpers import PhysPoly, random_triangle, single_cell, tri_integral

REF = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]])
MASS = [1, 2 / 3, 1 / 2, 16 / 15, 4 / 9, 1 / 3, 16 / 7, 4 / 5, 1 / 3, 1 / 4]


def _basis_fn(O, l, r=0, s=0):
    return np.vectorize(lambda x, y: O.sc_basis(x, y, r, s)[l])


def test_p3_basis_orthogonal_with_printed_mass(oracle_mod):
    """eq. (basisfunc): Psi^(0..9) orthogonal on the reference triangle; the
    masses a^(l) / |K| equal exact rationals and the oracle's 12-point values."""
    O = oracle_mod
    G = np.zeros((10, 10))
    for a in range(10):
        for b in range(a, 10):
            fa, fb = _basis_fn(O, a), _basis_fn(O, b)
            G[a, b] = G[b, a] = tri_integral(lambda x, y: fa(x, y) * fb(x, y), REF, n=8) / 0.5
    assert np.abs(G - np.diag(np.diag(G))).max() < 1e-12
    np.testing.assert_allclose(np.diag(G), MASS, rtol=1e-12)
    np.testing.assert_allclose(O.sc_mass_constants(3), MASS, rtol=1e-12)


def test_p3_basis_derivatives_match_differences(oracle_mod):
    O = oracle_mod
    rng = np.random.default_rng(5)
    h = 1e-4
    for _ in range(5):
        x, y = rng.uniform(0.1, 0.4, 2)
        for r, s in ((1, 0), (0, 1), (2, 0), (1, 1), (0, 2), (3, 0), (2, 1), (1, 2), (0, 3)):
            # central difference of the next lower derivative
            if r > 0:
                lo = (O.sc_basis(x + h, y, r - 1, s) - O.sc_basis(x - h, y, r - 1, s)) / (2 * h)
            else:
                lo = (O.sc_basis(x, y + h, r, s - 1) - O.sc_basis(x, y - h, r, s - 1)) / (2 * h)
            np.testing.assert_allclose(O.sc_basis(x, y, r, s), lo, rtol=1e-6, atol=1e-5)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_physical_derivatives_of_a_cubic(oracle_mod, seed):
    """A physical cubic is reproduced exactly by the P3 projection; every
    physical derivative up to order 3 matches the polynomial's."""
    O = oracle_mod
    rng = np.random.default_rng(seed)
    V = random_triangle(rng)
    xy, tri, bc = single_cell(V, tag=W.BC_TRANSMISSIVE)
    om = O.OracleMesh(xy, tri, None, bc)
    p = PhysPoly.random(3, rng)
    u = om.sc_project(3, p)
    for _ in range(4):
        b = rng.dirichlet([1, 1, 1])
        x, y = b @ V
        for j in range(4):
            for a in range(j + 1):
                got = om.sc_deriv(3, u, 0, x, y, a, j - a)
                want = p.d(a, j - a)(x, y)
                assert abs(got - want) <= 1e-9 * max(1.0, abs(want))


def _open_mesh(n=5, seed=21, tags=W.BC_TRANSMISSIVE):
    return W.jittered_grid(n, n + 1, (0, 1, 0, 1.2), seed=seed, side_tags={s: tags for s in ("left", "right", "bottom", "top")})


@pytest.mark.parametrize("k", [1, 2, 3])
def test_linear_operator_is_the_exact_divergence(oracle_mod, k):
    """eq. (DGScalar:Dis) with F = (a1 u, a2 u): for a global polynomial of
    degree k the traces agree across edges (transmissive boundary copies), the
    volume rule (degree 2k) and the Q = k + 1 Gauss rule are exact, so L(u) is
    the projection of -(a1 u_x + a2 u_y)."""
    O = oracle_mod
    rng = np.random.default_rng(10 + k)
    mesh = _open_mesh()
    om = O.OracleMesh.from_mesh(mesh)
    p = PhysPoly.random(k, rng)
    cf = O.make_sc_config(k, flux=0, ax=0.7, ay=-1.3)
    u = om.sc_project(k, p)
    L = om.sc_L(cf, u, alpha=om.sc_alpha(cf, u))
    want = om.sc_project(k, lambda x, y: -(0.7 * p.d(1, 0)(x, y) - 1.3 * p.d(0, 1)(x, y)))
    assert np.abs(L - want).max() < 1e-10 * max(1.0, np.abs(want).max())


def test_burgers_p1_operator_is_the_exact_divergence(oracle_mod):
    """Burgers with P1: F(u) . grad Psi has degree 2 = 2k and F Psi degree 3 =
    2Q - 1, so L(u) is the projection of -u (u_x + u_y) exactly."""
    O = oracle_mod
    rng = np.random.default_rng(7)
    mesh = _open_mesh()
    om = O.OracleMesh.from_mesh(mesh)
    p = PhysPoly.random(1, rng)
    cf = O.make_sc_config(1, flux=1)
    u = om.sc_project(1, p)
    L = om.sc_L(cf, u, alpha=om.sc_alpha(cf, u))
    want = om.sc_project(1, lambda x, y: -p(x, y) * (p.d(1, 0)(x, y) + p.d(0, 1)(x, y)))
    assert np.abs(L - want).max() < 1e-10 * max(1.0, np.abs(want).max())


def _volume_rule(N):
    rows = np.loadtxt(os.path.join(os.path.dirname(__file__), "golden", "volume_rules.txt"))
    return rows[rows[:, 0] == N][:, 1:]


@pytest.mark.parametrize("k", [1, 2, 3])
def test_normaliser_at_the_printed_rule(oracle_mod, k):
    """Domain mean from |K| u^(0) and sup |u - mean| at the printed volume
    points (eq. normOmg; Tables tab:2th, tab:4th, tab:6th)."""
    O = oracle_mod
    mesh = W.jittered_grid(5, 4, seed=8, periodic=True)
    om = O.OracleMesh.from_mesh(mesh)
    rng = np.random.default_rng(k)
    u = rng.uniform(-1, 1, (O.sc_nb(k), om.nt))
    cf = O.make_sc_config(k)
    st = om.sc_stats(cf, u)
    area, _, _ = om.geometry()
    mean = (u[0] * area).sum() / area.sum()
    D = 0.0
    for K in range(om.nt):
        V = mesh.xy[mesh.tri[K]]
        for b in _volume_rule({1: 3, 2: 6, 3: 12}[k])[:, :3]:
            D = max(D, abs(om.sc_eval(k, u, K, *(b @ V)) - mean))
    np.testing.assert_allclose(st, [mean, D, 1.0], rtol=1e-13)


@pytest.mark.parametrize("k,flux", [(1, 0), (2, 1), (3, 0), (3, 1)])
def test_sigma_by_hand(oracle_mod, k, flux):
    """eqs. (OEScalar:Coef1), (OEScalar:beta), (OEScalar:Coef2): for
    cell-wise physical polynomials, sigma^j = sum_i beta_i / h_i delta_i^j with
    the trapezoidal rule of the squared jumps of all derivatives of order j,
    weights C_j^{alpha_1}, A^{k,j} = (2j+1)/((2k-1) j!), h_i = 2|K| / l_i;
    transmissive and constant-state boundary edges included."""
    O = oracle_mod
    rng = np.random.default_rng(60 + 3 * k + flux)
    tag_of = lambda x, y: W.BC_DIRICHLET0 + 1 if x < 1e-12 else W.BC_TRANSMISSIVE
    mesh = W.jittered_grid(4, 4, (0, 1, 0, 1), seed=19,
                           side_tags={"left": tag_of, "right": W.BC_TRANSMISSIVE, "bottom": W.BC_TRANSMISSIVE,
                                      "top": W.BC_TRANSMISSIVE})
    om = O.OracleMesh.from_mesh(mesh)
    polys = [PhysPoly.random(k, rng, 0.3) + PhysPoly({(0, 0): 0.7}) for _ in range(mesh.nt)]
    xy = om.quad12_points()
    u = np.zeros((O.sc_nb(k), om.nt))
    for K in range(om.nt):
        # cell-wise projection of the cell's own polynomial (exact, degree k)
        single = O.OracleMesh(mesh.xy[mesh.tri[K]], np.array([[0, 1, 2]], np.int32), None,
                              np.full((1, 3), W.BC_TRANSMISSIVE, np.int8))
        u[:, K] = single.sc_project(k, polys[K])[:, 0]
    bc_val = 1.9
    cf = O.make_sc_config(k, flux=flux, ax=0.8, ay=0.4, bc_state=(0.0, bc_val, 0.0, 0.0))
    st = om.sc_stats(cf, u)
    _, sig = om.sc_oe(cf, u, dt=0.01, stats=st, want_sigma=True)
    nbr, _ = om.neighbors()
    area, ln, nrm = om.geometry()
    speed = (lambda v, n: 0.8 * n[0] + 0.4 * n[1]) if flux == 0 else (lambda v, n: v * (n[0] + n[1]))
    for K in range(om.nt):
        V = mesh.xy[mesh.tri[K]]
        expect = np.zeros(k + 1)
        for i in range(3):
            n, h, N = nrm[K, i], 2 * area[K] / ln[K, i], nbr[K, i]
            dirichlet = N < 0 and mesh.bc[K, i] == W.BC_DIRICHLET0 + 1
            J = np.zeros(k + 1)
            beta = 0.0
            for vv in ((i + 1) % 3, (i + 2) % 3):
                x, y = V[vv]
                for j in range(k + 1):
                    for a in range(j, -1, -1):
                        own = polys[K].d(a, j - a)(x, y)
                        if N >= 0:
                            ext = polys[N].d(a, j - a)(x, y)
                        elif dirichlet:
                            ext = bc_val if j == 0 else 0.0
                        else:
                            ext = own
                        J[j] += 0.5 * math.comb(j, a) * (own - ext) ** 2
                        if j == 0:
                            beta = max(beta, abs(speed(own, n)), abs(speed(ext, n)))
            for j in range(k + 1):
                A = (2 * j + 1) / ((2 * k - 1) * math.factorial(j))
                expect[j] += beta / h * A * h ** j * math.sqrt(J[j]) / st[1]
        # sigma^j rests on j-th derivatives of the projected state, whose
        # round-off grows like h^-j (h ~ 1/4 here): tolerance per order
        tol = np.array([1e-12, 1e-11, 1e-10, 1e-9])[: k + 1]
        assert (np.abs(sig[:, K] - expect) <= tol * np.abs(expect) + 1e-14).all(), (sig[:, K], expect)


def test_damping_is_the_exact_ode_solution(oracle_mod):
    """eq. (oe:scalar): mode 0 kept bitwise, modes of degree m multiplied by
    exp(-dt sum_{j <= m} sigma^j)."""
    O = oracle_mod
    mesh = W.jittered_grid(5, 5, seed=4, periodic=True)
    om = O.OracleMesh.from_mesh(mesh)
    u = np.random.default_rng(3).uniform(-1, 1, (10, om.nt))
    cf = O.make_sc_config(3, flux=1)
    dt = 0.02
    out, sig = om.sc_oe(cf, u, dt, want_sigma=True)
    assert np.array_equal(out[0], u[0])
    deg = [0, 1, 1, 2, 2, 2, 3, 3, 3, 3]
    for l in range(1, 10):
        np.testing.assert_allclose(out[l], u[l] * np.exp(-dt * sig[: deg[l] + 1].sum(0)), rtol=1e-14)


@pytest.mark.parametrize("k,flux", [(1, 1), (2, 0), (3, 1)])
def test_conservation_and_free_stream(oracle_mod, k, flux):
    O = oracle_mod
    mesh = W.jittered_grid(6, 6, seed=9, periodic=True)
    om = O.OracleMesh.from_mesh(mesh)
    area, _, _ = om.geometry()
    cf = O.make_sc_config(k, flux=flux)
    u0 = om.sc_project(k, lambda x, y: 0.4 + 0.5 * np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y))
    u, t, n, rc = om.sc_advance(cf, u0, 0.0, 1.0, max_steps=6)
    assert rc == 0 and n == 6
    assert abs((u[0] - u0[0]) @ area) <= 1e-14 * np.abs(u0[0]) @ area
    c = np.zeros_like(u0)
    c[0] = 0.37
    uc, _, _, rc = om.sc_advance(cf, c, 0.0, 1.0, max_steps=4)
    assert np.abs(uc[1:]).max() < 1e-14 and np.abs(uc[0] - 0.37).max() < 1e-14   # free stream, to round-off


def _errors(om, k, u, exact):
    xy = om.quad12_points()
    area, _, _ = om.geometry()
    w = _volume_rule(12)[:, 3]
    vals = np.array([[om.sc_eval(k, u, K, *xy[K, mu]) for mu in range(12)] for K in range(om.nt)])
    e = vals - exact(xy[..., 0], xy[..., 1])
    return np.array([(np.abs(e) * w).sum(1) @ area, math.sqrt(((e * e) * w).sum(1) @ area), np.abs(e).max()])


@pytest.mark.parametrize("k,flux,levels", [(1, 0, (1, 2)), (2, 0, (1, 2)), (3, 0, (1, 2)),
                                           (1, 1, (1, 2)), (2, 1, (1, 2)), (3, 1, (1, 2))])
@pytest.mark.slow
def test_design_order(oracle_mod, k, flux, levels):
    """The smooth linear (t = 0.1) and Burgers (t = 0.05) problems of Sec. 5 on
    a mesh and its refinement by quadrisection: the L1 and L2 errors fall at
    least at the design rate k + 1 minus 1/2 (the paper reports k + 1 and
    above on its meshes).  P3 runs SSP-RK(3,3) with dt scaled by h^(1/3) so
    that the time error stays below the space error."""
    O = oracle_mod
    make = W.scalar_linear_workload if flux == 0 else W.scalar_burgers_workload
    errs = []
    for lev in levels:
        wl = make(level=lev, k=k)
        om = O.OracleMesh.from_mesh(wl.mesh)
        cf = O.make_sc_config(k, flux=flux, cfl=0.5 ** ((lev - levels[0]) / 3.0) if k == 3 else 1.0)
        u, t, n, rc = om.sc_advance(cf, om.sc_project(k, wl.u0), 0.0, wl.t_end)
        assert rc == 0 and t == wl.t_end
        errs.append(_errors(om, k, u, lambda x, y: wl.exact(x, y, wl.t_end)))
    order = np.log2(errs[0] / errs[1])
    assert (order[:2] >= k + 0.5).all(), order

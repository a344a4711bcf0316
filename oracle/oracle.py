"""ctypes wrapper of the C oracle (test infrastructure only).

States are numpy float64 arrays shaped [4, nb, nt] (component, mode, cell).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None

OR_BC_NONE, OR_BC_REFLECT, OR_BC_TRANSMISSIVE, OR_BC_DIRICHLET0, OR_BC_SHOCK = 0, 1, 2, 3, 7


class Config(C.Structure):
    _fields_ = [("k", C.c_int32), ("oe", C.c_int32), ("bp", C.c_int32), ("decomp", C.c_int32),
                ("gamma", C.c_double), ("cfl", C.c_double), ("bc_state", (C.c_double * 4) * 4),
                ("shock_x0", C.c_double), ("shock_angle", C.c_double), ("shock_speed", C.c_double),
                ("shock_pre", C.c_int32), ("shock_post", C.c_int32)]


class ScConfig(C.Structure):
    _fields_ = [("k", C.c_int32), ("flux", C.c_int32), ("oe", C.c_int32), ("rk", C.c_int32),
                ("ax", C.c_double), ("ay", C.c_double), ("cfl", C.c_double), ("bc_state", C.c_double * 4)]


def make_sc_config(k, flux=0, oe=1, rk=None, ax=1.0, ay=1.0, cfl=1.0, bc_state=(0.0, 0.0, 0.0, 0.0)):
    """Scalar OEDG configuration; rk defaults to SSP-RK(2,2) for P1 and
    SSP-RK(3,3) otherwise (Sec. 5)."""
    cf = ScConfig()
    cf.k, cf.flux, cf.oe = k, flux, oe
    cf.rk = (2 if k == 1 else 3) if rk is None else rk
    cf.ax, cf.ay, cf.cfl = ax, ay, cfl
    for i in range(4):
        cf.bc_state[i] = float(bc_state[i])
    return cf


def sc_nb(k):
    return (k + 1) * (k + 2) // 2


def sc_basis(xi, eta, r=0, s=0):
    out = np.empty(10)
    lib().or_sc_basis(float(xi), float(eta), r, s, _p(out))
    return out


def sc_mass_constants(k):
    c = np.empty(10)
    lib().or_sc_mass_constants(k, _p(c))
    return c[: sc_nb(k)]


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        P = C.c_void_p
        i64, i32, dbl = C.c_int64, C.c_int32, C.c_double
        L.or_mesh_create.argtypes = [i64, P, i64, P, P, P, C.POINTER(P)]
        L.or_mesh_destroy.argtypes = [P]
        L.or_mesh_nt.argtypes = [P]; L.or_mesh_nt.restype = i64
        L.or_mesh_neighbors.argtypes = [P, P, P]
        L.or_mesh_geometry.argtypes = [P, P, P, P]
        L.or_decomposition.argtypes = [P, C.c_int, i64, P, P, P, P, P, P]
        L.or_min_cfl_area.argtypes = [P, C.c_int, C.c_int]; L.or_min_cfl_area.restype = dbl
        L.or_basis.argtypes = [dbl, dbl, P, P, P]
        L.or_mass_constants.argtypes = [C.c_int, P]
        L.or_quad12_points.argtypes = [P, P]
        L.or_project.argtypes = [P, C.c_int, P, P]
        L.or_eval.argtypes = [P, C.c_int, P, i64, dbl, dbl, P]
        L.or_alpha.argtypes = [P, P, P, dbl]; L.or_alpha.restype = dbl
        L.or_alpha_cells.argtypes = [P, P, P, dbl, P, i64]; L.or_alpha_cells.restype = dbl
        L.or_L.argtypes = [P, P, P, dbl, dbl, P, P, i64]
        L.or_rk_stage.argtypes = [P, P, P, P, dbl, dbl, dbl, dbl, dbl, P, P, i64]
        L.or_stats.argtypes = [P, P, P, P]
        L.or_stats_cells.argtypes = [P, P, P, P, i64, P]
        L.or_oe.argtypes = [P, P, P, dbl, P, dbl, P, P, P, i64]
        L.or_limit.argtypes = [P, P, P, P, P, P, i64]
        L.or_point_minima.argtypes = [P, P, P, P]
        L.or_step.argtypes = [P, P, P, P, dbl, P, P]
        L.or_advance.argtypes = [P, P, P, P, dbl, i64, P]
        L.or_num_threads.restype = C.c_int
        L.or_set_num_threads.argtypes = [C.c_int]
        L.or_sc_basis.argtypes = [dbl, dbl, C.c_int, C.c_int, P]
        L.or_sc_mass_constants.argtypes = [C.c_int, P]
        L.or_sc_eval.argtypes = [P, C.c_int, P, i64, dbl, dbl]; L.or_sc_eval.restype = dbl
        L.or_sc_deriv.argtypes = [P, C.c_int, P, i64, dbl, dbl, C.c_int, C.c_int]; L.or_sc_deriv.restype = dbl
        L.or_sc_project.argtypes = [P, C.c_int, P, P]
        L.or_sc_alpha.argtypes = [P, P, P]; L.or_sc_alpha.restype = dbl
        L.or_sc_L.argtypes = [P, P, P, dbl, P]
        L.or_sc_stats.argtypes = [P, P, P, P]
        L.or_sc_oe.argtypes = [P, P, P, dbl, P, P, P]
        L.or_sc_dt_base.argtypes = [P, C.c_int]; L.or_sc_dt_base.restype = dbl
        L.or_sc_step.argtypes = [P, P, P, P, dbl, P]
        L.or_sc_advance.argtypes = [P, P, P, P, dbl, i64, P]
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def make_config(k, oe=1, bp=1, decomp=0, gamma=1.4, cfl=1.0, bc_state=None, shock=(0.0, 0.0, 0.0, 0, 0)):
    cf = Config()
    cf.k, cf.oe, cf.bp, cf.decomp = k, oe, bp, decomp
    cf.gamma, cf.cfl = gamma, cfl
    if bc_state is not None:
        for i in range(4):
            for j in range(4):
                cf.bc_state[i][j] = float(bc_state[i][j])
    cf.shock_x0, cf.shock_angle, cf.shock_speed = float(shock[0]), float(shock[1]), float(shock[2])
    cf.shock_pre, cf.shock_post = int(shock[3]), int(shock[4])
    return cf


def config_for(workload, **kw):
    return make_config(workload.k, bc_state=workload.bc_state, shock=workload.shock,
                       gamma=workload.gamma, **kw)


class OracleMesh:
    def __init__(self, xy, tri, canon=None, bc=None):
        L = lib()
        self.xy = np.ascontiguousarray(xy, dtype=np.float64)
        self.tri = np.ascontiguousarray(tri, dtype=np.int32)
        self.canon = None if canon is None else np.ascontiguousarray(canon, dtype=np.int32)
        self.bc = None if bc is None else np.ascontiguousarray(bc, dtype=np.int8)
        h = C.c_void_p()
        rc = L.or_mesh_create(self.xy.shape[0], _p(self.xy), self.tri.shape[0], _p(self.tri),
                              _p(self.canon), _p(self.bc), C.byref(h))
        if rc != 0:
            raise ValueError(f"or_mesh_create failed: {rc}")
        self.h = h
        self.nt = int(self.tri.shape[0])

    @classmethod
    def from_mesh(cls, mesh):
        return cls(mesh.xy, mesh.tri, mesh.canon, mesh.bc)

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.or_mesh_destroy(self.h)
            self.h = None

    # -- geometry ---------------------------------------------------------
    def neighbors(self):
        nbr = np.empty((self.nt, 3), np.int32)
        ne = np.empty((self.nt, 3), np.int32)
        lib().or_mesh_neighbors(self.h, _p(nbr), _p(ne))
        return nbr, ne

    def geometry(self):
        area = np.empty(self.nt)
        ln = np.empty((self.nt, 3))
        nrm = np.empty((self.nt, 3, 2))
        lib().or_mesh_geometry(self.h, _p(area), _p(ln), _p(nrm))
        return area, ln, nrm

    def decomposition(self, k, K):
        w = np.empty(3); om = np.empty(2); nd = np.empty(4); cfl = np.empty(2)
        nn = np.zeros(1, np.int32); lv = np.zeros(2, np.int32)
        rc = lib().or_decomposition(self.h, k, K, _p(w), _p(om), _p(nd), _p(nn), _p(cfl), _p(lv))
        if rc != 0:
            raise ValueError(rc)
        return dict(w=w, omega=om, nodes=nd.reshape(2, 2), n_nodes=int(nn[0]),
                    c_dcw=float(cfl[0]), c_zxs=float(cfl[1]), limv=lv.copy())

    def min_cfl_area(self, k, decomp=0):
        return lib().or_min_cfl_area(self.h, k, decomp)

    # -- projection -------------------------------------------------------
    def quad12_points(self):
        xy = np.empty((self.nt, 12, 2))
        lib().or_quad12_points(self.h, _p(xy))
        return xy

    def project(self, k, fn=None, cell_fn=None):
        """L2 projection of a point-wise state fn(x, y) -> [..., 4]; cell_fn(cells) -> [nt, 4] for
        piecewise-constant data."""
        if cell_fn is not None:
            vals = np.repeat(np.asarray(cell_fn(np.arange(self.nt)), dtype=np.float64)[:, None, :], 12, axis=1)
        else:
            xy = self.quad12_points()
            vals = np.asarray(fn(xy[..., 0], xy[..., 1]), dtype=np.float64)
        vals = np.ascontiguousarray(vals.reshape(self.nt, 12, 4))
        nb = 3 if k == 1 else 6
        u = np.empty((4, nb, self.nt))
        lib().or_project(self.h, k, _p(vals), _p(u))
        return u

    def project_values(self, k, vals):
        """L2 projection of point values vals[nt, 12, 4] at the 12-point rule's points."""
        vals = np.ascontiguousarray(np.asarray(vals, dtype=np.float64).reshape(self.nt, 12, 4))
        nb = 3 if k == 1 else 6
        u = np.empty((4, nb, self.nt))
        lib().or_project(self.h, k, _p(vals), _p(u))
        return u

    def eval(self, k, u, K, x, y):
        out = np.empty(4)
        lib().or_eval(self.h, k, _p(np.ascontiguousarray(u)), K, x, y, _p(out))
        return out

    # -- stage operators --------------------------------------------------
    def alpha(self, cf, u, t=0.0, cells=None):
        u = np.ascontiguousarray(u)
        if cells is None:
            return lib().or_alpha(self.h, C.byref(cf), _p(u), t)
        cl = np.ascontiguousarray(cells, dtype=np.int64)
        return lib().or_alpha_cells(self.h, C.byref(cf), _p(u), t, _p(cl), cl.size)

    def L(self, cf, u, alpha, t=0.0, cells=None):
        u = np.ascontiguousarray(u)
        out = np.zeros_like(u)
        cl = None if cells is None else np.ascontiguousarray(cells, dtype=np.int64)
        lib().or_L(self.h, C.byref(cf), _p(u), alpha, t, _p(out), _p(cl), 0 if cl is None else cl.size)
        return out

    def rk_stage(self, cf, un, v, a, b, dt, alpha, t=0.0, cells=None):
        un = np.ascontiguousarray(un); v = np.ascontiguousarray(v)
        out = np.zeros_like(v)
        cl = None if cells is None else np.ascontiguousarray(cells, dtype=np.int64)
        lib().or_rk_stage(self.h, C.byref(cf), _p(un), _p(v), a, b, dt, alpha, t, _p(out), _p(cl),
                          0 if cl is None else cl.size)
        return out

    def stats(self, cf, u, cells=None):
        st = np.empty(10)
        u = np.ascontiguousarray(u)
        if cells is None:
            lib().or_stats(self.h, C.byref(cf), _p(u), _p(st))
        else:
            cl = np.ascontiguousarray(cells, dtype=np.int64)
            lib().or_stats_cells(self.h, C.byref(cf), _p(u), _p(cl), cl.size, _p(st))
        return st

    def oe(self, cf, u, dt, stats=None, t=0.0, cells=None, want_sigma=False):
        u = np.ascontiguousarray(u)
        if stats is None:
            stats = self.stats(cf, u)
        out = np.zeros_like(u)
        sig = np.zeros((4, 3, self.nt)) if want_sigma else None
        cl = None if cells is None else np.ascontiguousarray(cells, dtype=np.int64)
        lib().or_oe(self.h, C.byref(cf), _p(u), dt, _p(np.ascontiguousarray(stats)), t, _p(out), _p(sig),
                    _p(cl), 0 if cl is None else cl.size)
        return (out, sig) if want_sigma else out

    def limit(self, cf, u, cells=None):
        u = np.ascontiguousarray(u)
        out = np.zeros_like(u)
        cnt = np.zeros(2, np.int64)
        cl = None if cells is None else np.ascontiguousarray(cells, dtype=np.int64)
        lib().or_limit(self.h, C.byref(cf), _p(u), _p(out), _p(cnt), _p(cl), 0 if cl is None else cl.size)
        return out, cnt

    def point_minima(self, cf, u):
        out = np.empty((self.nt, 2))
        lib().or_point_minima(self.h, C.byref(cf), _p(np.ascontiguousarray(u)), _p(out))
        return out

    def step(self, cf, u, t, t_end):
        u = np.ascontiguousarray(u).copy()
        tt = np.array([t], dtype=np.float64)
        dt = np.zeros(1)
        cnt = np.zeros(4, np.int64)
        rc = lib().or_step(self.h, C.byref(cf), _p(u), _p(tt), t_end, _p(dt), _p(cnt))
        return u, float(tt[0]), float(dt[0]), cnt, rc

    def advance(self, cf, u, t, t_end, max_steps=1 << 60):
        u = np.ascontiguousarray(u).copy()
        tt = np.array([t], dtype=np.float64)
        cnt = np.zeros(4, np.int64)
        rc = lib().or_advance(self.h, C.byref(cf), _p(u), _p(tt), t_end, max_steps, _p(cnt))
        return u, float(tt[0]), cnt, rc


    # -- scalar conservation laws (Sec. 2) ------------------------------------
    def sc_project(self, k, fn):
        """L2 projection of a point-wise scalar fn(x, y) -> [...] (12-point rule)."""
        xy = self.quad12_points()
        vals = np.ascontiguousarray(np.asarray(fn(xy[..., 0], xy[..., 1]), dtype=np.float64).reshape(self.nt, 12))
        u = np.empty((sc_nb(k), self.nt))
        rc = lib().or_sc_project(self.h, k, _p(vals), _p(u))
        if rc != 0:
            raise ValueError(rc)
        return u

    def sc_eval(self, k, u, K, x, y):
        return lib().or_sc_eval(self.h, k, _p(np.ascontiguousarray(u)), K, x, y)

    def sc_deriv(self, k, u, K, x, y, p, q):
        return lib().or_sc_deriv(self.h, k, _p(np.ascontiguousarray(u)), K, x, y, p, q)

    def sc_alpha(self, cf, u):
        return lib().or_sc_alpha(self.h, C.byref(cf), _p(np.ascontiguousarray(u)))

    def sc_L(self, cf, u, alpha):
        L = np.empty_like(np.ascontiguousarray(u))
        rc = lib().or_sc_L(self.h, C.byref(cf), _p(np.ascontiguousarray(u)), alpha, _p(L))
        if rc != 0:
            raise ValueError(rc)
        return L

    def sc_stats(self, cf, u):
        st = np.empty(3)
        lib().or_sc_stats(self.h, C.byref(cf), _p(np.ascontiguousarray(u)), _p(st))
        return st

    def sc_oe(self, cf, u, dt, stats=None, want_sigma=False):
        u = np.ascontiguousarray(u)
        st = self.sc_stats(cf, u) if stats is None else np.ascontiguousarray(stats, dtype=np.float64)
        out = np.empty_like(u)
        sig = np.empty((cf.k + 1, self.nt)) if want_sigma else None
        rc = lib().or_sc_oe(self.h, C.byref(cf), _p(u), dt, _p(st), _p(out), _p(sig))
        if rc != 0:
            raise ValueError(rc)
        return (out, sig) if want_sigma else out

    def sc_dt_base(self, k):
        return lib().or_sc_dt_base(self.h, k)

    def sc_step(self, cf, u, t, t_end):
        u = np.ascontiguousarray(u).copy()
        tt = np.array([t], dtype=np.float64)
        dt = np.zeros(1)
        rc = lib().or_sc_step(self.h, C.byref(cf), _p(u), _p(tt), t_end, _p(dt))
        return u, float(tt[0]), float(dt[0]), rc

    def sc_advance(self, cf, u, t, t_end, max_steps=1 << 60):
        u = np.ascontiguousarray(u).copy()
        tt = np.array([t], dtype=np.float64)
        st = np.zeros(1, np.int64)
        rc = lib().or_sc_advance(self.h, C.byref(cf), _p(u), _p(tt), t_end, max_steps, _p(st))
        return u, float(tt[0]), int(st[0]), rc


def basis(xi, eta):
    psi = np.empty(6); d = np.empty(12); d2 = np.empty(18)
    lib().or_basis(float(xi), float(eta), _p(psi), _p(d), _p(d2))
    return psi, d.reshape(6, 2), d2.reshape(6, 3)


def mass_constants(k):
    c = np.empty(6)
    lib().or_mass_constants(k, _p(c))
    return c[: (3 if k == 1 else 6)]


def num_threads():
    return lib().or_num_threads()


def set_num_threads(n):
    lib().or_set_num_threads(int(n))


def project_workload(om, wl):
    """Initial modal state of a workload: L2 projection then one limiter pass."""
    u = om.project(wl.k, fn=wl.u0, cell_fn=wl.cell_u0)
    cf = config_for(wl)
    u, _ = om.limit(cf, u)
    return u

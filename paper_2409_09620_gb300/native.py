"""Thin ctypes binding of the C ABI in ``include/dg.h`` (argument marshalling
only: every step of the solver runs in the CUDA library).

Loading fails loudly when the library is missing or cannot be loaded: there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

DG_OK, DG_EINVAL, DG_EMESH, DG_ENOMEM, DG_ENONPHYS, DG_ECUDA, DG_ETIMEOUT, DG_EBUSY = 0, -1, -2, -3, -4, -5, -6, -7
PREC_FP64, PREC_MIXED = 0, 1
OE_OFF, OE_RI, OE_CW = 0, 1, 2
BP_OFF, BP_ON = 0, 1
DECOMP_OPTIMAL, DECOMP_ZXS = 0, 1

_lib = None
P = C.c_void_p
i64, i32, dbl = C.c_int64, C.c_int32, C.c_double


class DGError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"dg error {code}: {msg}")
        self.code = code


class Config(C.Structure):
    _fields_ = [("k", i32), ("precision", i32), ("oe", i32), ("bp", i32), ("decomp", i32), ("reserved", i32),
                ("gamma", dbl), ("cfl", dbl), ("bc_state", (dbl * 4) * 4), ("shock_x0", dbl),
                ("shock_angle", dbl), ("shock_speed", dbl), ("shock_pre", i32), ("shock_post", i32)]


class Stats(C.Structure):
    _fields_ = [("steps", i64), ("limited_cells", i64), ("nonphysical", i64), ("cfl_breaches", i64),
                ("t", dbl), ("dt_last", dbl), ("alpha", dbl)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


# name -> (restype, argtypes); every symbol of include/dg.h
FLUX_LINEAR, FLUX_BURGERS = 0, 1


class ScalarConfig(C.Structure):
    _fields_ = [("k", i32), ("flux", i32), ("oe", i32), ("rk", i32), ("ax", dbl), ("ay", dbl), ("cfl", dbl),
                ("bc_state", dbl * 4)]


SIGNATURES = {
    "dg_scalar_project": (i32, [P, i32, P, P]),
    "dg_scalar_init": (i32, [P, P, P, P, C.POINTER(P)]),
    "dg_scalar_advance": (i32, [P, dbl, i64, P]),
    "dg_scalar_advance_async": (i32, [P, i64]),
    "dg_scalar_stream": (P, [P]),
    "dg_scalar_get_state": (i32, [P, P, C.c_size_t, C.POINTER(dbl)]),
    "dg_scalar_errors": (i32, [P, P, P]),
    "dg_scalar_destroy": (None, [P]),
    "dg_mesh_create": (i32, [i64, P, i64, P, P, P, C.POINTER(P)]),
    "dg_mesh_destroy": (None, [P]),
    "dg_mesh_info": (i32, [P, i32, C.POINTER(i64), C.POINTER(dbl), C.POINTER(dbl)]),
    "dg_mesh_neighbors": (i32, [P, P, P]),
    "dg_mesh_geometry": (i32, [P, i32, i32, P, P, P, P, P, P]),
    "dg_quad_points": (i32, [P, P]),
    "dg_project": (i32, [P, i32, P, P]),
    "dg_init": (i32, [P, C.POINTER(Config), P, P, C.POINTER(P)]),
    "dg_advance": (i32, [P, dbl, i64, C.POINTER(Stats)]),
    "dg_advance_async": (i32, [P, i64]),
    "dg_sync": (i32, [P, C.POINTER(Stats)]),
    "dg_get_state": (i32, [P, P, C.c_size_t, C.POINTER(dbl)]),
    "dg_set_state": (i32, [P, P, dbl]),
    "dg_stream": (P, [P]),
    "dg_solver_destroy": (None, [P]),
    "dg_op_rk_stage": (i32, [P, P, P, dbl, dbl, dbl, dbl, dbl, P]),
    "dg_op_stats": (i32, [P, P, P]),
    "dg_op_oe": (i32, [P, P, dbl, P, dbl, P]),
    "dg_op_limit": (i32, [P, P, P, P]),
    "dg_op_alpha": (i32, [P, P, dbl, C.POINTER(dbl)]),
    "dg_profile_steps": (i32, [P, i64, P, P]),
    "dg_probe_fma_peak": (i32, [i32, C.POINTER(dbl), C.POINTER(dbl), P]),
    "dg_stats_noalloc": (i32, [P, i32, P, P, P]),
    "dg_batch_create": (i32, [i32, P, P, P, P, C.POINTER(P)]),
    "dg_batch_destroy": (None, [P]),
    "dg_batch_advance": (i32, [P, P, i64, P]),
    "dg_batch_advance_async": (i32, [P, i64]),
    "dg_batch_set_barrier": (i32, [P, i64, i32]),
    "dg_batch_sync": (i32, [P]),
    "dg_batch_solver": (i32, [P, i32, C.POINTER(P)]),
    "dg_batch_set_shape": (i32, [P, i32, i32, i32]),
    "dg_batch_shape": (i32, [P, C.POINTER(i32), C.POINTER(i32), C.POINTER(i32), C.POINTER(i32), C.POINTER(i32)]),
    "dg_batch_autotune": (i32, [P, i32, C.POINTER(i32), C.POINTER(i32), C.POINTER(i32), C.POINTER(dbl)]),
    "dg_server_create": (i32, [i32, C.c_size_t, i32, P, C.POINTER(P)]),
    "dg_server_destroy": (None, [P]),
    "dg_server_submit": (i32, [P, i64, P, i64, P, P, P, P, P, dbl, C.POINTER(i64)]),
    "dg_server_tick": (i32, [P, C.POINTER(i32), C.POINTER(i32)]),
    "dg_server_request": (i32, [P, i64, P]),
    "dg_server_result": (i32, [P, i64, P, C.c_size_t]),
    "dg_server_stats": (i32, [P, C.POINTER(i64), C.POINTER(i64)]),
    "dg_last_error": (C.c_char_p, []),
}


def library_path() -> str:
    return _build.LIB


def lib(build_if_missing: bool = True):
    """Load the CUDA library (building it if it is missing); raises if it cannot be loaded."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if not os.path.exists(path):
            if not build_if_missing:
                raise RuntimeError(f"CUDA library {path} is missing; run build()")
            _build.build()
        L = C.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(rc):
    if rc != DG_OK:
        raise DGError(rc, lib().dg_last_error().decode())


def _p(a):
    return None if a is None else a.ctypes.data_as(P)


def make_config(k, precision=PREC_FP64, oe=OE_RI, bp=BP_ON, decomp=DECOMP_OPTIMAL, gamma=1.4, cfl=1.0,
                bc_state=None, shock=(0.0, 0.0, 0.0, 0, 0)):
    cf = Config()
    cf.k, cf.precision, cf.oe, cf.bp, cf.decomp, cf.reserved = k, precision, oe, bp, decomp, 0
    cf.gamma, cf.cfl = gamma, cfl
    if bc_state is not None:
        for i in range(4):
            for j in range(4):
                cf.bc_state[i][j] = float(bc_state[i][j])
    cf.shock_x0, cf.shock_angle, cf.shock_speed = float(shock[0]), float(shock[1]), float(shock[2])
    cf.shock_pre, cf.shock_post = int(shock[3]), int(shock[4])
    return cf


def probe_fma_peak(precision=PREC_FP64, stream=None):
    """Measured FMA throughput of the current device (TFLOP/s, launch ms)."""
    tf, ms = dbl(), dbl()
    _check(lib().dg_probe_fma_peak(precision, C.byref(tf), C.byref(ms), None if stream is None else P(stream)))
    return tf.value, ms.value


def config_for(workload, **kw):
    return make_config(workload.k, bc_state=workload.bc_state, shock=workload.shock, gamma=workload.gamma, **kw)


class Mesh:
    """dg_mesh handle built from host arrays."""

    def __init__(self, xy, tri, canon=None, bc=None):
        L = lib()
        xy = np.ascontiguousarray(xy, dtype=np.float64)
        tri = np.ascontiguousarray(tri, dtype=np.int32)
        canon = None if canon is None else np.ascontiguousarray(canon, dtype=np.int32)
        bc = None if bc is None else np.ascontiguousarray(bc, dtype=np.int8)
        h = P()
        _check(L.dg_mesh_create(xy.shape[0] if xy.ndim == 2 else xy.size // 2, _p(xy),
                                tri.shape[0] if tri.ndim == 2 else tri.size // 3, _p(tri), _p(canon), _p(bc),
                                C.byref(h)))
        self.h = h
        nt = i64()
        L.dg_mesh_info(h, 0, C.byref(nt), None, None)
        self.nt = int(nt.value)

    @classmethod
    def from_mesh(cls, m):
        return cls(m.xy, m.tri, m.canon, m.bc)

    def close(self):
        if getattr(self, "h", None):
            lib().dg_mesh_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def min_cfl_area(self, k, decomp=DECOMP_OPTIMAL):
        p1, p2 = dbl(), dbl()
        _check(lib().dg_mesh_info(self.h, decomp, None, C.byref(p1), C.byref(p2)))
        return p1.value if k == 1 else p2.value

    def neighbors(self):
        nbr = np.empty((self.nt, 3), np.int32)
        ne = np.empty((self.nt, 3), np.int32)
        _check(lib().dg_mesh_neighbors(self.h, _p(nbr), _p(ne)))
        return nbr, ne

    def geometry(self, k, decomp=DECOMP_OPTIMAL):
        nt = self.nt
        out = dict(area=np.empty(nt), len=np.empty((nt, 3)), normal=np.empty((nt, 3, 2)), c_area=np.empty(nt),
                   nodes=np.empty((nt, 2, 2)), limv=np.empty((nt, 2), np.int8))
        _check(lib().dg_mesh_geometry(self.h, k, decomp, *[_p(out[n]) for n in
                                                             ("area", "len", "normal", "c_area", "nodes", "limv")]))
        return out

    def quad_points(self):
        xy = np.empty((self.nt, 12, 2))
        _check(lib().dg_quad_points(self.h, _p(xy)))
        return xy

    def project(self, k, fn=None, cell_fn=None):
        if cell_fn is not None:
            vals = np.repeat(np.asarray(cell_fn(np.arange(self.nt)), np.float64)[:, None, :], 12, axis=1)
        else:
            xy = self.quad_points()
            vals = np.asarray(fn(xy[..., 0], xy[..., 1]), np.float64)
        vals = np.ascontiguousarray(vals.reshape(self.nt, 12, 4))
        u = np.empty((4, 3 if k == 1 else 6, self.nt))
        _check(lib().dg_project(self.h, k, _p(vals), _p(u)))
        return u


class Solver:
    """dg_solver handle: state resident on the GPU."""

    def __init__(self, mesh: Mesh, cfg: Config, coeffs, stream=None):
        self.mesh = mesh
        self.cfg = cfg
        self.nb = 3 if cfg.k == 1 else 6
        u = np.ascontiguousarray(coeffs, dtype=np.float64)
        assert u.size == 4 * self.nb * mesh.nt
        h = P()
        st = None if stream is None else P(stream)
        _check(lib().dg_init(mesh.h, C.byref(cfg), _p(u), st, C.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().dg_solver_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def stream(self):
        return lib().dg_stream(self.h)

    def advance(self, t_end, max_steps=1 << 62, check=True):
        st = Stats()
        rc = lib().dg_advance(self.h, t_end, max_steps, C.byref(st))
        if check:
            _check(rc)
        return st.as_dict() if not check else st.as_dict(), rc

    def advance_async(self, n):
        _check(lib().dg_advance_async(self.h, n))

    def sync(self):
        st = Stats()
        _check(lib().dg_sync(self.h, C.byref(st)))
        return st.as_dict()

    def get_state(self, out=None):
        """Host copy of the state; `out` (C-contiguous float64, e.g. pinned memory) is written in place."""
        u = np.empty((4, self.nb, self.mesh.nt)) if out is None else out
        if u.dtype != np.float64 or not u.flags["C_CONTIGUOUS"] or u.size != 4 * self.nb * self.mesh.nt:
            raise ValueError("out must be a C-contiguous float64 array of the state's size")
        t = dbl()
        _check(lib().dg_get_state(self.h, _p(u), u.size, C.byref(t)))
        return u, t.value

    def set_state(self, u, t=0.0):
        u = np.ascontiguousarray(u, dtype=np.float64)
        _check(lib().dg_set_state(self.h, _p(u), t))

    KERNEL_KINDS = ("step_begin", "rk", "fin_mean", "stats", "fin_dev", "oe_bp", "fin_alpha")

    def profile_steps(self, n):
        """n instrumented steps; per kernel kind: (summed ms, launches)."""
        ms = np.zeros(len(self.KERNEL_KINDS))
        nl = np.zeros(len(self.KERNEL_KINDS), np.int64)
        _check(lib().dg_profile_steps(self.h, n, _p(ms), _p(nl)))
        return {k: (float(ms[i]), int(nl[i])) for i, k in enumerate(self.KERNEL_KINDS)}

    # -- single operators (leave the solver state undefined) --------------------
    def op_rk_stage(self, un, v, a, b, dt, alpha, t=0.0):
        un = np.ascontiguousarray(un, np.float64); v = np.ascontiguousarray(v, np.float64)
        out = np.empty_like(v)
        _check(lib().dg_op_rk_stage(self.h, _p(un), _p(v), a, b, dt, alpha, t, _p(out)))
        return out

    def op_stats(self, u):
        u = np.ascontiguousarray(u, np.float64)
        st = np.empty(10)
        _check(lib().dg_op_stats(self.h, _p(u), _p(st)))
        return st

    def op_oe(self, u, dt, stats, t=0.0):
        u = np.ascontiguousarray(u, np.float64)
        out = np.empty_like(u)
        _check(lib().dg_op_oe(self.h, _p(u), dt, _p(np.ascontiguousarray(stats, np.float64)), t, _p(out)))
        return out

    def op_limit(self, u):
        u = np.ascontiguousarray(u, np.float64)
        out = np.empty_like(u)
        cnt = np.zeros(2, np.int64)
        _check(lib().dg_op_limit(self.h, _p(u), _p(out), _p(cnt)))
        return out, cnt

    def op_alpha(self, u, t=0.0):
        u = np.ascontiguousarray(u, np.float64)
        a = dbl()
        _check(lib().dg_op_alpha(self.h, _p(u), t, C.byref(a)))
        return a.value


class _SolverView(Solver):
    """A solver owned by a batch (not destroyed by Python)."""

    def __init__(self, mesh, cfg, h):
        self.mesh, self.cfg, self.nb, self.h = mesh, cfg, (3 if cfg.k == 1 else 6), h

    def close(self):
        self.h = None


class Batch:
    """dg_batch handle: independent solves advanced together, over one work
    list with one launch per phase (form 3) or one cooperative launch per stage
    (form 1), or as the solves' own step kernels in parallel branches of one
    graph per step (form 0)."""

    def __init__(self, meshes, cfgs, coeffs, stream=None):
        n = len(meshes)
        self.meshes, self.cfgs = list(meshes), list(cfgs)
        self._u = [np.ascontiguousarray(u, np.float64) for u in coeffs]
        mh = (P * n)(*[m.h for m in meshes])
        cf = (Config * n)(*cfgs)
        up = (P * n)(*[_p(u) for u in self._u])
        h = P()
        _check(lib().dg_batch_create(n, C.cast(mh, P), C.cast(cf, P), C.cast(up, P),
                                     None if stream is None else P(stream), C.byref(h)))
        self.h = h
        self.n = n

    def close(self):
        if getattr(self, "h", None):
            lib().dg_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solver(self, i):
        s = P()
        _check(lib().dg_batch_solver(self.h, i, C.byref(s)))
        return _SolverView(self.meshes[i], self.cfgs[i], s)

    def advance(self, t_end=None, max_steps=1 << 62):
        te = None if t_end is None else np.ascontiguousarray(np.broadcast_to(t_end, (self.n,)), np.float64)
        st = (Stats * self.n)()
        _check(lib().dg_batch_advance(self.h, _p(te), max_steps, C.cast(st, P)))
        return [s.as_dict() for s in st]

    def advance_async(self, n):
        _check(lib().dg_batch_advance_async(self.h, n))

    def sync(self):
        _check(lib().dg_batch_sync(self.h))

    def set_barrier(self, timeout_ns=2_000_000_000, extra_arrivals=0):
        """Wait limit of the cooperative form's grid barriers; extra_arrivals > 0
        (tests only) makes every barrier wait run out."""
        _check(lib().dg_batch_set_barrier(self.h, int(timeout_ns), int(extra_arrivals)))

    def set_shape(self, cells_per_block, blocks_per_sm, launches_per_stage=3):
        _check(lib().dg_batch_set_shape(self.h, cells_per_block, blocks_per_sm, launches_per_stage))

    def shape(self):
        a, b, f, g, gr = i32(), i32(), i32(), i32(), i32()
        _check(lib().dg_batch_shape(self.h, C.byref(a), C.byref(b), C.byref(f), C.byref(g), C.byref(gr)))
        return dict(cells_per_block=a.value, blocks_per_sm=b.value, launches_per_stage=f.value, grid=g.value,
                    graph=bool(gr.value))

    def autotune(self, steps=3):
        a, b, f, ms = i32(), i32(), i32(), dbl()
        _check(lib().dg_batch_autotune(self.h, steps, C.byref(a), C.byref(b), C.byref(f), C.byref(ms)))
        return dict(cells_per_block=a.value, blocks_per_sm=b.value, launches_per_stage=f.value,
                    ms_per_step=ms.value)


REQ_QUEUED, REQ_RUNNING, REQ_DONE, REQ_FAILED = 0, 1, 2, 3


class RequestInfo(C.Structure):
    _fields_ = [("state", i32), ("error", i32), ("cells", i64), ("steps", i64), ("t", dbl), ("t_end", dbl),
                ("submit_s", dbl), ("start_s", dbl), ("done_s", dbl), ("device_bytes", i64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class Server:
    """dg_server handle: continuous batching of solve requests."""

    def __init__(self, precision=PREC_FP64, budget_bytes=8 << 30, steps_per_tick=8, stream=None):
        h = P()
        _check(lib().dg_server_create(precision, budget_bytes, steps_per_tick,
                                      None if stream is None else P(stream), C.byref(h)))
        self.h = h
        self._nb = {}

    def close(self):
        if getattr(self, "h", None):
            lib().dg_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, mesh, cfg, coeffs, t_end):
        """mesh: a workloads.Mesh (host arrays); returns the request id."""
        xy = np.ascontiguousarray(mesh.xy, np.float64)
        tri = np.ascontiguousarray(mesh.tri, np.int32)
        canon = np.ascontiguousarray(mesh.canon, np.int32)
        bc = np.ascontiguousarray(mesh.bc, np.int8)
        u = np.ascontiguousarray(coeffs, np.float64)
        rid = i64()
        _check(lib().dg_server_submit(self.h, xy.shape[0], _p(xy), tri.shape[0], _p(tri), _p(canon), _p(bc),
                                      C.byref(cfg), _p(u), t_end, C.byref(rid)))
        self._nb[rid.value] = (u.shape, tri.shape[0])
        return rid.value

    def tick(self):
        r, q = i32(), i32()
        _check(lib().dg_server_tick(self.h, C.byref(r), C.byref(q)))
        return r.value, q.value

    def info(self, rid):
        inf = RequestInfo()
        _check(lib().dg_server_request(self.h, rid, C.byref(inf)))
        return inf.as_dict()

    def result(self, rid):
        shape, _ = self._nb[rid]
        out = np.empty(shape)
        _check(lib().dg_server_result(self.h, rid, _p(out), out.size))
        return out

    def stats(self):
        a, b = i64(), i64()
        _check(lib().dg_server_stats(self.h, C.byref(a), C.byref(b)))
        return dict(bytes_in_use=a.value, cell_stages_done=b.value)


def make_scalar_config(k, flux=FLUX_LINEAR, oe=1, rk=None, ax=1.0, ay=1.0, cfl=1.0, bc_state=(0.0, 0.0, 0.0, 0.0)):
    """Scalar OEDG configuration; rk defaults to SSP-RK(2,2) for P1 and
    SSP-RK(3,3) otherwise."""
    cf = ScalarConfig()
    cf.k, cf.flux, cf.oe = k, flux, oe
    cf.rk = (2 if k == 1 else 3) if rk is None else rk
    cf.ax, cf.ay, cf.cfl = ax, ay, cfl
    for i in range(4):
        cf.bc_state[i] = float(bc_state[i])
    return cf


def scalar_project(mesh: Mesh, k, fn):
    """L2 projection of a point-wise scalar fn(x, y) with the library's 12-point rule."""
    xy = mesh.quad_points()
    vals = np.ascontiguousarray(np.asarray(fn(xy[..., 0], xy[..., 1]), np.float64).reshape(mesh.nt, 12))
    u = np.empty(((k + 1) * (k + 2) // 2, mesh.nt))
    _check(lib().dg_scalar_project(mesh.h, k, _p(vals), _p(u)))
    return u


class ScalarSolver:
    """dg_scalar handle: the scalar OEDG solver, state resident on the GPU."""

    def __init__(self, mesh: Mesh, cfg: ScalarConfig, coeffs, stream=None):
        self.mesh = mesh
        self.cfg = cfg
        self.nb = (cfg.k + 1) * (cfg.k + 2) // 2
        u = np.ascontiguousarray(coeffs, dtype=np.float64)
        if u.size != self.nb * mesh.nt:
            raise ValueError("coefficient array has the wrong size")
        h = P()
        _check(lib().dg_scalar_init(mesh.h, C.byref(cfg), _p(u), stream, C.byref(h)))
        self.h = h

    @property
    def stream(self):
        return lib().dg_scalar_stream(self.h)

    def advance(self, t_end, max_steps=1 << 62):
        st = Stats()
        _check(lib().dg_scalar_advance(self.h, t_end, max_steps, C.byref(st)))
        return st.as_dict()

    def advance_async(self, n):
        _check(lib().dg_scalar_advance_async(self.h, n))

    def get_state(self):
        u = np.empty((self.nb, self.mesh.nt))
        t = dbl()
        _check(lib().dg_scalar_get_state(self.h, _p(u), u.size, C.byref(t)))
        return u, t.value

    def errors(self, exact_values):
        """(L1, L2, Linf) against exact values [nt, 12] at the mesh's quad points."""
        ex = np.ascontiguousarray(np.asarray(exact_values, np.float64).reshape(self.mesh.nt, 12))
        out = np.empty(3)
        _check(lib().dg_scalar_errors(self.h, _p(ex), _p(out)))
        return tuple(float(v) for v in out)

    def close(self):
        if getattr(self, "h", None):
            lib().dg_scalar_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def initial_state(mesh: Mesh, workload):
    """Projection of a workload's initial data with the library's own projection."""
    return mesh.project(workload.k, fn=workload.u0, cell_fn=workload.cell_u0)

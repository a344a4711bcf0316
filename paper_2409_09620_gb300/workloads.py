"""Seeded synthetic inputs: jittered triangulations and initial states.

This module holds no arithmetic of the DG method.  It builds the inputs that
both the CUDA path and the CPU oracle consume:

* a structured ``nx x ny`` grid on a rectangle, each square split along a
  seeded random diagonal, interior vertices moved by ``U(-0.2h, 0.2h)`` per
  coordinate (boundary vertices and listed fixed points stay put);
* counter-clockwise triangles, a periodic vertex identity map ``canon`` and a
  per-edge boundary tag (edge ``i`` of a triangle is the edge opposite its
  vertex ``i``, as in the paper's Fig. 1);
* point-wise initial states in conservative variables ``(rho, m1, m2, E)``
  for the isentropic vortex, the Sedov-type blast, the 60-degree double Mach
  reflection and the four-quadrant Riemann problem;
* near-equilateral lattice triangulations of non-rectangular domains (the
  paper's forward-facing-step tunnel and 30-degree wedge) with their
  boundary conditions.

Projection of a point-wise state onto the modal basis is method arithmetic
and lives on each side of the boundary separately.

The paper's EasyMesh meshes are not available; these jittered grids stand in
for them.  Random numbers come from numpy's PCG64 generator with the seed
recorded by the caller.
"""
from __future__ import annotations

import functools
import math
from dataclasses import dataclass, field

import numpy as np

# Boundary tags of an edge without a neighbour (an interface shared with the
# C ABI; the numeric values are fixed there).
BC_NONE = 0          # must have a neighbour (interior or periodic via canon)
BC_REFLECT = 1
BC_TRANSMISSIVE = 2
BC_DIRICHLET0 = 3    # constant states 0..3 -> tags 3..6
BC_SHOCK = 7         # moving oblique shock (double Mach reflection top wall)

GAMMA = 1.4


@dataclass
class Mesh:
    xy: np.ndarray            # float64 [nv, 2]
    tri: np.ndarray           # int32 [nt, 3], counter-clockwise
    canon: np.ndarray         # int32 [nv]
    bc: np.ndarray            # int8 [nt, 3], tag of the edge opposite vertex i
    nx: int = 0
    ny: int = 0
    box: tuple = (0.0, 1.0, 0.0, 1.0)
    meta: dict = field(default_factory=dict)

    @property
    def nv(self) -> int:
        return int(self.xy.shape[0])

    @property
    def nt(self) -> int:
        return int(self.tri.shape[0])


def jittered_grid(nx: int, ny: int, box=(0.0, 1.0, 0.0, 1.0), seed: int = 0,
                  jitter: float = 0.2, periodic: bool = False,
                  fixed_points=(), side_tags=None) -> Mesh:
    """Jittered structured triangulation of ``box = (x0, x1, y0, y1)``.

    ``side_tags`` maps a side name ('left', 'right', 'bottom', 'top') to a
    boundary tag or to a callable ``f(xmid, ymid) -> tag`` evaluated at the
    edge midpoint.  With ``periodic=True`` opposite sides are identified
    through ``canon`` and no side tags are needed.
    """
    if nx < 2 or ny < 2:
        raise ValueError("need nx, ny >= 2")
    x0, x1, y0, y1 = box
    hx = (x1 - x0) / nx
    hy = (y1 - y0) / ny
    rng = np.random.default_rng(seed)
    ii, jj = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), indexing="xy")
    ii = ii.reshape(-1)
    jj = jj.reshape(-1)
    xy = np.stack([x0 + ii * hx, y0 + jj * hy], axis=1).astype(np.float64)
    interior = (ii > 0) & (ii < nx) & (jj > 0) & (jj < ny)
    for (px, py) in fixed_points:
        hit = (np.abs(xy[:, 0] - px) < 1e-12 * max(1.0, abs(px))) & \
              (np.abs(xy[:, 1] - py) < 1e-12 * max(1.0, abs(py)))
        interior &= ~hit
    dj = rng.uniform(-jitter, jitter, size=(xy.shape[0], 2))
    dj[~interior] = 0.0
    xy[:, 0] += dj[:, 0] * hx
    xy[:, 1] += dj[:, 1] * hy

    def vid(i, j):
        return j * (nx + 1) + i

    qi, qj = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    qi = qi.reshape(-1)
    qj = qj.reshape(-1)
    v00 = vid(qi, qj)
    v10 = vid(qi + 1, qj)
    v01 = vid(qi, qj + 1)
    v11 = vid(qi + 1, qj + 1)
    diag = rng.integers(0, 2, size=qi.shape[0])
    tri = np.empty((2 * qi.shape[0], 3), dtype=np.int32)
    a = diag == 0
    # diagonal v00-v11: (v00, v10, v11), (v00, v11, v01)
    tri[0::2][a] = np.stack([v00[a], v10[a], v11[a]], axis=1)
    tri[1::2][a] = np.stack([v00[a], v11[a], v01[a]], axis=1)
    b = ~a
    # diagonal v10-v01: (v00, v10, v01), (v10, v11, v01)
    tri[0::2][b] = np.stack([v00[b], v10[b], v01[b]], axis=1)
    tri[1::2][b] = np.stack([v10[b], v11[b], v01[b]], axis=1)

    if periodic:
        canon = (jj % ny) * (nx + 1) + (ii % nx)
    else:
        canon = np.arange(xy.shape[0])
    canon = canon.astype(np.int32)

    bc = np.zeros(tri.shape, dtype=np.int8)
    if not periodic:
        side_tags = side_tags or {}
        # edge e opposite local vertex e joins local vertices e+1, e+2
        for e in range(3):
            va = tri[:, (e + 1) % 3]
            vb = tri[:, (e + 2) % 3]
            ia, ja = ii[va], jj[va]
            ib, jb = ii[vb], jj[vb]
            xm = 0.5 * (xy[va, 0] + xy[vb, 0])
            ym = 0.5 * (xy[va, 1] + xy[vb, 1])
            for side, sel in (("left", (ia == 0) & (ib == 0)),
                              ("right", (ia == nx) & (ib == nx)),
                              ("bottom", (ja == 0) & (jb == 0)),
                              ("top", (ja == ny) & (jb == ny))):
                if not sel.any():
                    continue
                tag = side_tags.get(side, BC_TRANSMISSIVE)
                if callable(tag):
                    bc[sel, e] = np.asarray([tag(x, y) for x, y in zip(xm[sel], ym[sel])],
                                            dtype=np.int8)
                else:
                    bc[sel, e] = tag
    return Mesh(xy=xy, tri=tri, canon=canon, bc=bc, nx=nx, ny=ny, box=tuple(box),
                meta={"seed": seed, "jitter": jitter, "periodic": periodic})


# ----------------------------------------------------------------------------
# Near-equilateral lattice triangulations of non-rectangular domains
# ----------------------------------------------------------------------------

def _lattice_row(x0, x1, h, offset, required, rng, jitter):
    """Sorted x positions of one row on [x0, x1]: the end points, the required
    points, and the lattice points j h + offset at least 0.7 h away from them,
    each moved by U(-jitter, jitter) h."""
    fixed = sorted({x0, x1, *[r for r in required if x0 <= r <= x1]})
    cand = offset + h * np.arange(math.ceil((x0 - offset) / h), math.floor((x1 - offset) / h) + 1)
    keep = np.ones(cand.shape, bool)
    for f in fixed:
        keep &= np.abs(cand - f) > 0.7 * h
    cand = cand[keep] + rng.uniform(-jitter, jitter, int(keep.sum())) * h
    return np.unique(np.concatenate([np.asarray(fixed, dtype=np.float64), cand]))


def _rows(y0, y1, dy):
    n = max(1, int(round((y1 - y0) / dy)))
    return [y0 + (y1 - y0) * r / n for r in range(n + 1)]


def lattice_mesh(ys, spans, strips, h, seed=0, jitter=0.1, required=(), classify=None) -> Mesh:
    """Triangulation of a domain swept by horizontal rows of points.

    Row r lies at height ``ys[r]`` and spans ``spans[r] = (x0, x1)``; its
    points are a lattice of spacing ``h`` shifted by h/2 on odd rows (so the
    triangles are close to equilateral when the row spacing is about
    h sqrt(3)/2), plus the span's end points and the ``required`` (x, y)
    points on that row.  The strip between rows r and r+1 joins the points of
    row r within ``strips[r][0]`` and those of row r+1 within ``strips[r][1]``
    (x-ranges) by a zipper: walking left to right, the next triangle takes the
    next point of whichever row has the smaller x.  Boundary edges (used by
    one triangle) get ``classify(pa, pb) -> tag``.
    """
    rng = np.random.default_rng(seed)
    rows, base, pts = [], [], []
    for r, y in enumerate(ys):
        req = [x for (x, yy) in required if abs(yy - y) < 1e-12]
        xs = _lattice_row(spans[r][0], spans[r][1], h, 0.5 * h * (r % 2), req, rng, jitter)
        base.append(sum(len(q) for q in rows))
        rows.append(xs)
        pts.append(np.stack([xs, np.full(xs.shape, y)], axis=1))
    xy = np.concatenate(pts).astype(np.float64)
    tris = []
    for r in range(len(ys) - 1):
        (aL, bL), (aU, bU) = strips[r]
        xl, xu = rows[r], rows[r + 1]
        lo = base[r] + np.nonzero((xl >= aL - 1e-12) & (xl <= bL + 1e-12))[0]
        up = base[r + 1] + np.nonzero((xu >= aU - 1e-12) & (xu <= bU + 1e-12))[0]
        xlo, xup = xy[lo, 0], xy[up, 0]
        i = j = 0
        nl, nu = len(lo) - 1, len(up) - 1
        out = []
        while i < nl or j < nu:
            if j == nu or (i < nl and xlo[i + 1] <= xup[j + 1]):
                out.append((lo[i], lo[i + 1], up[j]))   # counter-clockwise: lower edge, then up
                i += 1
            else:
                out.append((lo[i], up[j + 1], up[j]))
                j += 1
        tris.append(np.asarray(out, dtype=np.int64))
    tri = np.concatenate(tris).astype(np.int32)
    # boundary edges: edges used by one triangle
    bc = np.zeros(tri.shape, dtype=np.int8)
    a = tri[:, [1, 2, 0]].reshape(-1).astype(np.int64)
    b = tri[:, [2, 0, 1]].reshape(-1).astype(np.int64)
    key = np.minimum(a, b) * xy.shape[0] + np.maximum(a, b)
    _, inv, cnt = np.unique(key, return_inverse=True, return_counts=True)
    once = np.nonzero(cnt[inv] == 1)[0]
    tags = np.asarray([classify(xy[a[e]], xy[b[e]]) for e in once], dtype=np.int8)
    bc.reshape(-1)[once] = tags
    return Mesh(xy=xy, tri=tri, canon=np.arange(xy.shape[0], dtype=np.int32), bc=bc,
                box=(min(s[0] for s in spans), max(s[1] for s in spans), ys[0], ys[-1]),
                meta={"seed": seed, "jitter": jitter, "h": h, "lattice": True})


def ffs_mesh(h=1.0 / 112, seed=21):
    """Wind tunnel [0, 3] x [0, 1] with a step of height 0.2 from x = 0.6
    (Sec. 5, flow past a forward facing step): inflow (constant state 0) at
    x = 0, outflow at x = 3, reflecting walls elsewhere."""
    dy = h * math.sqrt(3.0) / 2.0
    lo, hi = _rows(0.0, 0.2, dy), _rows(0.2, 1.0, dy)
    ys = lo + hi[1:]
    nlo = len(lo) - 1
    spans = [(0.0, 0.6) if r < nlo else (0.0, 3.0) for r in range(len(ys))]
    strips = [((0.0, 0.6), (0.0, 0.6)) if r < nlo else ((0.0, 3.0), (0.0, 3.0)) for r in range(len(ys) - 1)]

    def classify(pa, pb):
        if pa[0] == 0.0 and pb[0] == 0.0:
            return BC_DIRICHLET0
        if pa[0] == 3.0 and pb[0] == 3.0:
            return BC_TRANSMISSIVE
        return BC_REFLECT
    return lattice_mesh(ys, spans, strips, h, seed=seed, required=[(0.6, 0.2)], classify=classify)


def wedge_mesh(h=1.0 / 320, seed=22, x_wedge=0.1, length=2.8, height=2.0):
    """Tube [0, length] x [0, height] over a 30-degree wedge rising from
    (x_wedge, 0) (Sec. 5, double Mach reflection): inflow (constant state 0)
    at x = 0, outflow at x = length, the moving-shock exact solution on the top
    and on the bottom segment before the wedge, reflection on the wedge."""
    dy = h * math.sqrt(3.0) / 2.0
    s3 = math.sqrt(3.0)
    yc = (length - x_wedge) / s3                       # where the wedge meets the outflow side
    ys = _rows(0.0, yc, dy) + _rows(yc, height, dy)[1:]
    xe = lambda y: min(length, x_wedge + y * s3)
    spans = [(0.0, xe(y)) for y in ys]
    strips = [((0.0, xe(ys[r])), (0.0, xe(ys[r + 1]))) for r in range(len(ys) - 1)]

    def classify(pa, pb):
        if pa[0] == 0.0 and pb[0] == 0.0:
            return BC_DIRICHLET0
        if pa[0] == length and pb[0] == length:
            return BC_TRANSMISSIVE
        if (pa[1] == height and pb[1] == height) or (pa[1] == 0.0 and pb[1] == 0.0):
            return BC_SHOCK
        return BC_REFLECT
    return lattice_mesh(ys, spans, strips, h, seed=seed, classify=classify)


def refine_mesh(mesh: Mesh) -> Mesh:
    """Split every triangle into four through its edge midpoints (the paper's
    refinement of its scalar meshes, Sec. 5).  Midpoints of the two copies of
    a periodic edge are identified through ``canon``; boundary edges keep
    their tags on both halves."""
    xy = [tuple(p) for p in mesh.xy]
    canon = list(mesh.canon)
    mids, cmid = {}, {}

    def mid(a, b):
        key = (min(a, b), max(a, b))
        if key not in mids:
            mids[key] = len(xy)
            xy.append(tuple(0.5 * (mesh.xy[a] + mesh.xy[b])))
            ck = (min(mesh.canon[a], mesh.canon[b]), max(mesh.canon[a], mesh.canon[b]))
            canon.append(cmid.setdefault(ck, mids[key]))
        return mids[key]
    tri, bc = [], []
    for (a, b, c), (ta, tb, tc) in zip(mesh.tri, mesh.bc):
        ma, mb, mc = mid(b, c), mid(c, a), mid(a, b)
        tri += [(a, mc, mb), (mc, b, ma), (mb, ma, c), (ma, mb, mc)]
        bc += [(0, tb, tc), (ta, 0, tc), (ta, tb, 0), (0, 0, 0)]
    return Mesh(xy=np.asarray(xy, dtype=np.float64), tri=np.asarray(tri, dtype=np.int32),
                canon=np.asarray(canon, dtype=np.int32), bc=np.asarray(bc, dtype=np.int8),
                box=mesh.box, meta={**mesh.meta, "refined": mesh.meta.get("refined", 0) + 1})


@functools.lru_cache(maxsize=8)
def scalar_mesh(level: int, n0: int = 5, seed: int = 31) -> Mesh:
    """Periodic unit square: a jittered n0 x n0 grid (2 n0^2 = 50 cells, about
    the paper's 44-cell coarsest mesh) refined ``level`` times."""
    m = jittered_grid(n0, n0, (0.0, 1.0, 0.0, 1.0), seed=seed, periodic=True)
    for _ in range(level):
        m = refine_mesh(m)
    return m


def linear_smooth(x, y, t=0.0):
    """u_t + u_x + u_y = 0 from sin(2 pi (x + y)) (Sec. 5, smooth linear problem)."""
    return np.sin(2.0 * np.pi * (np.asarray(x) + np.asarray(y) - 2.0 * t))


def burgers_smooth(x, y, t=0.0, iters=60):
    """u_t + (u^2/2)_x + (u^2/2)_y = 0 from 0.5 sin(2 pi (x + y)) (Sec. 5),
    exact while smooth (t < 1 / (2 pi)): u = 0.5 sin(2 pi (x + y - 2 u t)),
    solved by Newton's method along the characteristics."""
    s = np.asarray(x, dtype=np.float64) + np.asarray(y, dtype=np.float64)
    u = 0.5 * np.sin(2.0 * np.pi * s)
    for _ in range(iters):
        ph = 2.0 * np.pi * (s - 2.0 * u * t)
        g = u - 0.5 * np.sin(ph)
        u = u - g / (1.0 + 2.0 * np.pi * t * np.cos(ph))
    return u


@dataclass
class ScalarWorkload:
    name: str
    mesh: Mesh
    k: int
    flux: int                  # 0 linear (velocity (1, 1)), 1 Burgers
    t_end: float
    u0: object                 # callable (x, y) -> values
    exact: object = None       # callable (x, y, t) -> values, where known
    bc_state: tuple = (0.0, 0.0, 0.0, 0.0)


def scalar_linear_workload(level=3, k=2):
    return ScalarWorkload(name=f"linear_L{level}_P{k}", mesh=scalar_mesh(level), k=k, flux=0, t_end=0.1,
                          u0=lambda x, y: linear_smooth(x, y), exact=linear_smooth)


def scalar_burgers_workload(level=3, k=2):
    return ScalarWorkload(name=f"burgers_L{level}_P{k}", mesh=scalar_mesh(level), k=k, flux=1, t_end=0.05,
                          u0=lambda x, y: burgers_smooth(x, y), exact=burgers_smooth)


def burgers_riemann2_workload(n=64, k=2, seed=32):
    """Burgers Riemann problem II (Sec. 5): 2 for x, y < 0.25, 3 for x, y >=
    0.25, 1 elsewhere; inflow (the initial values) on the left and bottom
    sides, outflow on the right and top, to t = 1/12."""
    inflow = lambda x, y: BC_DIRICHLET0 if (x < 0.25 and y < 0.25) else BC_DIRICHLET0 + 1
    mesh = jittered_grid(n, n, (0.0, 1.0, 0.0, 1.0), seed=seed,
                         side_tags={"left": lambda x, y: BC_DIRICHLET0 if y < 0.25 else BC_DIRICHLET0 + 1,
                                    "bottom": lambda x, y: BC_DIRICHLET0 if x < 0.25 else BC_DIRICHLET0 + 1,
                                    "right": BC_TRANSMISSIVE, "top": BC_TRANSMISSIVE})
    del inflow

    def u0(x, y):
        x = np.asarray(x, dtype=np.float64)
        y = np.asarray(y, dtype=np.float64)
        return np.where((x < 0.25) & (y < 0.25), 2.0, np.where((x >= 0.25) & (y >= 0.25), 3.0, 1.0))
    return ScalarWorkload(name=f"burgers_rm2_{n}_P{k}", mesh=mesh, k=k, flux=1, t_end=1.0 / 12.0, u0=u0,
                          bc_state=(2.0, 1.0, 0.0, 0.0))


# ----------------------------------------------------------------------------
# Point-wise initial states (conservative variables), vectorised over points.
# ----------------------------------------------------------------------------

def prim_to_cons(rho, u, v, p, gamma=GAMMA):
    rho = np.asarray(rho, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64)
    v = np.asarray(v, dtype=np.float64)
    p = np.asarray(p, dtype=np.float64)
    E = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)
    return np.stack(np.broadcast_arrays(rho, rho * u, rho * v, E), axis=-1)


def vortex_state(x, y, t=0.0, strength=5.0, radius=0.1, center=(0.5, 0.5),
                 background=(1.0, 1.0, 1.0, 1.0), box=(0.0, 1.0, 0.0, 1.0),
                 gamma=GAMMA, images=1):
    """Isentropic vortex advected by the background flow on a periodic box.

    The classic vortex on [-5, 5]^2 mapped to a radius scale ``radius``:
    with r' = |x - x_c(t)| / radius,
    dv = strength/(2 pi) exp((1 - r'^2)/2) (-y', x'),
    T = 1 - (gamma-1) strength^2 / (8 gamma pi^2) exp(1 - r'^2),
    rho = T^(1/(gamma-1)), p = rho T  (for rho_inf = p_inf = 1).
    Periodic images within ``images`` box lengths are summed in the velocity
    and temperature perturbations.
    """
    rho0, u0, v0, p0 = background
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    Lx = box[1] - box[0]
    Ly = box[3] - box[2]
    cx = box[0] + ((center[0] + u0 * t - box[0]) % Lx)
    cy = box[2] + ((center[1] + v0 * t - box[2]) % Ly)
    du = np.zeros_like(x)
    dv = np.zeros_like(x)
    dT = np.zeros_like(x)
    for a in range(-images, images + 1):
        for b in range(-images, images + 1):
            xr = (x - (cx + a * Lx)) / radius
            yr = (y - (cy + b * Ly)) / radius
            r2 = xr * xr + yr * yr
            f = strength / (2.0 * math.pi) * np.exp(0.5 * (1.0 - r2))
            du += -yr * f
            dv += xr * f
            dT += -(gamma - 1.0) * strength ** 2 / (8.0 * gamma * math.pi ** 2) * np.exp(1.0 - r2)
    T = p0 / rho0 + dT
    rho = rho0 * (T / (p0 / rho0)) ** (1.0 / (gamma - 1.0))
    p = rho * T
    return prim_to_cons(rho, u0 + du, v0 + dv, p, gamma)


def dmr_states(gamma=GAMMA):
    """Post- and pre-shock states of the Mach-10 double Mach reflection.

    The post-shock velocity (8.25 along the shock normal) is split with the
    shock inclined at 60 degrees to the x-axis: (8.25 cos30, -8.25 sin30).
    """
    post = prim_to_cons(8.0, 8.25 * math.cos(math.pi / 6), -8.25 * math.sin(math.pi / 6), 116.5, gamma)
    pre = prim_to_cons(1.4, 0.0, 0.0, 1.0, gamma)
    return post.reshape(4), pre.reshape(4)


# ----------------------------------------------------------------------------
# Workload recipes (mesh + point-wise initial state + configuration)
# ----------------------------------------------------------------------------

@dataclass
class Workload:
    name: str
    mesh: Mesh
    k: int
    t_end: float
    u0: object                 # callable (x, y) -> [.., 4] conservative state
    cell_u0: object = None     # optional callable (cell ids) -> [.., 4] piecewise-constant state
    bc_state: np.ndarray = field(default_factory=lambda: np.zeros((4, 4)))
    shock: tuple = (0.0, 0.0, 0.0, 0, 0)   # x0, angle, speed, pre index, post index
    gamma: float = GAMMA


def vortex_workload(n=32, k=1, seed=1, radius=0.1, t_end=0.5, strength=5.0):
    mesh = jittered_grid(n, n, (0.0, 1.0, 0.0, 1.0), seed=seed, periodic=True)
    return Workload(name=f"vortex{n}x{n}_P{k}", mesh=mesh, k=k, t_end=t_end,
                    u0=lambda x, y: vortex_state(x, y, 0.0, strength=strength, radius=radius))


def sedov_workload(n=256, k=2, seed=2, t_end=1.0, energy=0.244816, p_floor=1e-10):
    L = 1.1
    mesh = jittered_grid(n, n, (-L, L, -L, L), seed=seed, fixed_points=[(0.0, 0.0)],
                         side_tags={s: BC_REFLECT for s in ("left", "right", "bottom", "top")})
    xy = mesh.xy
    origin = np.argmin(xy[:, 0] ** 2 + xy[:, 1] ** 2)
    touch = np.any(mesh.tri == origin, axis=1)
    x0 = xy[mesh.tri[:, 0]]
    x1 = xy[mesh.tri[:, 1]]
    x2 = xy[mesh.tri[:, 2]]
    area = 0.5 * ((x1[:, 0] - x0[:, 0]) * (x2[:, 1] - x0[:, 1]) - (x2[:, 0] - x0[:, 0]) * (x1[:, 1] - x0[:, 1]))
    p_blast = (GAMMA - 1.0) * energy / area[touch].sum()
    p_cell = np.where(touch, p_blast, p_floor)
    cons = prim_to_cons(np.ones(mesh.nt), np.zeros(mesh.nt), np.zeros(mesh.nt), p_cell)

    def cell_u0(cells):
        return cons[np.asarray(cells)]
    return Workload(name=f"sedov{n}x{n}_P{k}", mesh=mesh, k=k, t_end=t_end,
                    u0=None, cell_u0=cell_u0)


def dmr_workload(nx=1440, ny=360, k=2, seed=3, t_end=0.2, right=BC_DIRICHLET0 + 1):
    """60-degree double Mach reflection on [0, 4] x [0, 1].  The right side
    holds the pre-shock state (tag 4), which is the exact solution there until
    the incident shock reaches x = 4 at t ~ 0.28; right=BC_TRANSMISSIVE gives
    the zero-gradient outflow instead (the cell average as exterior state)."""
    post, pre = dmr_states()
    x0 = 1.0 / 6.0
    bottom = lambda x, y: BC_DIRICHLET0 if x < x0 else BC_REFLECT
    mesh = jittered_grid(nx, ny, (0.0, 4.0, 0.0, 1.0), seed=seed,
                         side_tags={"left": BC_DIRICHLET0, "right": right,
                                    "bottom": bottom, "top": BC_SHOCK})
    bc_state = np.zeros((4, 4))
    bc_state[0] = post
    bc_state[1] = pre
    s3 = math.sqrt(3.0)

    def u0(x, y):
        x = np.asarray(x, dtype=np.float64)
        y = np.asarray(y, dtype=np.float64)
        behind = x < x0 + y / s3
        return np.where(behind[..., None], post, pre)
    return Workload(name=f"dmr{nx}x{ny}_P{k}", mesh=mesh, k=k, t_end=t_end, u0=u0,
                    bc_state=bc_state, shock=(x0, math.pi / 3.0, 10.0, 1, 0))


def riemann4_workload(n=64, k=1, seed=4, t_end=0.2):
    rng = np.random.default_rng(seed + 1000)
    rho = rng.uniform(0.1, 2.0, 4)
    p = rng.uniform(0.01, 2.0, 4)
    u = rng.uniform(-1.0, 1.0, 4)
    v = rng.uniform(-1.0, 1.0, 4)
    states = prim_to_cons(rho, u, v, p)
    mesh = jittered_grid(n, n, (0.0, 1.0, 0.0, 1.0), seed=seed,
                         side_tags={s: BC_TRANSMISSIVE for s in ("left", "right", "bottom", "top")})

    def u0(x, y):
        x = np.asarray(x, dtype=np.float64)
        y = np.asarray(y, dtype=np.float64)
        q = (x >= 0.5).astype(int) + 2 * (y >= 0.5).astype(int)
        return states[q]
    return Workload(name=f"riemann4_{n}x{n}_P{k}", mesh=mesh, k=k, t_end=t_end, u0=u0)


def uniform_workload(n=16, k=2, seed=5, state=(1.0, 0.3, -0.2, 2.5), periodic=True):
    mesh = jittered_grid(n, n, (0.0, 1.0, 0.0, 1.0), seed=seed, periodic=periodic,
                         side_tags=None if periodic else
                         {s: BC_TRANSMISSIVE for s in ("left", "right", "bottom", "top")})
    st = np.asarray(state, dtype=np.float64)
    return Workload(name=f"uniform{n}_P{k}", mesh=mesh, k=k, t_end=0.1,
                    u0=lambda x, y: np.broadcast_to(st, np.shape(x) + (4,)).copy())


def ffs_workload(h=1.0 / 112, k=2, seed=21, t_end=4.0):
    """Mach 3 flow past a forward facing step (Sec. 5): uniform
    (rho, v1, v2, p) = (1.4, 3, 0, 1), which is also the inflow state.  The
    paper's mesh (73,862 cells, h = 1/80 refined to 1/320 near the corner) is
    not available; the default h = 1/112 gives a uniform lattice mesh of about
    the same cell count."""
    mesh = ffs_mesh(h, seed)
    inflow = prim_to_cons(1.4, 3.0, 0.0, 1.0).reshape(4)
    bc_state = np.zeros((4, 4))
    bc_state[0] = inflow
    return Workload(name=f"ffs_h{round(1.0 / h)}_P{k}", mesh=mesh, k=k, t_end=t_end,
                    u0=lambda x, y: np.broadcast_to(inflow, np.shape(x) + (4,)).copy(), bc_state=bc_state)


def wedge_dmr_workload(h=1.0 / 320, k=2, seed=22, t_end=0.2):
    """Double Mach reflection in a tube over a 30-degree wedge (Sec. 5): a
    Mach-10 shock at x = 0.1 moving right, post-shock (8, 8.25, 0, 116.5)
    behind it and (1.4, 0, 0, 1) ahead.  The default h = 1/320 gives about the
    paper's 828,840 cells."""
    mesh = wedge_mesh(h, seed)
    post = prim_to_cons(8.0, 8.25, 0.0, 116.5).reshape(4)
    pre = prim_to_cons(1.4, 0.0, 0.0, 1.0).reshape(4)
    bc_state = np.zeros((4, 4))
    bc_state[0] = post
    bc_state[1] = pre

    def u0(x, y):
        x = np.asarray(x, dtype=np.float64)
        return np.where((x <= 0.1)[..., None], post, pre)
    return Workload(name=f"wedge_dmr_h{round(1.0 / h)}_P{k}", mesh=mesh, k=k, t_end=t_end, u0=u0,
                    bc_state=bc_state, shock=(0.1, math.pi / 2.0, 10.0, 1, 0))


def random_modal_state(nt: int, k: int, seed: int, mean=(1.0, 0.2, -0.1, 2.5),
                       amp=0.05, mean_jitter=0.1):
    """Random modal coefficients [4][nb][nt] with a positive mean state.

    Used for parity tests only (a perturbation of a constant state, so that
    density and pressure stay positive at every point).
    """
    nb = 3 if k == 1 else 6
    rng = np.random.default_rng(seed)
    u = np.zeros((4, nb, nt))
    mean = np.asarray(mean, dtype=np.float64)
    u[:, 0, :] = mean[:, None] * (1.0 + mean_jitter * rng.uniform(-1, 1, (4, nt)))
    u[:, 1:, :] = amp * np.abs(mean)[:, None, None] * rng.uniform(-1, 1, (4, nb - 1, nt))
    return u


def batch_workloads(n=64, seed=7, cmin=2000, cmax=200000):
    """Independent solves of the batch benchmark: P1 or P2 (seeded 50/50),
    cell counts log-uniform in [cmin, cmax] (unit square, n x n squares split
    in two), four-quadrant Riemann data with per-solve seeded states,
    transmissive boundaries."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        k = int(rng.integers(1, 3))
        cells = math.exp(rng.uniform(math.log(cmin), math.log(cmax)))
        side = max(4, int(round(math.sqrt(cells / 2.0))))
        out.append(riemann4_workload(n=side, k=k, seed=seed * 1000 + i))
    return out


def serving_requests(n=24, seed=11, rate=30.0, cmin=1000, cmax=100000, t_end=(0.005, 0.02)):
    """Seeded solve requests of the serving benchmark: Poisson arrivals at
    `rate` per second, cells log-uniform in [cmin, cmax], P1 or P2, initial data
    drawn from the isentropic vortex, the Sedov-type blast and the four-quadrant
    Riemann problem, end time uniform in t_end.  Returns (workload, t_end,
    arrival offset in s) triples."""
    rng = np.random.default_rng(seed)
    out, at = [], 0.0
    for i in range(n):
        at += rng.exponential(1.0 / rate)
        k = int(rng.integers(1, 3))
        cells = math.exp(rng.uniform(math.log(cmin), math.log(cmax)))
        side = max(4, int(round(math.sqrt(cells / 2.0))))
        kind = int(rng.integers(0, 3))
        if kind == 0:
            wl = vortex_workload(n=side, k=k, seed=seed * 100 + i)
        elif kind == 1:
            wl = sedov_workload(n=side + (side % 2), k=k, seed=seed * 100 + i)
        else:
            wl = riemann4_workload(n=side, k=k, seed=seed * 100 + i)
        out.append((wl, float(rng.uniform(*t_end)), at))
    return out

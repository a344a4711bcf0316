"""Independent test-side utilities: exact integration on triangles and
segments by collapsed Gauss-Legendre rules, random physical polynomials and
small meshes.  Nothing here restates the DG method."""
from __future__ import annotations

import math

import numpy as np

_GL = {n: np.polynomial.legendre.leggauss(n) for n in (4, 6, 8, 10)}


def tri_integral(f, V, n=8):
    """Integral of f(x, y) over the triangle with vertices V[3, 2] (Duffy map)."""
    x, w = _GL[n]
    s = 0.5 * (x + 1.0)
    ws = 0.5 * w
    S, T = np.meshgrid(s, s, indexing="ij")
    WS, WT = np.meshgrid(ws, ws, indexing="ij")
    xi = S * (1.0 - T)
    eta = S * T
    jac = S * WS * WT
    V = np.asarray(V, dtype=np.float64)
    X = V[0, 0] + (V[1, 0] - V[0, 0]) * xi + (V[2, 0] - V[0, 0]) * eta
    Y = V[0, 1] + (V[1, 1] - V[0, 1]) * xi + (V[2, 1] - V[0, 1]) * eta
    det = (V[1, 0] - V[0, 0]) * (V[2, 1] - V[0, 1]) - (V[2, 0] - V[0, 0]) * (V[1, 1] - V[0, 1])
    return float(np.sum(f(X, Y) * jac) * det)


def seg_integral(f, A, B, n=8):
    x, w = _GL[n]
    s = 0.5 * (x + 1.0)
    A = np.asarray(A, float)
    B = np.asarray(B, float)
    X = A[0] + (B[0] - A[0]) * s
    Y = A[1] + (B[1] - A[1]) * s
    L = math.hypot(B[0] - A[0], B[1] - A[1])
    return float(np.sum(f(X, Y) * 0.5 * w) * L)


class PhysPoly:
    """Polynomial sum c_ab x^a y^b of total degree <= k with its derivatives."""

    def __init__(self, coeffs):
        self.c = dict(coeffs)

    @classmethod
    def random(cls, k, rng, scale=1.0):
        return cls({(a, b): scale * rng.uniform(-1, 1) for a in range(k + 1) for b in range(k + 1 - a)})

    def __call__(self, x, y):
        x = np.asarray(x, float)
        y = np.asarray(y, float)
        return sum(c * x ** a * y ** b for (a, b), c in self.c.items()) + 0.0 * x

    def d(self, dx, dy):
        out = {}
        for (a, b), c in self.c.items():
            if a < dx or b < dy:
                continue
            f = c * math.factorial(a) / math.factorial(a - dx) * math.factorial(b) / math.factorial(b - dy)
            out[(a - dx, b - dy)] = out.get((a - dx, b - dy), 0.0) + f
        return PhysPoly(out)

    def scaled(self, s):
        return PhysPoly({key: s * v for key, v in self.c.items()})

    def __add__(self, o):
        out = dict(self.c)
        for key, v in o.c.items():
            out[key] = out.get(key, 0.0) + v
        return PhysPoly(out)


def single_cell(V, tag=1):
    V = np.asarray(V, dtype=np.float64)
    tri = np.array([[0, 1, 2]], dtype=np.int32)
    bc = np.full((1, 3), tag, dtype=np.int8)
    return V, tri, bc


def random_triangle(rng):
    while True:
        V = rng.uniform(-1, 1, (3, 2))
        det = (V[1, 0] - V[0, 0]) * (V[2, 1] - V[0, 1]) - (V[2, 0] - V[0, 0]) * (V[1, 1] - V[0, 1])
        if abs(det) < 0.05:
            continue
        if det < 0:
            V = V[[0, 2, 1]]
        return V


def rotate_mesh_state(mesh, u, phi):
    """Rotate coordinates counter-clockwise by phi; rotate momentum modes alike."""
    c, s = math.cos(phi), math.sin(phi)
    xy = mesh.xy @ np.array([[c, s], [-s, c]])
    ur = u.copy()
    ur[1] = c * u[1] - s * u[2]
    ur[2] = s * u[1] + c * u[2]
    return xy, ur


def rel_err(a, b):
    """Largest error of a against the oracle result b, relative to the largest
    oracle magnitude of each conserved quantity: density, energy, and the
    momentum vector, whose two components share one scale (the scheme is
    rotation invariant, so a flow along x must not be judged by the round-off
    of its tiny y-momentum alone)."""
    import numpy as np
    mag = np.abs(b).reshape(4, -1).max(1)
    mag[1] = mag[2] = max(mag[1], mag[2])
    scale = np.maximum(mag, 1e-300)
    return float((np.abs(a - b).reshape(4, -1).max(1) / scale).max())

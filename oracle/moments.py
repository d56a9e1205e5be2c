"""Exact RWG and pulse moments (oracle; test infrastructure only).

Eq. TAfactor and Sec. VI-A: for a basis function associated with leaf box b,
    m_{d,n}[i] = int f_{n,d}(x) l_{i,b}(x) dS     (d = 1..3, RWG)
    m^phi_c[i] = int_c (1/a_c) l_{i,b}(x) dS     (pulse)
with l_{i,b} the tensor-product B-splines of the box's extended equidistant
knot vector (Sec. III-B).  The paper says only "numerical quadrature"; we
integrate exactly (the paper only says numerical quadrature): each triangle is split by every interior knot
plane into convex pieces on which the integrand is a polynomial of degree
<= 3p+1, each piece is fanned into triangles and integrated with a collapsed
Gauss rule of that degree.
"""
from __future__ import annotations

import math

import numpy as np

from .bspline import basis, open_knots
from .geometry import RWGMesh
from .quadrature import map_rule


def split_polygon(poly, axis, value):
    """Split a convex polygon [k,3] by the plane x_axis = value."""
    sd = poly[:, axis] - value
    left, right = [], []
    k = len(poly)
    for i in range(k):
        a, b = poly[i], poly[(i + 1) % k]
        sa, sb = sd[i], sd[(i + 1) % k]
        if sa <= 0:
            left.append(a)
        if sa >= 0:
            right.append(a)
        if (sa < 0 < sb) or (sb < 0 < sa):
            t = sa / (sa - sb)
            x = a + t * (b - a)
            x[axis] = value
            left.append(x)
            right.append(x)
    out = []
    for P in (left, right):
        if len(P) >= 3:
            out.append(np.array(P))
    return out


def clip_triangle(tri, planes):
    """Convex pieces of a triangle cut by knot planes; planes = 3 arrays of
    interior knot positions per axis."""
    pieces = [np.asarray(tri, dtype=np.float64)]
    for axis in range(3):
        for v in planes[axis]:
            nxt = []
            for P in pieces:
                lo, hi = P[:, axis].min(), P[:, axis].max()
                if lo < v < hi:
                    nxt.extend(split_polygon(P, axis, v))
                else:
                    nxt.append(P)
            pieces = nxt
    tris = []
    for P in pieces:
        for i in range(1, len(P) - 1):
            t = np.stack([P[0], P[i], P[i + 1]])
            if np.linalg.norm(np.cross(t[1] - t[0], t[2] - t[0])) > 0:
                tris.append(t)
    return np.array(tris)


class LeafSplines:
    """Knot vectors of the extended equidistant splines of one leaf box."""

    def __init__(self, ext_lo, sp, p, delta):
        self.p = p
        self.knots = [open_knots(ext_lo[d], ext_lo[d] + (sp - p) * delta, sp, p) for d in range(3)]
        self.planes = [U[p + 1:len(U) - p - 1] for U in self.knots]

    def tensor(self, X, w, f):
        """sum_q w_q f_q l_i(x_q) as an [s',s',s'] tensor; f [Q] or [Q,k]."""
        B = [basis(self.knots[d], self.p, X[:, d]) for d in range(3)]
        n = B[0].shape[1]
        ab = (B[0][:, :, None] * B[1][:, None, :]).reshape(len(w), n * n)   # [Q, a*b]
        if f.ndim == 1:
            return ((ab * (w * f)[:, None]).T @ B[2]).reshape(n, n, n)
        return np.stack([((ab * (w * f[:, i])[:, None]).T @ B[2]).reshape(n, n, n)
                         for i in range(f.shape[1])])


def quad_order(p):
    # collapsed rule with n points is exact to total degree 2n - 2 >= 3p + 1
    return int(math.ceil((3 * p + 3) / 2.0))


def rwg_moments(mesh: RWGMesh, tree, subset=None):
    """[N, 3, s', s', s'] RWG moments in each RWG's leaf box (or only for the
    RWGs listed in subset, in that order)."""
    L = tree.levels[tree.D]
    p = tree.p
    n = quad_order(p)
    ids = np.arange(mesh.N) if subset is None else np.asarray(subset)
    out = np.zeros((len(ids), 3, L.sp, L.sp, L.sp))
    cache = {}
    for oi, m in enumerate(ids):
        b = tree.rwg_box[m]
        if b not in cache:
            cache[b] = LeafSplines(L.box_ext_lo(tree.root_lo, L.ijk[b]), L.sp, p, L.delta)
        spl = cache[b]
        for side in range(2):
            c = mesh.tri_pm[m, side]
            xv = mesh.V[mesh.free_pm[m, side]]
            sgn = 1.0 if side == 0 else -1.0
            pieces = clip_triangle(mesh.V[mesh.T[c]], spl.planes)
            X, w = map_rule(pieces, n)
            X = X.reshape(-1, 3)
            w = w.reshape(-1)
            f = sgn * (X - xv) / (2.0 * mesh.area[c])
            out[oi] += spl.tensor(X, w, f)
    return out


def pulse_moments(mesh: RWGMesh, tree, subset=None):
    """[Nt, s', s', s'] pulse moments in each triangle's leaf box (or only for
    the triangles listed in subset)."""
    L = tree.levels[tree.D]
    p = tree.p
    n = quad_order(p)
    ids = np.arange(mesh.Nt) if subset is None else np.asarray(subset)
    out = np.zeros((len(ids), L.sp, L.sp, L.sp))
    cache = {}
    for oi, c in enumerate(ids):
        b = tree.tri_box[c]
        if b not in cache:
            cache[b] = LeafSplines(L.box_ext_lo(tree.root_lo, L.ijk[b]), L.sp, p, L.delta)
        spl = cache[b]
        pieces = clip_triangle(mesh.V[mesh.T[c]], spl.planes)
        X, w = map_rule(pieces, n)
        X = X.reshape(-1, 3)
        w = w.reshape(-1)
        out[oi] = spl.tensor(X, w, np.full(len(w), 1.0 / mesh.area[c]))
    return out

"""Pins of the exact moments (oracle/moments.py) by the B-splines' own
identities, independent of the far pipeline: the splines of a box's
extended knot vector sum to one and reproduce linear functions through their
Greville abscissae (xi_i = mean of the p interior knots of spline i), and
their tensor products reproduce x_a x_b.  So, for a triangle c of area a and
an RWG f (Sec. II):

    sum_i m^phi_c[i]              = 1
    sum_i xi_a(i) m^phi_c[i]      = centroid_a
    sum_i xi_a(i) xi_b(j) m^phi_c = (1/a) int_c x_a x_b dS          (a != b)
    sum_i m_{d,n}[i]              = int f_{n,d} dS
    sum_i xi_a(i) m_{d,n}[i]      = int x_a f_{n,d} dS

The right-hand sides come from the edge-midpoint rule, exact for quadratics on
a triangle.  A missing clipped piece, a shifted knot vector or box, swapped
axes, a wrong sign on the minus triangle or a wrong area factor fails one."""
import numpy as np
import pytest

import efie_inputs as E
from oracle.bspline import open_knots
from oracle.geometry import build_rwg
from oracle.moments import pulse_moments, rwg_moments
from oracle.tree import build_tree


def _midpoint_rule(tri):
    """Points and weights of the edge-midpoint rule (exact to degree 2)."""
    a, b, c = tri
    area = 0.5 * np.linalg.norm(np.cross(b - a, c - a))
    return np.array([(a + b) / 2, (b + c) / 2, (c + a) / 2]), np.full(3, area / 3)


def _greville(tree, box):
    L = tree.levels[tree.D]
    lo = L.box_ext_lo(tree.root_lo, L.ijk[box])
    out = []
    for d in range(3):
        U = open_knots(lo[d], lo[d] + (L.sp - tree.p) * L.delta, L.sp, tree.p)
        out.append(np.array([U[i + 1:i + tree.p + 1].mean() for i in range(L.sp)]))
    return out


@pytest.fixture(scope="module", params=[2, 3, 5])
def setting(request):
    p = request.param
    V, T = E.icosphere(6, 0.35)
    m = build_rwg(V, T)
    tree = build_tree(m, 2 * np.pi, p, 0.07, 2)
    return m, tree


def test_pulse_moments_identities(setting):
    m, tree = setting
    ids = np.random.default_rng(1).choice(m.Nt, 40, replace=False)
    M = pulse_moments(m, tree, subset=ids)
    for mm, c in zip(M, ids):
        g = _greville(tree, tree.tri_box[c])
        X, w = _midpoint_rule(m.V[m.T[c]])
        assert abs(mm.sum() - 1.0) < 1e-13
        lin = [np.einsum("i,ijk->", g[0], mm), np.einsum("j,ijk->", g[1], mm), np.einsum("k,ijk->", g[2], mm)]
        assert np.allclose(lin, m.centroid[c], rtol=0, atol=1e-13)
        area = w.sum()
        for (a, b, sub) in ((0, 1, "i,j,ijk->"), (1, 2, "j,k,ijk->"), (0, 2, "i,k,ijk->")):
            want = np.sum(w * X[:, a] * X[:, b]) / area
            assert abs(np.einsum(sub, g[a], g[b], mm) - want) < 1e-13


def test_rwg_moments_identities(setting):
    m, tree = setting
    ids = np.random.default_rng(2).choice(m.N, 40, replace=False)
    M = rwg_moments(m, tree, subset=ids)
    for mm, n in zip(M, ids):
        g = _greville(tree, tree.rwg_box[n])
        want0 = np.zeros(3)
        want1 = np.zeros((3, 3))     # [a][d] = int x_a f_d
        for side, sgn in ((0, 1.0), (1, -1.0)):
            c = m.tri_pm[n, side]
            X, w = _midpoint_rule(m.V[m.T[c]])
            f = sgn * (X - m.V[m.free_pm[n, side]]) / (2.0 * w.sum())
            want0 += w @ f
            want1 += np.einsum("q,qa,qd->ad", w, X, f)
        assert np.allclose(mm.sum(axis=(1, 2, 3)), want0, rtol=0, atol=1e-13)
        got1 = np.stack([np.einsum("i,dijk->d", g[0], mm), np.einsum("j,dijk->d", g[1], mm),
                         np.einsum("k,dijk->d", g[2], mm)])
        assert np.allclose(got1, want1, rtol=0, atol=1e-13)

"""B-spline algebra for the oracle (test infrastructure only).

* Open equidistant knot vectors (Eq. eqknots), extended by buffer knots
  (Sec. III-B).
* Cox-de Boor evaluation of all B-splines of a knot vector.
* Boehm knot insertion with the alpha_i weights of Sec. IV-B.
* Interlevel transfer matrices C (Sec. IV-B): row j = coefficients, in the
  child basis, of parent spline j restricted to the child's extended domain,
  obtained by inserting knots into the unit curve e_j.
* Knot-removal stabilization (Sec. V-B, Table I): the first and the last
  s_remove interior knots are removed (Table I's count read as per side);
  S maps equidistant to stabilized splines by knot insertion; interpolation
  points are s_hat equispaced points including both ends of the extended
  domain (equispaced, both ends included); P = B_stab^{-1} S, W_stab = P^T G P.

Knot positions are handled in integer lattice units (the finest spacing of the
pair of levels involved), so equality tests between knots are exact.
"""
from __future__ import annotations

import numpy as np

# Table I: recommended number of knots to remove, per polynomial degree p
S_REMOVE = {1: 0, 2: 0, 3: 1, 4: 1, 5: 2, 6: 2}


def open_knots(lo, hi, n_splines, p):
    """Open equidistant knot vector with n_splines B-splines of degree p on
    [lo, hi] (Eq. eqknots, scaled and shifted)."""
    m = n_splines - p
    if m < 1:
        raise ValueError("need n_splines > p")
    inner = [lo + (hi - lo) * i / m for i in range(1, m)]
    return np.array([lo] * (p + 1) + inner + [hi] * (p + 1), dtype=np.float64)


def basis(knots, p, x):
    """Values of all B-splines of degree p of the knot vector at points x.
    Returns [len(x), n_splines].  Spans are half-open [u_i, u_{i+1}) except the
    last non-empty span, which is closed (so x = right end is covered)."""
    U = np.asarray(knots, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    nk = len(U)
    ns = nk - p - 1
    last = np.max(np.nonzero(U[:-1] < U[1:])[0])
    N = np.zeros((len(x), nk - 1))
    for i in range(nk - 1):
        if U[i] < U[i + 1]:
            inside = (x >= U[i]) & (x < U[i + 1])
            if i == last:
                inside = (x >= U[i]) & (x <= U[i + 1])
            N[:, i] = inside
    for q in range(1, p + 1):
        Nn = np.zeros((len(x), nk - 1 - q))
        for i in range(nk - 1 - q):
            t = np.zeros(len(x))
            d1 = U[i + q] - U[i]
            if d1 > 0:
                t += (x - U[i]) / d1 * N[:, i]
            d2 = U[i + q + 1] - U[i + 1]
            if d2 > 0:
                t += (U[i + q + 1] - x) / d2 * N[:, i + 1]
            Nn[:, i] = t
        N = Nn
    assert N.shape[1] == ns
    return N


def insert_knot(knots, p, w, ubar):
    """Boehm insertion of ubar (Sec. IV-B): with u_k <= ubar < u_{k+1},
    w_bar_i = alpha_i w_i + (1 - alpha_i) w_{i-1},
    alpha_i = 1 (i <= k-p), (ubar - u_i)/(u_{i+p} - u_i) (k-p+1 <= i <= k),
    0 (i >= k+1).  Returns (new_knots, new_w)."""
    U = np.asarray(knots, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    if not (U[0] <= ubar < U[-1]):
        raise ValueError("knot outside the open interval of the knot vector")
    k = int(np.searchsorted(U, ubar, side="right") - 1)
    n = len(w)
    wb = np.zeros(n + 1)
    for i in range(n + 1):
        if i <= k - p:
            wb[i] = w[i]
        elif i >= k + 1:
            wb[i] = w[i - 1]
        else:
            alpha = (ubar - U[i]) / (U[i + p] - U[i])
            wb[i] = alpha * w[i] + (1.0 - alpha) * w[i - 1]
    Ub = np.concatenate([U[:k + 1], [ubar], U[k + 1:]])
    return Ub, wb


def refine_to(knots, p, w, target_knots):
    """Insert knots into (knots, w) until the knot multiset contains
    target_knots (a multiset)."""
    U = np.asarray(knots, dtype=np.float64)
    for t in np.unique(target_knots):
        need = int(np.sum(np.asarray(target_knots) == t)) - int(np.sum(U == t))
        for _ in range(max(need, 0)):
            U, w = insert_knot(U, p, w, float(t))
    return U, w


def restriction_matrix(parent_knots, child_knots, p):
    """C[j, i]: coefficient of child spline i in the restriction of parent
    spline j to the child domain [child_knots[0], child_knots[-1]] (Sec. IV-B).
    Knot vectors in integer lattice units; every interior child knot must be a
    lattice point and every parent knot inside the child domain a child knot."""
    Up = np.asarray(parent_knots, dtype=np.float64)
    Uc = np.asarray(child_knots, dtype=np.float64)
    a, b = Uc[0], Uc[-1]
    ns_p = len(Up) - p - 1
    ns_c = len(Uc) - p - 1
    # knots to have after refinement: the child's interior knots and p+1-fold
    # ends, plus every parent knot outside the child domain (kept as they are)
    target = [t for t in Up if t < a or t > b] + list(Uc)
    C = np.zeros((ns_p, ns_c))
    for j in range(ns_p):
        w = np.zeros(ns_p)
        w[j] = 1.0
        U, wr = refine_to(Up, p, w, target)
        k0 = int(np.searchsorted(U, a, side="left"))
        seg = U[k0:k0 + ns_c + p + 1]
        if not np.array_equal(seg, Uc):
            raise RuntimeError("child knot vector not nested in the refined parent")
        C[j] = wr[k0:k0 + ns_c]
    return C


def stabilized_knots(eq_knots, p, s_remove):
    """Remove the first and the last s_remove interior knots (Sec. V-B)."""
    U = np.asarray(eq_knots, dtype=np.float64)
    lo, hi = U[0], U[-1]
    inner = U[p + 1:len(U) - p - 1]
    if s_remove:
        inner = inner[s_remove:len(inner) - s_remove]
    return np.concatenate([[lo] * (p + 1), inner, [hi] * (p + 1)])


def stabilization_matrix(eq_knots, stab_knots, p):
    """S[j, i]: coefficient of equidistant spline i in stabilized spline j,
    by inserting the removed knots (Sec. V-B)."""
    Us = np.asarray(stab_knots, dtype=np.float64)
    Ue = np.asarray(eq_knots, dtype=np.float64)
    ns_s = len(Us) - p - 1
    ns_e = len(Ue) - p - 1
    S = np.zeros((ns_s, ns_e))
    for j in range(ns_s):
        w = np.zeros(ns_s)
        w[j] = 1.0
        U, wr = refine_to(Us, p, w, Ue)
        if not np.array_equal(U, Ue):
            raise RuntimeError("stabilized knots not contained in the equidistant knots")
        S[j] = wr
    return S


def interpolation_points(lo, hi, n_points):
    """n_points equispaced points including both ends (Eq. avgknots for p = 3)."""
    return lo + (hi - lo) * np.arange(n_points) / (n_points - 1)


def sampling_matrix(knots, p, points):
    """[B]_{m,n} = b_m(x_n) (Sec. III-A)."""
    return basis(knots, p, points).T


def projector(eq_knots, p, s_remove):
    """P = B_stab^{-1} S (s_hat x s'), the map from equidistant moments to
    transformed stabilized moments (Sec. III-C, Sec. V-B)."""
    Us = stabilized_knots(eq_knots, p, s_remove)
    S = stabilization_matrix(eq_knots, Us, p)
    ns_hat = len(Us) - p - 1
    x = interpolation_points(eq_knots[0], eq_knots[-1], ns_hat)
    B = sampling_matrix(Us, p, x)
    return np.linalg.solve(B, S), S, B, x


def averaged_knots(n_splines, p):
    """Averaged knot vector of Eq. avgknots on [0, 1]."""
    inner = [(2 * i - p - 3) / (2 * (n_splines - 1)) for i in range(p + 2, n_splines + 1)]
    return np.array([0.0] * (p + 1) + inner + [1.0] * (p + 1))

"""Quadrature for the oracle (test infrastructure only).

* Gauss-Legendre rules generated at run time by the Golub-Welsch eigenvalue
  method (no stored tables).
* Collapsed ("Duffy") tensor rules on the reference triangle
  {xi >= 0, eta >= 0, xi + eta <= 1}: (u, v) in [0,1]^2 -> (xi, eta) = (u, (1-u) v),
  Jacobian (1-u).  An n-point rule integrates total degree <= 2n-2 exactly.
* Analytic static potentials of a flat triangle, int 1/R dS' and
  int (r' - rho)/R dS' (Wilton et al. 1984; Graglia 1993), derived from the
  surface divergence/gradient theorems.
* A polar-coordinate brute-force integrator (the r-Jacobian cancels 1/R); it is
  independent of the analytic formulas and is used only to pin them.
"""
from __future__ import annotations

import functools

import numpy as np


@functools.lru_cache(maxsize=None)
def gauss_legendre01(n: int):
    """n-point Gauss-Legendre rule on [0,1] (Golub-Welsch)."""
    if n < 1:
        raise ValueError("n >= 1")
    k = np.arange(1, n)
    beta = k / np.sqrt(4.0 * k * k - 1.0)
    J = np.diag(beta, 1) + np.diag(beta, -1)
    x, vec = np.linalg.eigh(J)
    w = 2.0 * vec[0, :] ** 2
    return (x + 1.0) / 2.0, w / 2.0


@functools.lru_cache(maxsize=None)
def triangle_rule(n: int):
    """Collapsed n x n Gauss-Legendre rule on the reference triangle.
    Returns (xi [n*n], eta [n*n], w [n*n]) with sum(w) = 1/2."""
    u, wu = gauss_legendre01(n)
    U, Vv = np.meshgrid(u, u, indexing="ij")
    WU, WV = np.meshgrid(wu, wu, indexing="ij")
    xi = U
    eta = Vv * (1.0 - U)
    w = WU * WV * (1.0 - U)
    return xi.ravel(), eta.ravel(), w.ravel()


def map_rule(tri_xyz, n):
    """Physical points [..., Q, 3] and weights [..., Q] of the n-rule on triangles
    tri_xyz [..., 3, 3] (weights include the area Jacobian 2a)."""
    xi, eta, w = triangle_rule(n)
    v0 = tri_xyz[..., 0, :]
    e1 = tri_xyz[..., 1, :] - v0
    e2 = tri_xyz[..., 2, :] - v0
    pts = v0[..., None, :] + xi[:, None] * e1[..., None, :] + eta[:, None] * e2[..., None, :]
    twoa = np.linalg.norm(np.cross(e1, e2), axis=-1)
    return pts, twoa[..., None] * w


def _safe_log_ratio(Rp, lp, Rm, lm, R0sq):
    """ln((R+ + l+)/(R- + l-)) evaluated without cancellation (R +/- l with l < 0
    is rewritten as R0^2 / (R - l))."""
    num = np.where(lp >= 0, Rp + lp, R0sq / np.maximum(Rp - lp, 1e-300))
    den = np.where(lm >= 0, Rm + lm, R0sq / np.maximum(Rm - lm, 1e-300))
    with np.errstate(divide="ignore", invalid="ignore"):
        out = np.log(num / den)
    return np.where((num > 0) & (den > 0), out, 0.0)


def static_potentials(r, tri):
    """Analytic static integrals over flat triangles for observation points:
        I1 = int_T 1/|r - r'| dS'          [..., Q]
        Iv = int_T (r' - rho)/|r - r'| dS' [..., Q, 3]
    r [..., Q, 3], tri [..., 3, 3] (leading dims broadcast); rho is the
    projection of r onto the triangle's plane.

    Derivation: with rho, the signed height d and the edge frames
    (l_hat along edge i, u_hat = l_hat x n_hat its outward in-plane normal),
      grad'_s R = (r' - rho)/R        -> Iv = sum_i u_hat_i int_edge R dl,
      div'_s[(r'-rho)(R-|d|)/|r'-rho|^2] = 1/R
                                       -> I1 = sum_i P0_i int_edge (R-|d|)/(t^2+P0_i^2) dt,
    both line integrals in closed form."""
    r = np.asarray(r, dtype=np.float64)
    v = np.asarray(tri, dtype=np.float64)
    if r.ndim == 1:
        r = r[None, :]
    n = np.cross(v[..., 1, :] - v[..., 0, :], v[..., 2, :] - v[..., 0, :])
    n = n / np.linalg.norm(n, axis=-1, keepdims=True)
    n_ = n[..., None, :]                                   # [...,1,3]
    d = np.sum((r - v[..., 0:1, :]) * n_, axis=-1)         # [...,Q]
    rho = r - d[..., None] * n_
    ad = np.abs(d)
    I1 = np.zeros(r.shape[:-1])
    Iv = np.zeros(r.shape)
    for i in range(3):
        a = v[..., i:i + 1, :]
        b = v[..., (i + 1) % 3:(i + 1) % 3 + 1, :]
        L = b - a
        lh = L / np.linalg.norm(L, axis=-1, keepdims=True)
        uh = np.cross(lh, n_)
        lm = np.sum((a - rho) * lh, axis=-1)
        lp = np.sum((b - rho) * lh, axis=-1)
        P0 = np.sum((a - rho) * uh, axis=-1)
        R0sq = P0 * P0 + d * d
        Rm = np.linalg.norm(r - a, axis=-1)
        Rp = np.linalg.norm(r - b, axis=-1)
        lg = _safe_log_ratio(Rp, lp, Rm, lm, R0sq)
        Iv = Iv + 0.5 * (R0sq * lg + lp * Rp - lm * Rm)[..., None] * uh
        with np.errstate(divide="ignore", invalid="ignore"):
            at = (np.arctan2(P0 * lp, R0sq + ad * Rp) - np.arctan2(P0 * lm, R0sq + ad * Rm))
        term = P0 * lg - ad * at
        I1 = I1 + np.where(np.abs(P0) > 1e-300, term, 0.0)
    return I1, Iv


def polar_integrate(r, tri, func, n_theta=24, n_rho=24, subdiv=1):
    """Brute-force int_T func(r', |r - r'|) dS' by polar coordinates around the
    projection rho of r onto the plane of T.  The triangle is written as a signed
    sum of the three triangles (rho, v_i, v_{i+1}); in each, theta runs between
    the two vertex directions and t in [0, t_max(theta)], dS' = t dt dtheta, so a
    1/R singularity at rho is cancelled by the Jacobian.  func(x [Q,3], R [Q])
    returns values [Q] or [Q,k].  Used only as an independent pin."""
    r = np.asarray(r, dtype=np.float64)
    v = np.asarray(tri, dtype=np.float64)
    n = np.cross(v[1] - v[0], v[2] - v[0])
    n = n / np.linalg.norm(n)
    d = (r - v[0]) @ n
    rho = r - d * n
    gt, wt = gauss_legendre01(n_theta)
    gr, wr = gauss_legendre01(n_rho)
    total = None
    for i in range(3):
        a = v[i] - rho
        b = v[(i + 1) % 3] - rho
        la, lb = np.linalg.norm(a), np.linalg.norm(b)
        if la < 1e-300 or lb < 1e-300:
            continue
        ea = a / la
        eb_perp = b - (b @ ea) * ea
        nb = np.linalg.norm(eb_perp)
        if nb < 1e-300:
            continue  # rho on the edge line: zero-area sub-triangle
        sign = np.sign(np.cross(a, b) @ n)
        ey = eb_perp / nb
        th_b = np.arctan2(b @ ey, b @ ea)     # in (0, pi)
        # edge line from a to b in the local (ea, ey) frame
        ab = b - a
        # distance from origin to the edge line
        nrm = np.cross(ab, n)
        nrm = nrm / np.linalg.norm(nrm)
        p0 = abs(a @ nrm)
        th0 = np.arctan2(nrm @ ey, nrm @ ea)
        if (a @ nrm) < 0:
            th0 = np.arctan2(-(nrm @ ey), -(nrm @ ea))
        for s in range(subdiv):
            t_lo = th_b * s / subdiv
            t_hi = th_b * (s + 1) / subdiv
            th = t_lo + (t_hi - t_lo) * gt
            wth = (t_hi - t_lo) * wt
            tmax = p0 / np.cos(th - th0)
            # points
            T_ = tmax[:, None] * gr[None, :]
            W_ = (wth[:, None] * tmax[:, None] * wr[None, :]) * T_
            dirs = np.cos(th)[:, None] * ea[None, :] + np.sin(th)[:, None] * ey[None, :]
            X = rho[None, None, :] + T_[:, :, None] * dirs[:, None, :]
            R = np.sqrt(T_ * T_ + d * d)
            val = func(X.reshape(-1, 3), R.reshape(-1))
            val = np.asarray(val)
            if val.ndim == 1:
                contrib = sign * np.sum(W_.reshape(-1) * val)
            else:
                contrib = sign * np.sum(W_.reshape(-1)[:, None] * val, axis=0)
            total = contrib if total is None else total + contrib
    return total

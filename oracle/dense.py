"""Dense Galerkin RWG EFIE (oracle; test infrastructure only).

Sec. II (Eq. discretizedEFIE, Eq. matTA, Eq. matTPhi) with the star form of
Sec. VI-A.  With div f_m = sum_c Sigma[m,c] phi_c and phi_c = 1/a_c:

    A[m,n] = int int f_m(x) . f_n(y) g(x,y)
    V[c,c'] = int int phi_c(x) g(x,y) phi_c'(y) = (1/(a_c a_c')) int_c int_c' g
    T = jk A + (jk)^-1 Sigma V Sigma^T                       (sign fixed by the Mie series; Eq. matTPhi's minus is absorbed)

e^{j w t} convention, g = exp(-jkR)/(4 pi R).  The paper writes the scalar part
as -(jk)^-1 T_Phi with a leading minus inside Eq. matTPhi and later
T_Phi = Sigma V Sigma^T; the two cannot both hold.  We take the physical EFIE
(-E^s_tan = E^i_tan), which gives +(jk)^-1 Sigma V Sigma^T; the Mie series pins
the sign.

Triangle-pair quadrature (the same rule is used by the library's near field):
  * close pair (|cen_c - cen_c'|^2 < 4 max(emax_c, emax_c')^2): outer n_out x
    n_out collapsed Gauss rule on c; inner = analytic static part 1/(4 pi R)
    plus the smooth remainder (exp(-jkR)-1)/(4 pi R) on the n_in rule of c';
    the result is the mean of this rule and the same rule with the roles of c
    and c' swapped (symmetrized, so A = A^T and V = V^T exactly);
  * regular pair: n_reg rule on both triangles.
Defaults n_reg = 3, n_out = 4, n_in = 4.
"""
from __future__ import annotations

import numpy as np

from .geometry import RWGMesh
from .quadrature import map_rule, static_potentials, triangle_rule

FOUR_PI = 4.0 * np.pi
N_REG, N_OUT, N_IN = 3, 4, 4


def green(R, k):
    return np.exp(-1j * k * R) / (FOUR_PI * R)


def smooth_remainder(R, k):
    """(exp(-jkR) - 1)/(4 pi R), with its limit -jk/(4 pi) at R = 0; the real
    part is written as -2 sin^2(kR/2)/R to avoid cancellation."""
    R = np.asarray(R, dtype=np.float64)
    pos = R > 0
    Rs = np.where(pos, R, 1.0)
    s_half = np.sin(0.5 * k * Rs)
    val = (-2.0 * s_half * s_half - 1j * np.sin(k * Rs)) / Rs
    return np.where(pos, val, -1j * k) / FOUR_PI


def tri_vertices(mesh: RWGMesh, c):
    return mesh.V[mesh.T[np.asarray(c)]]          # [..., 3, 3]


def max_edge_sq(mesh: RWGMesh):
    v = mesh.V[mesh.T]
    e0 = np.sum((v[:, 1] - v[:, 0]) ** 2, axis=1)
    e1 = np.sum((v[:, 2] - v[:, 1]) ** 2, axis=1)
    e2 = np.sum((v[:, 0] - v[:, 2]) ** 2, axis=1)
    return np.maximum(np.maximum(e0, e1), e2)


def close_mask(mesh: RWGMesh, c, cp):
    emax2 = max_edge_sq(mesh)
    dc = mesh.centroid[c] - mesh.centroid[cp]
    d2 = np.sum(dc * dc, axis=-1)
    return d2 < 4.0 * np.maximum(emax2[c], emax2[cp])


def _regular(mesh, c, cp, k, n, kernel):
    """Regular tensor rule for pairs (c [P], cp [P]).  Returns I0 [P], Ivv [P,3,3]."""
    X, wx = map_rule(tri_vertices(mesh, c), n)    # [P,Q,3], [P,Q]
    Y, wy = map_rule(tri_vertices(mesh, cp), n)
    Vc = tri_vertices(mesh, c)                    # [P,3,3]
    Vp = tri_vertices(mesh, cp)
    D = X[:, :, None, :] - Y[:, None, :, :]       # [P,Q,Q,3]
    if kernel is None:
        R = np.sqrt(np.sum(D * D, axis=-1))
        G = green(R, k)
    else:
        G = kernel(D)
    W = wx[:, :, None] * wy[:, None, :] * G       # [P,Q,Q]
    I0 = W.sum(axis=(1, 2))
    # (x - v_i).(y - v'_j) = x.y - v_i.y - x.v'_j + v_i.v'_j
    Sx = np.einsum("pab,pad->pbd", W, X)          # sum_x,y W x  -> [P,Q(y),3]
    Sxy = np.einsum("pbd,pbd->p", Sx, Y)          # int x.y g
    Ix = Sx.sum(axis=1)                           # int x g   [P,3]
    Iy = np.einsum("pab,pbd->pd", W, Y)           # int y g   [P,3]
    Ivv = (Sxy[:, None, None]
           - np.einsum("pid,pd->pi", Vc, Iy)[:, :, None]
           - np.einsum("pjd,pd->pj", Vp, Ix)[:, None, :]
           + np.einsum("pid,pjd->pij", Vc, Vp) * I0[:, None, None])
    return I0, Ivv


def _close_oriented(mesh, c, cp, k, n_out, n_in):
    """One orientation of the singular rule: outer rule on c, inner analytic
    static part + smooth remainder on c'.  Vectorized over pairs."""
    Vc = tri_vertices(mesh, c)                     # [P,3,3]
    Vp = tri_vertices(mesh, cp)
    X, wx = map_rule(Vc, n_out)                    # [P,Qx,3]
    Y, wy = map_rule(Vp, n_in)                     # [P,Qy,3]
    n_hat = np.cross(Vp[:, 1] - Vp[:, 0], Vp[:, 2] - Vp[:, 0])
    n_hat = n_hat / np.linalg.norm(n_hat, axis=1, keepdims=True)
    dh = np.einsum("pqd,pd->pq", X - Vp[:, None, 0, :], n_hat)
    rho = X - dh[..., None] * n_hat[:, None, :]
    I1, Iv = static_potentials(X, Vp)              # [P,Qx], [P,Qx,3]
    D = X[:, :, None, :] - Y[:, None, :, :]
    R = np.sqrt(np.sum(D * D, axis=-1))            # [P,Qx,Qy]
    Gs = smooth_remainder(R, k) * wy[:, None, :]
    in0 = I1 / FOUR_PI + Gs.sum(axis=2)                                   # [P,Qx]
    in_y = (Iv + rho * I1[..., None]) / FOUR_PI + np.einsum("pab,pbd->pad", Gs, Y)
    I0 = np.sum(wx * in0, axis=1)
    # Ivv[i,j] = int_c (x - v_i) . (in_y - v'_j in0)
    xv = X[:, None, :, :] - Vc[:, :, None, :]                             # [P,3,Qx,3]
    inner = in_y[:, None, :, :] - Vp[:, :, None, :] * in0[:, None, :, None]  # [P,3,Qx,3]
    Ivv = np.einsum("pq,piqd,pjqd->pij", wx, xv, inner)
    return I0, Ivv


def _close(mesh, c, cp, k, n_out, n_in, chunk=2048):
    """Symmetrized singular rule: the mean of the two orientations, so that the
    Galerkin matrices are exactly symmetric."""
    P = len(c)
    I0 = np.zeros(P, dtype=np.complex128)
    Ivv = np.zeros((P, 3, 3), dtype=np.complex128)
    for s in range(0, P, chunk):
        sl = slice(s, s + chunk)
        a0, av = _close_oriented(mesh, c[sl], cp[sl], k, n_out, n_in)
        b0, bv = _close_oriented(mesh, cp[sl], c[sl], k, n_out, n_in)
        I0[sl] = 0.5 * (a0 + b0)
        Ivv[sl] = 0.5 * (av + np.transpose(bv, (0, 2, 1)))
    return I0, Ivv


def pair_integrals(mesh: RWGMesh, c, cp, k, kernel=None, n_reg=N_REG, n_out=N_OUT,
                   n_in=N_IN, chunk=4096):
    """I0[p] = int_c int_c' g, Ivv[p,i,j] = int_c int_c' (x - v_i).(y - v'_j) g for
    triangle pairs (c[p], cp[p]); v_i are the vertices of c in mesh order.
    With kernel(D [...,3]) given, a regular rule with that translation-invariant
    kernel is used for every pair (no singularity extraction)."""
    c = np.asarray(c, dtype=np.int64)
    cp = np.asarray(cp, dtype=np.int64)
    P = len(c)
    I0 = np.zeros(P, dtype=np.complex128)
    Ivv = np.zeros((P, 3, 3), dtype=np.complex128)
    if kernel is None:
        close = close_mask(mesh, c, cp)
    else:
        close = np.zeros(P, dtype=bool)
    reg_idx = np.nonzero(~close)[0]
    for s in range(0, len(reg_idx), chunk):
        idx = reg_idx[s:s + chunk]
        I0[idx], Ivv[idx] = _regular(mesh, c[idx], cp[idx], k, n_reg, kernel)
    cl_idx = np.nonzero(close)[0]
    if len(cl_idx):
        I0[cl_idx], Ivv[cl_idx] = _close(mesh, c[cl_idx], cp[cl_idx], k, n_out, n_in)
    return I0, Ivv


def rwg_sides(mesh: RWGMesh):
    """Per RWG and side s in {+,-}: triangle id [N,2], local vertex index of the
    free vertex in that triangle [N,2], and coefficient sigma/(2a) [N,2]."""
    tri = mesh.tri_pm
    loc = np.zeros_like(tri)
    coef = np.zeros(tri.shape)
    for s in range(2):
        t = tri[:, s]
        fv = mesh.free_pm[:, s]
        loc[:, s] = np.argmax(mesh.T[t] == fv[:, None], axis=1)
        coef[:, s] = (1.0 if s == 0 else -1.0) / (2.0 * mesh.area[t])
    return tri, loc, coef


def assemble_dense(mesh: RWGMesh, k, kernel=None, **quad):
    """Dense A [N,N] and V [Nt,Nt] (Eq. matTA; Sec. VI-A)."""
    Nt = mesh.Nt
    cc, cpp = np.meshgrid(np.arange(Nt), np.arange(Nt), indexing="ij")
    I0, Ivv = pair_integrals(mesh, cc.ravel(), cpp.ravel(), k, kernel=kernel, **quad)
    I0 = I0.reshape(Nt, Nt)
    Ivv = Ivv.reshape(Nt, Nt, 3, 3)
    V = I0 / (mesh.area[:, None] * mesh.area[None, :])
    tri, loc, coef = rwg_sides(mesh)
    N = mesh.N
    A = np.zeros((N, N), dtype=np.complex128)
    for s in range(2):
        for sp in range(2):
            blk = Ivv[tri[:, s][:, None], tri[:, sp][None, :], loc[:, s][:, None], loc[:, sp][None, :]]
            A += coef[:, s][:, None] * coef[:, sp][None, :] * blk
    return A, V


def efie_matrix(mesh: RWGMesh, k, A=None, V=None, **quad):
    """T = jk A + (jk)^-1 Sigma V Sigma^T (the physical sign, pinned by the Mie series)."""
    if A is None or V is None:
        A, V = assemble_dense(mesh, k, **quad)
    S = mesh.sigma_dense()
    return 1j * k * A + (1.0 / (1j * k)) * (S @ V @ S.T)


def rows_dense(mesh: RWGMesh, k, rows, x, kernel=None, **quad):
    """(T x)[rows] without forming T: exact rows for a subset of test functions.
    Returns (yA, yV) with y = jk yA + (jk)^-1 yV, x [N] or [R,N]."""
    rows = np.asarray(rows, dtype=np.int64)
    x = np.atleast_2d(np.asarray(x, dtype=np.complex128))
    tri, loc, coef = rwg_sides(mesh)
    Nt = mesh.Nt
    rho = mesh.sigmaT_apply(x)                     # [R,Nt]
    test_tris = np.unique(tri[rows].ravel())
    cc, cpp = np.meshgrid(test_tris, np.arange(Nt), indexing="ij")
    I0, Ivv = pair_integrals(mesh, cc.ravel(), cpp.ravel(), k, kernel=kernel, **quad)
    I0 = I0.reshape(len(test_tris), Nt)
    Ivv = Ivv.reshape(len(test_tris), Nt, 3, 3)
    pos = {int(t): i for i, t in enumerate(test_tris)}
    # source side: per triangle c' and local vertex j, the accumulated coefficient
    src = np.zeros((x.shape[0], Nt, 3), dtype=np.complex128)
    for sp in range(2):
        for r in range(x.shape[0]):
            np.add.at(src[r], (tri[:, sp], loc[:, sp]), coef[:, sp] * x[r])
    yA = np.zeros((x.shape[0], len(rows)), dtype=np.complex128)
    yV = np.zeros((x.shape[0], len(rows)), dtype=np.complex128)
    for ri, m in enumerate(rows):
        for s in range(2):
            t = pos[int(tri[m, s])]
            # sum_{c',j} Ivv[t, c', loc, j] src[c', j]
            yA[:, ri] += coef[m, s] * np.einsum("cj,rcj->r", Ivv[t, :, loc[m, s], :], src)
            sgn = 1.0 if s == 0 else -1.0
            yV[:, ri] += sgn * (I0[t] / (mesh.area[tri[m, s]] * mesh.area)) @ rho.T
    return yA, yV


def rhs_planewave(mesh: RWGMesh, k, khat, pol, n=6):
    """[e^i]_m = int f_m . p_hat exp(-jk khat.x) dS (Sec. II), degree-(2n-2) rule."""
    khat = np.atleast_2d(np.asarray(khat, dtype=np.float64))
    pol = np.atleast_2d(np.asarray(pol, dtype=np.float64))
    X, w = map_rule(tri_vertices(mesh, np.arange(mesh.Nt)), n)   # [Nt,Q,3]
    tri, loc, coef = rwg_sides(mesh)
    out = np.zeros((khat.shape[0], mesh.N), dtype=np.complex128)
    for r in range(khat.shape[0]):
        ph = np.exp(-1j * k * (X @ khat[r]))                      # [Nt,Q]
        F0 = np.einsum("tq,tq->t", w, ph)                         # int e
        F1 = np.einsum("tq,tqd->td", w * ph, X)                   # int x e
        for s in range(2):
            t = tri[:, s]
            fv = mesh.V[mesh.free_pm[:, s]]
            out[r] += coef[:, s] * ((F1[t] - fv * F0[t][:, None]) @ pol[r])
    return out

"""Straightforward multilevel B-spline fast EFIE matvec (oracle; test
infrastructure only).  FP64 throughout; translations either by the plain
Toeplitz definition (dense G per box pair) or by NumPy FFTs of size
n = 2 s_hat - 1 (any n >= 2 s_hat - 1 gives the same result up to rounding,
the paper does not fix n).

Steps, in the paper's order:
  1. rho = Sigma^T j                                         (Sec. VI-A)
  2. leaf anterpolation q_{d,b} = sum_{n in b} j_n m_{d,n},
     q_{4,b} = sum_{c in b} rho_c m^phi_c                    (Eq. TAfactor, Sec. VI-A)
  3. upward q_P += (C^{c1} x C^{c2} x C^{c3}) q_c            (Eq. interleveltransfer, Sec. IV-B)
  4. q~ = P^{x3} q, P = B_stab^{-1} S                        (Sec. III-C, Sec. V-B)
  5. r~_x = sum_{y in IL(x)} G_xy q~_y, G_xy[a,b] = g(pt_x[a], pt_y[b])
     (3-level Toeplitz, FFT-accelerated; Eq. TAfactorBspline), r_x = (P^T)^{x3} r~_x
  6. downward r_c += (C^{c1} x C^{c2} x C^{c3})^T r_P
  7. y_m = jk sum_d m_{d,m}.r_{d,b(m)} + (jk)^-1 sum_c Sigma[m,c] m^phi_c.r_{4,b(c)}
  8. y += jk A_near j + (jk)^-1 Sigma V_near Sigma^T j       (Sec. VI-A)
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import dense
from .bspline import S_REMOVE, open_knots, projector, restriction_matrix
from .geometry import RWGMesh
from .moments import pulse_moments, rwg_moments
from .tree import build_tree, interaction_lists, near_box_pairs


def mode3(M1, M2, M3, T):
    """(M1 x M2 x M3) applied to the last three axes of T."""
    T = np.tensordot(T, M1, axes=([-3], [1]))       # [..., b, c, a']
    T = np.tensordot(T, M2, axes=([-3], [1]))       # [..., c, a', b']
    T = np.tensordot(T, M3, axes=([-3], [1]))       # [..., a', b', c']
    return T


class BsplineEFIE:
    def __init__(self, mesh: RWGMesh, k, p, grid_spacing, levels, n_splines=None,
                 kernel=None, near="auto", dense_AV=None, translation="fft",
                 allow_overlap=False):
        """kernel: optional translation-invariant kernel kappa(D [...,3]) that
        replaces g everywhere (used by the polynomial exactness pin).
        near: "auto" computes A_near/V_near with the dense quadrature rule,
        None leaves the near field out (far part only).
        dense_AV: optional (A, V) dense matrices to take the near entries from.
        allow_overlap: skip the far-domain separation check (only meaningful for
        a non-singular test kernel)."""
        self.mesh = mesh
        self.k = k
        self.p = p
        self.kernel = kernel
        self.translation = translation
        self.tree = tree = build_tree(mesh, k, p, grid_spacing, levels, n_splines, allow_overlap)
        D, top = tree.D, tree.top
        self.grid_levels = list(range(D, top - 1, -1))

        # interlevel transfers C^L, C^R (child level ell -> parent ell-1)
        self.CL, self.CR = {}, {}
        for ell in range(D, top, -1):
            c, pa = tree.levels[ell], tree.levels[ell - 1]
            r = int(round(pa.delta / c.delta))
            Up = open_knots(-pa.sb * r, (pa.s - p + pa.sb) * r, pa.sp, p)
            UcL = open_knots(-c.sb, (c.s - p) + c.sb, c.sp, p)
            UcR = open_knots((c.s - p) - c.sb, 2 * (c.s - p) + c.sb, c.sp, p)
            self.CL[ell] = restriction_matrix(Up, UcL, p)
            self.CR[ell] = restriction_matrix(Up, UcR, p)

        # projectors P = B_stab^{-1} S per level
        self.P = {}
        for ell in self.grid_levels:
            L = tree.levels[ell]
            Ue = open_knots(0.0, float(L.sp - p), L.sp, p)
            self.P[ell] = projector(Ue, p, S_REMOVE[p])[0]

        self.m_rwg = rwg_moments(mesh, tree)       # [N,3,s',s',s']
        self.m_tri = pulse_moments(mesh, tree)     # [Nt,s',s',s']

        self.IL = {ell: interaction_lists(tree, ell) for ell in self.grid_levels}

        if near is None:
            self.A_near = sp.csr_matrix((mesh.N, mesh.N), dtype=np.complex128)
            self.V_near = sp.csr_matrix((mesh.Nt, mesh.Nt), dtype=np.complex128)
        else:
            self.A_near, self.V_near = self._near(dense_AV)

    # ---------------------------------------------------------------- near
    def near_masks(self):
        nb = near_box_pairs(self.tree)
        rb, tb = self.tree.rwg_box, self.tree.tri_box
        return nb, rb, tb

    def _near(self, dense_AV):
        mesh = self.mesh
        nb, rb, tb = self.near_masks()
        if dense_AV is not None:
            A, V = dense_AV
            mA = nb[rb[:, None], rb[None, :]]
            mV = nb[tb[:, None], tb[None, :]]
            return sp.csr_matrix(np.where(mA, A, 0)), sp.csr_matrix(np.where(mV, V, 0))
        # V: triangle pairs in adjacent boxes
        ci, cj = np.nonzero(nb[tb[:, None], tb[None, :]])
        I0, _ = dense.pair_integrals(mesh, ci, cj, self.k, kernel=self.kernel)
        V = sp.csr_matrix((I0 / (mesh.area[ci] * mesh.area[cj]), (ci, cj)), shape=(mesh.Nt, mesh.Nt))
        # A: RWG pairs in adjacent boxes, from their triangle-pair integrals
        mi, mj = np.nonzero(nb[rb[:, None], rb[None, :]])
        tri, loc, coef = dense.rwg_sides(mesh)
        pairs = np.unique(np.concatenate([np.stack([tri[mi, s], tri[mj, t]], 1)
                                          for s in range(2) for t in range(2)]), axis=0)
        _, Ivv = dense.pair_integrals(mesh, pairs[:, 0], pairs[:, 1], self.k, kernel=self.kernel)
        key = pairs[:, 0] * mesh.Nt + pairs[:, 1]
        order = np.argsort(key)
        key_s = key[order]
        vals = np.zeros(len(mi), dtype=np.complex128)
        for s in range(2):
            for t in range(2):
                kk = tri[mi, s] * mesh.Nt + tri[mj, t]
                pos = order[np.searchsorted(key_s, kk)]
                vals += coef[mi, s] * coef[mj, t] * Ivv[pos, loc[mi, s], loc[mj, t]]
        A = sp.csr_matrix((vals, (mi, mj)), shape=(mesh.N, mesh.N))
        return A, V

    # ---------------------------------------------------------------- far
    def _kernel_fn(self, D):
        if self.kernel is not None:
            return self.kernel(D)
        R = np.sqrt(np.sum(D * D, axis=-1))
        return dense.green(R, self.k)

    def _translate_level(self, ell, qt):
        """r~_x = sum_{y in IL(x)} G_xy q~_y for all boxes; qt [B,4,n,n,n]."""
        L = self.tree.levels[ell]
        ns = L.shat
        xs, ys = self.IL[ell]
        out = np.zeros_like(qt)
        if len(xs) == 0:
            return out
        offs = L.ijk[xs] - L.ijk[ys]
        uo, inv = np.unique(offs, axis=0, return_inverse=True)
        inv = inv.reshape(-1)
        t = np.arange(-(ns - 1), ns)
        if self.translation == "fft":
            n = 2 * ns - 1
            Q = np.fft.fftn(np.pad(qt, [(0, 0), (0, 0)] + [(0, n - ns)] * 3), axes=(-3, -2, -1))
            R = np.zeros_like(Q)
            for oi, o in enumerate(uo):
                Dv = (o[None, None, None, :] * L.h
                      + np.stack(np.meshgrid(t, t, t, indexing="ij"), axis=-1) * L.Delta)
                Kt = self._kernel_fn(Dv)                              # [2ns-1]^3, index t+ns-1
                Kc = np.zeros((n, n, n), dtype=np.complex128)
                idx = np.mod(t, n)
                Kc[np.ix_(idx, idx, idx)] = Kt
                Kh = np.fft.fftn(Kc)
                sel = np.nonzero(inv == oi)[0]
                for pi in sel:
                    R[xs[pi]] += Kh[None] * Q[ys[pi]]
            r = np.fft.ifftn(R, axes=(-3, -2, -1))[..., :ns, :ns, :ns]
            return r
        # plain Toeplitz definition
        a = np.stack(np.meshgrid(np.arange(ns), np.arange(ns), np.arange(ns), indexing="ij"), -1).reshape(-1, 3)
        for oi, o in enumerate(uo):
            Dv = o[None, None, :] * L.h + (a[:, None, :] - a[None, :, :]) * L.Delta
            G = self._kernel_fn(Dv)                                   # [ns^3, ns^3]
            sel = np.nonzero(inv == oi)[0]
            for pi in sel:
                x, y = xs[pi], ys[pi]
                out[x] += (G @ qt[y].reshape(4, -1).T).T.reshape(4, ns, ns, ns)
        return out

    def far_grids(self, j):
        """Leaf far-field output grids r [B_D,4,s',s',s'] for one current vector."""
        tree, mesh = self.tree, self.mesh
        D = tree.D
        rho = mesh.sigmaT_apply(j)
        LD = tree.levels[D]
        q = {D: np.zeros((len(LD.boxes), 4, LD.sp, LD.sp, LD.sp), dtype=np.complex128)}
        np.add.at(q[D], (tree.rwg_box, slice(0, 3)), j[:, None, None, None, None] * self.m_rwg)
        np.add.at(q[D], (tree.tri_box, 3), rho[:, None, None, None] * self.m_tri)
        for ell in range(D, tree.top, -1):
            pa = tree.levels[ell - 1]
            qp = np.zeros((len(pa.boxes), 4, pa.sp, pa.sp, pa.sp), dtype=np.complex128)
            ijk = tree.levels[ell].ijk
            for b in range(len(ijk)):
                bits = ijk[b] % 2
                M = [self.CR[ell] if bb else self.CL[ell] for bb in bits]
                qp[tree.parent[ell][b]] += mode3(M[0], M[1], M[2], q[ell][b])
            q[ell - 1] = qp
        r = {}
        for ell in self.grid_levels:
            P = self.P[ell]
            qt = mode3(P, P, P, q[ell])
            rt = self._translate_level(ell, qt)
            r[ell] = mode3(P.T, P.T, P.T, rt)
        for ell in range(tree.top + 1, D + 1):
            ijk = tree.levels[ell].ijk
            for b in range(len(ijk)):
                bits = ijk[b] % 2
                M = [self.CR[ell] if bb else self.CL[ell] for bb in bits]
                r[ell][b] += mode3(M[0].T, M[1].T, M[2].T, r[ell - 1][tree.parent[ell][b]])
        return r[D]

    def far_parts(self, j):
        """(yA_far, yV_far): y_far = jk yA_far + (jk)^-1 yV_far."""
        mesh, tree = self.mesh, self.tree
        r = self.far_grids(j)
        yA = np.einsum("ndabc,ndabc->n", self.m_rwg, r[tree.rwg_box, :3])
        u = np.einsum("tabc,tabc->t", self.m_tri, r[tree.tri_box, 3])
        yV = mesh.sigma_apply(u)
        return yA, yV

    def matvec_parts(self, j):
        """(yA, yV) for the full operator: y = jk yA + (jk)^-1 yV."""
        j = np.asarray(j, dtype=np.complex128)
        yA, yV = self.far_parts(j)
        yA = yA + self.A_near @ j
        yV = yV + self.mesh.sigma_apply(self.V_near @ self.mesh.sigmaT_apply(j))
        return yA, yV

    def matvec(self, j):
        j = np.asarray(j, dtype=np.complex128)
        if j.ndim == 2:
            return np.stack([self.matvec(x) for x in j])
        yA, yV = self.matvec_parts(j)
        return 1j * self.k * yA + (1.0 / (1j * self.k)) * yV

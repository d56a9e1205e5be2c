"""Direct and dyadic factorizations of the B-spline fast EFIE (oracle; test
infrastructure only).  Sec. VI: the star-based factorization of `fastmv`
interpolates the kernel of V in T_Phi = Sigma V Sigma^T; the other two
factorizations the paper discusses are

* direct (Sec. VI-B): the vector and the scalar potential are interpolated
  together.  Every RWG carries four moments in its own leaf box: the three
  components of f_m and its surface divergence,
      m_{d,m}[i]   = int f_{m,d} l_i dS,
      m^div_m[i]   = int (div f_m) l_i dS = sum_{c in {c+, c-}} (+-1/a_c) int_c l_i dS,
  so y_m = jk m_m . (G q) + (jk)^-1 m^div_m (G q^div).  One near set (RWG
  pairs in adjacent leaf boxes) holds both parts.
* dyadic (Sec. VI-C): T_mn = jk int int f_m . (I + grad grad / k^2) g . f_n.
  Only the three RWG moment components are anterpolated; the translation is
  the 3 x 3 dyad g delta_ij + (d_i d_j g)/k^2 (symmetric: 6 distinct kernels
  per offset).  The second part equals -Phi_mn per RWG pair (integration by
  parts twice: the RWG normal component vanishes on the support boundary, and
  grad_x g = -grad_y g), so the dyadic far part is returned in the
  (yA, yV) split as yV = -(H x), H_mn = int int f_m . grad grad g . f_n.
  Near field as in the direct form.

Both reuse the uniform tree, transfers, projectors, lists and FFT
translations of `fastmv`.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import dense, fastmv
from .geometry import RWGMesh
from .moments import LeafSplines, clip_triangle, quad_order
from .quadrature import map_rule


def divergence_moments(mesh: RWGMesh, tree, subset=None):
    """[N, s', s', s'] divergence moments in each RWG's leaf box (or only for
    the RWGs listed in subset)."""
    L = tree.levels[tree.D]
    p = tree.p
    n = quad_order(p)
    ids = np.arange(mesh.N) if subset is None else np.asarray(subset)
    out = np.zeros((len(ids), L.sp, L.sp, L.sp))
    cache = {}
    for oi, m in enumerate(ids):
        b = tree.rwg_box[m]
        if b not in cache:
            cache[b] = LeafSplines(L.box_ext_lo(tree.root_lo, L.ijk[b]), L.sp, p, L.delta)
        spl = cache[b]
        for side, sgn in ((0, 1.0), (1, -1.0)):
            c = mesh.tri_pm[m, side]
            X, w = map_rule(clip_triangle(mesh.V[mesh.T[c]], spl.planes), n)
            out[oi] += spl.tensor(X.reshape(-1, 3), w.reshape(-1), np.full(w.size, sgn / mesh.area[c]))
    return out


def green_hessian(D, k):
    """d_i d_j g at separation D [..., 3], g = exp(-jkR)/(4 pi R):
    g'' r_i r_j + (g'/R)(delta_ij - r_i r_j), g' = -(jk + 1/R) g,
    g'' = ((jk + 1/R)^2 + 1/R^2) g, r = D/R."""
    R = np.sqrt(np.sum(D * D, axis=-1))
    g = dense.green(R, k)
    a = 1j * k + 1.0 / R
    g1 = -a * g
    g2 = (a * a + 1.0 / (R * R)) * g
    r = D / R[..., None]
    rr = r[..., :, None] * r[..., None, :]
    return g2[..., None, None] * rr + (g1 / R)[..., None, None] * (np.eye(3) - rr)


class _RwgNearMixin:
    def _near_rwg(self, dense_AV):
        """A_near and Phi_near (= Sigma V Sigma^T restricted) on RWG pairs in
        adjacent leaf boxes."""
        mesh = self.mesh
        nb, rb, _ = self.near_masks()
        mask = nb[rb[:, None], rb[None, :]]
        if dense_AV is not None:
            A, V = dense_AV
            S = mesh.sigma_dense()
            return sp.csr_matrix(np.where(mask, A, 0)), sp.csr_matrix(np.where(mask, S @ V @ S.T, 0))
        mi, mj = np.nonzero(mask)
        tri, loc, coef = dense.rwg_sides(mesh)
        pairs = np.unique(np.concatenate([np.stack([tri[mi, s], tri[mj, t]], 1)
                                          for s in range(2) for t in range(2)]), axis=0)
        I0, Ivv = dense.pair_integrals(mesh, pairs[:, 0], pairs[:, 1], self.k, kernel=self.kernel)
        key = pairs[:, 0] * mesh.Nt + pairs[:, 1]
        order = np.argsort(key)
        key_s = key[order]
        va = np.zeros(len(mi), dtype=np.complex128)
        vp = np.zeros(len(mi), dtype=np.complex128)
        for s, ss in ((0, 1.0), (1, -1.0)):
            for t, st in ((0, 1.0), (1, -1.0)):
                ca, cb = tri[mi, s], tri[mj, t]
                pos = order[np.searchsorted(key_s, ca * mesh.Nt + cb)]
                va += coef[mi, s] * coef[mj, t] * Ivv[pos, loc[mi, s], loc[mj, t]]
                vp += ss * st * I0[pos] / (mesh.area[ca] * mesh.area[cb])
        shape = (mesh.N, mesh.N)
        return sp.csr_matrix((va, (mi, mj)), shape=shape), sp.csr_matrix((vp, (mi, mj)), shape=shape)

    def matvec_parts(self, j):
        j = np.asarray(j, dtype=np.complex128)
        yA, yV = self.far_parts(j)
        return yA + self.A_near @ j, yV + self.Phi_near @ j


class DirectBsplineEFIE(_RwgNearMixin, fastmv.BsplineEFIE):
    """Direct factorization: RWG and divergence moments in the RWG's box."""

    def __init__(self, mesh: RWGMesh, k, p, grid_spacing, levels, n_splines=None, kernel=None,
                 near="auto", dense_AV=None, translation="fft", allow_overlap=False):
        super().__init__(mesh, k, p, grid_spacing, levels, n_splines, kernel, near=None,
                         translation=translation, allow_overlap=allow_overlap)
        self.m_div = divergence_moments(mesh, self.tree)
        if near is None:
            self.A_near = sp.csr_matrix((mesh.N, mesh.N), dtype=np.complex128)
            self.Phi_near = sp.csr_matrix((mesh.N, mesh.N), dtype=np.complex128)
        else:
            self.A_near, self.Phi_near = self._near_rwg(dense_AV)

    def far_parts(self, j):
        tree = self.tree
        D = tree.D
        LD = tree.levels[D]
        q = {D: np.zeros((len(LD.boxes), 4, LD.sp, LD.sp, LD.sp), dtype=np.complex128)}
        np.add.at(q[D], (tree.rwg_box, slice(0, 3)), j[:, None, None, None, None] * self.m_rwg)
        np.add.at(q[D], (tree.rwg_box, 3), j[:, None, None, None] * self.m_div)
        r = self._far_pass(q)
        yA = np.einsum("ndabc,ndabc->n", self.m_rwg, r[tree.rwg_box, :3])
        yV = np.einsum("nabc,nabc->n", self.m_div, r[tree.rwg_box, 3])
        return yA, yV

    def _far_pass(self, q):
        """Upward transfers, stabilized translations, downward transfers of
        leaf grids q[D] [B,C,s',s',s']; returns the leaf output grids."""
        tree = self.tree
        D = tree.D
        C = q[D].shape[1]
        for ell in range(D, tree.top, -1):
            pa = tree.levels[ell - 1]
            qp = np.zeros((len(pa.boxes), C, pa.sp, pa.sp, pa.sp), dtype=np.complex128)
            ijk = tree.levels[ell].ijk
            for b in range(len(ijk)):
                M = [self.CR[ell] if bb else self.CL[ell] for bb in ijk[b] % 2]
                qp[tree.parent[ell][b]] += fastmv.mode3(M[0], M[1], M[2], q[ell][b])
            q[ell - 1] = qp
        r = {}
        for ell in self.grid_levels:
            P = self.P[ell]
            r[ell] = fastmv.mode3(P.T, P.T, P.T, self._translate(ell, fastmv.mode3(P, P, P, q[ell])))
        for ell in range(tree.top + 1, D + 1):
            ijk = tree.levels[ell].ijk
            for b in range(len(ijk)):
                M = [self.CR[ell] if bb else self.CL[ell] for bb in ijk[b] % 2]
                r[ell][b] += fastmv.mode3(M[0].T, M[1].T, M[2].T, r[ell - 1][tree.parent[ell][b]])
        return r[D]

    def _translate(self, ell, qt):
        return self._translate_level(ell, qt)


class DyadicBsplineEFIE(DirectBsplineEFIE):
    """Dyadic factorization: three RWG moment components, 3 x 3 dyadic
    translation.  kernel_hessian(D) -> [..., 3, 3] must accompany a custom
    kernel."""

    def __init__(self, mesh: RWGMesh, k, p, grid_spacing, levels, n_splines=None, kernel=None,
                 kernel_hessian=None, near="auto", dense_AV=None, translation="fft", allow_overlap=False):
        if (kernel is None) != (kernel_hessian is None):
            raise ValueError("a custom kernel needs its Hessian")
        self.kernel_hessian = kernel_hessian
        super().__init__(mesh, k, p, grid_spacing, levels, n_splines, kernel, near, dense_AV, translation,
                         allow_overlap)

    def _hess(self, D):
        if self.kernel_hessian is not None:
            return self.kernel_hessian(D)
        return green_hessian(D, self.k)

    def far_parts(self, j):
        tree = self.tree
        D = tree.D
        LD = tree.levels[D]
        q = {D: np.zeros((len(LD.boxes), 3, LD.sp, LD.sp, LD.sp), dtype=np.complex128)}
        np.add.at(q[D], tree.rwg_box, j[:, None, None, None, None] * self.m_rwg)
        r = self._far_pass(q)              # [B, 6, ...]: g q_d, then sum_e H_de q_e (see _translate_dyad)
        yA = np.einsum("ndabc,ndabc->n", self.m_rwg, r[tree.rwg_box, :3])
        yH = np.einsum("ndabc,ndabc->n", self.m_rwg, r[tree.rwg_box, 3:])
        return yA, -yH

    def _translate(self, ell, qt):
        return self._translate_dyad(ell, qt)

    def _translate_dyad(self, ell, qt):
        """r~_x = [sum_y G_xy q~_y (3 comps), sum_y sum_e H_xy,de q~_y,e (3 comps)],
        H = grad grad g, by FFTs of size 2 s_hat - 1; qt [B,3,n,n,n]."""
        L = self.tree.levels[ell]
        ns = L.shat
        xs, ys = self.IL[ell]
        B = qt.shape[0]
        n = 2 * ns - 1
        if len(xs) == 0:
            return np.zeros((B, 6, ns, ns, ns), dtype=np.complex128)
        offs = L.ijk[xs] - L.ijk[ys]
        uo, inv = np.unique(offs, axis=0, return_inverse=True)
        inv = inv.reshape(-1)
        t = np.arange(-(ns - 1), ns)
        idx = np.mod(t, n)
        Q = np.fft.fftn(np.pad(qt, [(0, 0), (0, 0)] + [(0, n - ns)] * 3), axes=(-3, -2, -1))
        R = np.zeros((B, 6, n, n, n), dtype=np.complex128)
        for oi, o in enumerate(uo):
            Dv = (o[None, None, None, :] * L.h + np.stack(np.meshgrid(t, t, t, indexing="ij"), axis=-1) * L.Delta)
            Kg = np.zeros((n, n, n), dtype=np.complex128)
            Kg[np.ix_(idx, idx, idx)] = self._kernel_fn(Dv)
            Kg = np.fft.fftn(Kg)
            H = self._hess(Dv)                                       # [2ns-1]^3 x 3 x 3
            Kh = np.zeros((3, 3, n, n, n), dtype=np.complex128)
            for a in range(3):
                for b in range(3):
                    Kc = np.zeros((n, n, n), dtype=np.complex128)
                    Kc[np.ix_(idx, idx, idx)] = H[..., a, b]
                    Kh[a, b] = np.fft.fftn(Kc)
            for pi in np.nonzero(inv == oi)[0]:
                x, y = xs[pi], ys[pi]
                R[x, :3] += Kg[None] * Q[y]
                R[x, 3:] += np.einsum("abxyz,bxyz->axyz", Kh, Q[y])
        return np.fft.ifftn(R, axes=(-3, -2, -1))[..., :ns, :ns, :ns]


# ------------------------------------------------------------ nonuniform tree
# The direct and dyadic factorizations on the nonuniform octree of Sec. VII
# (`oracle.nonuniform`): every RWG's moments (and, for the direct form, its
# divergence moments) in its own leaf with that level's splines; the leaves of
# every level anterpolated into, and interpolated from, their own level's grids;
# the near field on the RWG pairs of near leaves (ancestors on the coarser of
# the two levels adjacent or equal).

from . import nonuniform as _nu  # noqa: E402  (the nonuniform tree does not import this module)


class AdaptiveDirectBsplineEFIE(_RwgNearMixin, _nu.AdaptiveBsplineEFIE):
    """Direct factorization (Sec. VI-B) on the nonuniform octree."""

    n_comp = 4

    def __init__(self, mesh: RWGMesh, k, p, max_elems=200, max_prot=0.25, top=2, n_splines=None, kernel=None,
                 near="auto", dense_AV=None, translation="fft", root=None, max_depth=30, allow_overlap=False):
        super().__init__(mesh, k, p, max_elems, max_prot, top, n_splines, kernel, near=None, dense_AV=None,
                         translation=translation, root=root, max_depth=max_depth, allow_overlap=allow_overlap)
        self.m_div_l = {ell: divergence_moments(mesh, _nu._LevelView(self.tree, ell), self.rwg_at[ell])
                        for ell in self.grid_levels}
        if near is None:
            self.A_near = sp.csr_matrix((mesh.N, mesh.N), dtype=np.complex128)
            self.Phi_near = sp.csr_matrix((mesh.N, mesh.N), dtype=np.complex128)
        else:
            self.A_near, self.Phi_near = self._near_rwg(dense_AV)

    def _leaf_grids(self, j):
        """Grids of every level with the anterpolated moments of the RWGs whose
        leaves lie there: components 0..2 the RWG moments, 3 (direct form) the
        divergence moments."""
        tree = self.tree
        q = {}
        for ell in self.grid_levels:
            L = tree.levels[ell]
            q[ell] = np.zeros((len(L.boxes), self.n_comp, L.sp, L.sp, L.sp), dtype=np.complex128)
            ra = self.rwg_at[ell]
            np.add.at(q[ell], (tree.rwg_box[ra], slice(0, 3)), j[ra][:, None, None, None, None] * self.m_rwg_l[ell])
            if self.n_comp == 4:
                np.add.at(q[ell], (tree.rwg_box[ra], 3), j[ra][:, None, None, None] * self.m_div_l[ell])
        return q

    def _far_pass_levels(self, q):
        """Upward transfers (children added into their parents), stabilized
        translations of every level, downward transfers; the output grids of
        every level."""
        tree = self.tree
        for ell in range(tree.D, tree.top, -1):
            ijk = tree.levels[ell].ijk
            for b in range(len(ijk)):
                M = [self.CR[ell] if bb else self.CL[ell] for bb in ijk[b] % 2]
                q[ell - 1][tree.parent[ell][b]] += fastmv.mode3(M[0], M[1], M[2], q[ell][b])
        r = {}
        for ell in self.grid_levels:
            P = self.P[ell]
            r[ell] = fastmv.mode3(P.T, P.T, P.T, self._translate(ell, fastmv.mode3(P, P, P, q[ell])))
        for ell in range(tree.top + 1, tree.D + 1):
            ijk = tree.levels[ell].ijk
            for b in range(len(ijk)):
                M = [self.CR[ell] if bb else self.CL[ell] for bb in ijk[b] % 2]
                r[ell][b] += fastmv.mode3(M[0].T, M[1].T, M[2].T, r[ell - 1][tree.parent[ell][b]])
        return r

    def _translate(self, ell, qt):
        return self._translate_level(ell, qt)

    def far_parts(self, j):
        j = np.asarray(j, dtype=np.complex128)
        tree = self.tree
        r = self._far_pass_levels(self._leaf_grids(j))
        yA = np.zeros(self.mesh.N, dtype=np.complex128)
        yV = np.zeros(self.mesh.N, dtype=np.complex128)
        for ell in self.grid_levels:
            ra = self.rwg_at[ell]
            rb = r[ell][tree.rwg_box[ra]]
            yA[ra] = np.einsum("ndabc,ndabc->n", self.m_rwg_l[ell], rb[:, :3])
            yV[ra] = np.einsum("nabc,nabc->n", self.m_div_l[ell], rb[:, 3])
        return yA, yV

    def matvec_parts(self, j):
        return _RwgNearMixin.matvec_parts(self, j)


class AdaptiveDyadicBsplineEFIE(AdaptiveDirectBsplineEFIE):
    """Dyadic factorization (Sec. VI-C) on the nonuniform octree: three RWG
    moment components, translated with g and with the Hessian of g; the
    scalar part is returned as -(H x).  kernel_hessian(D) -> [..., 3, 3] must
    accompany a custom kernel."""

    n_comp = 3

    def __init__(self, mesh: RWGMesh, k, p, max_elems=200, max_prot=0.25, top=2, n_splines=None, kernel=None,
                 kernel_hessian=None, near="auto", dense_AV=None, translation="fft", root=None, max_depth=30,
                 allow_overlap=False):
        if (kernel is None) != (kernel_hessian is None):
            raise ValueError("a custom kernel needs its Hessian")
        self.kernel_hessian = kernel_hessian
        super().__init__(mesh, k, p, max_elems, max_prot, top, n_splines, kernel, near, dense_AV, translation,
                         root, max_depth, allow_overlap)

    def _hess(self, D):
        if self.kernel_hessian is not None:
            return self.kernel_hessian(D)
        return green_hessian(D, self.k)

    def _translate(self, ell, qt):
        return DyadicBsplineEFIE._translate_dyad(self, ell, qt)

    def far_parts(self, j):
        j = np.asarray(j, dtype=np.complex128)
        tree = self.tree
        r = self._far_pass_levels(self._leaf_grids(j))    # [B, 6, ...]: g q_d, then sum_e H_de q_e
        yA = np.zeros(self.mesh.N, dtype=np.complex128)
        yH = np.zeros(self.mesh.N, dtype=np.complex128)
        for ell in self.grid_levels:
            ra = self.rwg_at[ell]
            rb = r[ell][tree.rwg_box[ra]]
            yA[ra] = np.einsum("ndabc,ndabc->n", self.m_rwg_l[ell], rb[:, :3])
            yH[ra] = np.einsum("ndabc,ndabc->n", self.m_rwg_l[ell], rb[:, 3:])
        return yA, -yH

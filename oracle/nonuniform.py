"""Nonuniform octree variant of the multilevel B-spline fast EFIE (oracle;
test infrastructure only).

Tree (Sec. VII): starting from the root cube, a box is subdivided while it
holds more than `max_elems` elements (triangles, by centroid), and subdivision
stops where a basis function of the box would protrude from its child box by
more than `max_prot` of the child's edge.  Leaves therefore sit on several
levels; a box exists when it holds a basis function.

Spline parameters per level ell (box edge h_ell), from the deepest level D up
to the top grid level:
  * s_D = n_splines (default p + 4, Sec. VII-B); going up, s stays while the
    box edge is below lambda/2 and becomes 2s - p otherwise (Sec. IV-C, IV-D;
    the level's own box edge decides); delta_ell = h_ell/(s_ell - p).
  * buffer splines (Sec. IV-C, IV-D, including the rule for leaves on the
    parent level):  s_b = max(ceil(s_b,child / 2), s_b,leaves) for constant s,
    s_b = max(s_b,child, s_b,leaves) for s -> 2s - p, where
    s_b,leaves = ceil(largest protrusion of the level's own leaf functions
    beyond their boxes / delta_ell).

Every basis function sits in the leaf holding its point (edge midpoint for an
RWG, centroid for a triangle) and is anterpolated and interpolated
there with that box's splines.  The grids of every box go up by knot
insertion and come down by the transpose; level ell translates the pairs of
non-adjacent boxes with adjacent parents, and every non-adjacent pair on the
top grid level (standard H2 admissibility).  Two leaves x, y on levels lx <= ly are near
when x and the ancestor of y on level lx are adjacent or equal: the
inadmissible leaf blocks of the level-consistent block tree.  Every pair of
leaves is thus either near or translated on exactly one level.

With every box subdivided down to one depth the construction is the uniform
tree of `oracle.tree` (the uniform-limit pin).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import fastmv
from .bspline import S_REMOVE, open_knots, projector, restriction_matrix
from .geometry import RWGMesh
from .moments import pulse_moments, rwg_moments
from .tree import LevelParams, box_ijk, interaction_lists


@dataclass
class AdaptiveTree:
    root_lo: np.ndarray
    root_edge: float
    D: int                       # deepest level
    p: int
    top: int                     # top grid level
    levels: dict                 # level -> LevelParams (boxes, ijk of every box on the level)
    is_leaf: dict                # level -> [B_l] bool
    parent: dict                 # level -> [B_l] index of the parent box on level - 1
    rwg_level: np.ndarray        # [N] level of the RWG's leaf
    rwg_box: np.ndarray          # [N] index of the leaf on that level
    tri_level: np.ndarray        # [Nt]
    tri_box: np.ndarray          # [Nt]


def _supports(mesh: RWGMesh):
    V = mesh.V
    rs = np.concatenate([V[mesh.T[mesh.tri_pm[:, 0]]], V[mesh.T[mesh.tri_pm[:, 1]]]], axis=1)   # [N,6,3]
    ts = V[mesh.T]                                                                          # [Nt,3,3]
    mid = (V[mesh.edges[:, 0]] + V[mesh.edges[:, 1]]) * 0.5
    return (mid, rs.min(axis=1), rs.max(axis=1)), (mesh.centroid, ts.min(axis=1), ts.max(axis=1))


def _protrusion(pt, smin, smax, root_lo, root_edge, level):
    """Largest distance by which the supports leave the boxes of their points
    on the given level (0 for none)."""
    if len(pt) == 0:
        return 0.0
    h = root_edge / (2 ** level)
    blo = root_lo + box_ijk(pt, root_lo, root_edge, level) * h
    return float(max(np.max(np.maximum(blo - smin, 0.0)), np.max(np.maximum(smax - (blo + h), 0.0)), 0.0))


def build_adaptive_tree(mesh: RWGMesh, k, p, max_elems=200, max_prot=0.25, top=2, n_splines=None,
                        root=None, max_depth=30, allow_overlap=False) -> AdaptiveTree:
    if p not in S_REMOVE:
        raise ValueError("p must be in 1..6")
    (rpt, rmin, rmax), (tpt, tmin, tmax) = _supports(mesh)
    V = mesh.V
    if root is None:
        lo, hi = V.min(axis=0), V.max(axis=0)
        root_edge = float(np.max(hi - lo))
        root_lo = (lo + hi) * 0.5 - root_edge * 0.5
    else:
        root_lo, root_edge = np.asarray(root[0], dtype=np.float64), float(root[1])

    # subdivision, level by level: key (i, j, k) -> (RWG ids, triangle ids)
    boxes = {0: {(0, 0, 0): (np.arange(mesh.N), np.arange(mesh.Nt))}}
    leaf_keys = {}
    level = 0
    while boxes[level]:
        nxt = {}
        leaf_keys[level] = set()
        for key, (rw, tr) in boxes[level].items():
            split = len(tr) > max_elems and level < max_depth
            if split:
                prot = max(_protrusion(rpt[rw], rmin[rw], rmax[rw], root_lo, root_edge, level + 1),
                           _protrusion(tpt[tr], tmin[tr], tmax[tr], root_lo, root_edge, level + 1))
                split = prot <= max_prot * root_edge / (2 ** (level + 1))
            if not split:
                leaf_keys[level].add(key)
                continue
            rc = box_ijk(rpt[rw], root_lo, root_edge, level + 1)
            tc = box_ijk(tpt[tr], root_lo, root_edge, level + 1)
            for ids, cc, slot in ((rw, rc, 0), (tr, tc, 1)):
                for i, c in zip(ids, map(tuple, cc)):
                    ent = nxt.setdefault(c, ([], []))
                    ent[slot].append(i)
        boxes[level + 1] = {c: (np.array(a, dtype=np.int64), np.array(b, dtype=np.int64))
                            for c, (a, b) in nxt.items()}
        level += 1
    D = max(lv for lv, ks in leaf_keys.items() if ks)
    if any(leaf_keys.get(lv) for lv in range(0, top)):
        raise ValueError("a leaf lies above the top grid level")
    if top > D:
        raise ValueError("top grid level below the deepest leaf")

    lam = 2.0 * math.pi / k
    s_leaf = n_splines if n_splines else p + 4
    lv = {}
    is_leaf, parent = {}, {}
    rwg_level = np.full(mesh.N, -1, dtype=np.int64)
    rwg_box = np.full(mesh.N, -1, dtype=np.int64)
    tri_level = np.full(mesh.Nt, -1, dtype=np.int64)
    tri_box = np.full(mesh.Nt, -1, dtype=np.int64)
    cur_s, cur_sb = s_leaf, 0
    for ell in range(D, top - 1, -1):
        h = root_edge / (2 ** ell)
        if ell < D and h >= 0.5 * lam:
            cur_s = 2 * cur_s - p
        delta = h / (cur_s - p)
        keys = sorted(boxes[ell].keys())
        leaves = leaf_keys.get(ell, set())
        # protrusion of this level's own leaf functions
        prot = 0.0
        for key in leaves:
            rw, tr = boxes[ell][key]
            prot = max(prot, _protrusion(rpt[rw], rmin[rw], rmax[rw], root_lo, root_edge, ell),
                       _protrusion(tpt[tr], tmin[tr], tmax[tr], root_lo, root_edge, ell))
        sb_leaves = int(math.ceil(prot / delta))
        if ell == D:
            cur_sb = sb_leaves
        else:
            child_s = lv[ell + 1].s
            cur_sb = max((cur_sb + 1) // 2 if cur_s == child_s else cur_sb, sb_leaves)
        if 2 * cur_sb >= cur_s - p and not allow_overlap:
            raise ValueError("buffer splines leave no gap between far interpolation domains "
                             f"on level {ell} (s_b = {cur_sb}, s = {cur_s})")
        sp_ = cur_s + 2 * cur_sb
        shat = sp_ - 2 * S_REMOVE[p]
        if shat <= p:
            raise ValueError("too few splines after stabilization")
        L = LevelParams(level=ell, h=h, s=cur_s, sb=cur_sb, sp=sp_, shat=shat, delta=delta,
                        Delta=(sp_ - p) * delta / (shat - 1))
        L.boxes = {key: i for i, key in enumerate(keys)}
        L.ijk = np.array(keys, dtype=np.int64).reshape(-1, 3)
        lv[ell] = L
        is_leaf[ell] = np.array([key in leaves for key in keys], dtype=bool)
        for key in leaves:
            rw, tr = boxes[ell][key]
            rwg_level[rw], rwg_box[rw] = ell, L.boxes[key]
            tri_level[tr], tri_box[tr] = ell, L.boxes[key]
    for ell in range(D, top, -1):
        up = lv[ell - 1].boxes
        parent[ell] = np.array([up[(i // 2, j // 2, kk // 2)] for (i, j, kk) in map(tuple, lv[ell].ijk)],
                               dtype=np.int64)
    assert (rwg_level >= 0).all() and (tri_level >= 0).all()
    return AdaptiveTree(root_lo=root_lo, root_edge=root_edge, D=D, p=p, top=top, levels=lv,
                        is_leaf=is_leaf, parent=parent, rwg_level=rwg_level, rwg_box=rwg_box,
                        tri_level=tri_level, tri_box=tri_box)


def leaf_index(tree: AdaptiveTree):
    """Global numbering of the leaves of all levels: returns (level [n_leaves],
    ijk [n_leaves,3], offset per level) and the leaf of every RWG / triangle."""
    lvl, ijk, off = [], [], {}
    for ell in range(tree.top, tree.D + 1):
        L = tree.levels[ell]
        sel = np.nonzero(tree.is_leaf[ell])[0]
        off[ell] = (len(lvl), sel)
        lvl.extend([ell] * len(sel))
        ijk.extend(L.ijk[sel].tolist())
    lvl = np.array(lvl, dtype=np.int64)
    ijk = np.array(ijk, dtype=np.int64).reshape(-1, 3)

    def glob(levels, box):
        out = np.empty(len(levels), dtype=np.int64)
        for ell, (o, sel) in off.items():
            pos = {b: o + i for i, b in enumerate(sel)}
            m = levels == ell
            out[m] = [pos[b] for b in box[m]]
        return out

    return lvl, ijk, glob(tree.rwg_level, tree.rwg_box), glob(tree.tri_level, tree.tri_box)


def near_leaf_pairs(tree: AdaptiveTree):
    """[n_leaves, n_leaves] bool: leaves x, y near when, on the coarser of their
    two levels, x's and y's ancestors are adjacent or equal."""
    lvl, ijk, _, _ = leaf_index(tree)
    lmin = np.minimum(lvl[:, None], lvl[None, :])
    ax = ijk[:, None, :] >> (lvl[:, None] - lmin)[..., None]
    ay = ijk[None, :, :] >> (lvl[None, :] - lmin)[..., None]
    return np.abs(ax - ay).max(axis=2) <= 1


class _LevelView:
    """One level of an adaptive tree seen as the leaf level of a uniform tree,
    so that the oracle's moment routines serve every leaf level."""

    def __init__(self, tree: AdaptiveTree, ell):
        self.levels = {ell: tree.levels[ell]}
        self.D = ell
        self.p = tree.p
        self.root_lo = tree.root_lo
        self.rwg_box = tree.rwg_box
        self.tri_box = tree.tri_box


class AdaptiveBsplineEFIE(fastmv.BsplineEFIE):
    """The fast operator of `oracle.fastmv` on a nonuniform octree: the same
    moments, transfers, projectors and translations, with anterpolation and
    interpolation on the leaves of every level and the near field of the
    level-consistent block tree."""

    def __init__(self, mesh: RWGMesh, k, p, max_elems=200, max_prot=0.25, top=2, n_splines=None,
                 kernel=None, near="auto", dense_AV=None, translation="fft", root=None, max_depth=30,
                 allow_overlap=False):
        self.mesh = mesh
        self.k = k
        self.p = p
        self.kernel = kernel
        self.translation = translation
        self.tree = tree = build_adaptive_tree(mesh, k, p, max_elems, max_prot, top, n_splines, root,
                                               max_depth, allow_overlap)
        D, top = tree.D, tree.top
        self.grid_levels = list(range(D, top - 1, -1))
        self.CL, self.CR = {}, {}
        for ell in range(D, top, -1):
            c, pa = tree.levels[ell], tree.levels[ell - 1]
            r = int(round(pa.delta / c.delta))
            Up = open_knots(-pa.sb * r, (pa.s - p + pa.sb) * r, pa.sp, p)
            UcL = open_knots(-c.sb, (c.s - p) + c.sb, c.sp, p)
            UcR = open_knots((c.s - p) - c.sb, 2 * (c.s - p) + c.sb, c.sp, p)
            self.CL[ell] = restriction_matrix(Up, UcL, p)
            self.CR[ell] = restriction_matrix(Up, UcR, p)
        self.P = {}
        for ell in self.grid_levels:
            L = tree.levels[ell]
            self.P[ell] = projector(open_knots(0.0, float(L.sp - p), L.sp, p), p, S_REMOVE[p])[0]
        # moments of every function in its own leaf box, grouped by leaf level
        self.rwg_at, self.tri_at, self.m_rwg_l, self.m_tri_l = {}, {}, {}, {}
        for ell in self.grid_levels:
            view = _LevelView(tree, ell)
            self.rwg_at[ell] = np.nonzero(tree.rwg_level == ell)[0]
            self.tri_at[ell] = np.nonzero(tree.tri_level == ell)[0]
            self.m_rwg_l[ell] = rwg_moments(mesh, view, self.rwg_at[ell])
            self.m_tri_l[ell] = pulse_moments(mesh, view, self.tri_at[ell])
        self.IL = {ell: interaction_lists(tree, ell) for ell in self.grid_levels}
        self._leaves = leaf_index(tree)
        if near is None:
            import scipy.sparse as sp_
            self.A_near = sp_.csr_matrix((mesh.N, mesh.N), dtype=np.complex128)
            self.V_near = sp_.csr_matrix((mesh.Nt, mesh.Nt), dtype=np.complex128)
        else:
            self.A_near, self.V_near = self._near(dense_AV)

    def near_masks(self):
        _, _, rl, tl = self._leaves
        return near_leaf_pairs(self.tree), rl, tl

    def far_grids(self, j):
        """Far-field output grids r[level] [B_l,4,s',s',s'] for one current vector."""
        tree, mesh = self.tree, self.mesh
        rho = mesh.sigmaT_apply(j)
        q = {}
        for ell in self.grid_levels:
            L = tree.levels[ell]
            q[ell] = np.zeros((len(L.boxes), 4, L.sp, L.sp, L.sp), dtype=np.complex128)
            ra, ta = self.rwg_at[ell], self.tri_at[ell]
            np.add.at(q[ell], (tree.rwg_box[ra], slice(0, 3)), j[ra][:, None, None, None, None] * self.m_rwg_l[ell])
            np.add.at(q[ell], (tree.tri_box[ta], 3), rho[ta][:, None, None, None] * self.m_tri_l[ell])
        for ell in range(tree.D, tree.top, -1):
            ijk = tree.levels[ell].ijk
            for b in range(len(ijk)):
                M = [self.CR[ell] if bb else self.CL[ell] for bb in ijk[b] % 2]
                q[ell - 1][tree.parent[ell][b]] += fastmv.mode3(M[0], M[1], M[2], q[ell][b])
        r = {}
        for ell in self.grid_levels:
            P = self.P[ell]
            r[ell] = fastmv.mode3(P.T, P.T, P.T, self._translate_level(ell, fastmv.mode3(P, P, P, q[ell])))
        for ell in range(tree.top + 1, tree.D + 1):
            ijk = tree.levels[ell].ijk
            for b in range(len(ijk)):
                M = [self.CR[ell] if bb else self.CL[ell] for bb in ijk[b] % 2]
                r[ell][b] += fastmv.mode3(M[0].T, M[1].T, M[2].T, r[ell - 1][tree.parent[ell][b]])
        return r

    def far_parts(self, j):
        mesh, tree = self.mesh, self.tree
        r = self.far_grids(j)
        yA = np.zeros(mesh.N, dtype=np.complex128)
        u = np.zeros(mesh.Nt, dtype=np.complex128)
        for ell in self.grid_levels:
            ra, ta = self.rwg_at[ell], self.tri_at[ell]
            yA[ra] = np.einsum("ndabc,ndabc->n", self.m_rwg_l[ell], r[ell][tree.rwg_box[ra], :3])
            u[ta] = np.einsum("tabc,tabc->t", self.m_tri_l[ell], r[ell][tree.tri_box[ta], 3])
        return yA, mesh.sigma_apply(u)


def far_coverage(op: AdaptiveBsplineEFIE, kind="rwg"):
    """[n, n] count of the levels on which each pair of functions is
    translated (brute force over the interaction lists and the subtrees)."""
    tree = op.tree
    lvl_f = tree.rwg_level if kind == "rwg" else tree.tri_level
    box_f = tree.rwg_box if kind == "rwg" else tree.tri_box
    n = len(lvl_f)
    cov = np.zeros((n, n), dtype=np.int16)
    for ell in op.grid_levels:
        # ancestor on level ell of every function (or -1 above its leaf)
        anc = np.full(n, -1, dtype=np.int64)
        ok = lvl_f >= ell
        key = tree.levels[ell].boxes
        Lf = {e: tree.levels[e].ijk for e in op.grid_levels}
        for i in np.nonzero(ok)[0]:
            c = Lf[lvl_f[i]][box_f[i]] >> (lvl_f[i] - ell)
            anc[i] = key[tuple(c)]
        xs, ys = op.IL[ell]
        pair = np.zeros((len(key), len(key)), dtype=np.int16)
        pair[xs, ys] = 1
        sel = np.nonzero(anc >= 0)[0]
        cov[np.ix_(sel, sel)] += pair[np.ix_(anc[sel], anc[sel])]
    return cov

"""Uniform octree and per-level spline parameters (oracle; test
infrastructure only).

* Regular octree of axis-aligned cubes (Sec. III, Sec. IV).  Root cube centred
  on the bounding-box centre with edge h_leaf 2^D, D the smallest depth with
  h_leaf 2^D >= bounding-box edge.  Box index floor((x - root_lo)/h_l), clamped;
  an RWG sits in the box of its edge midpoint, a triangle in the box of its
  centroid (the paper does not say; ties go to the box below by the floor).
* Leaf level: s = p + 4 splines by default (Sec. VII-B), knot spacing
  delta = grid_spacing, box edge h = (s - p) delta, buffer splines
  s_b = ceil(max protrusion / delta) (Sec. III-B).  We require 2 s_b < s - p at
  every level, so the extended interpolation domains of boxes two apart stay
  disjoint (Sec. VII-B: one buffer spline at s = p + 4 leaves half a box).
* Going to the parent level (Sec. IV-C, IV-D; the parent's box edge, without
  buffers, is the edge length compared with lambda/2): if h_parent < lambda/2,
  s stays and s_b = ceil(s_b/2); else s = 2s - p and s_b stays.  s' = s + 2 s_b, s_hat = s' - 2 s_remove(p).
* `levels` levels, counted up from the leaf, carry grids (a parameter of this library, not the paper's); the
  top grid level translates every non-adjacent pair, lower levels the standard
  interaction list (non-adjacent boxes with adjacent parents: the standard H2 rule, which the paper does not spell out).
  Near field: leaf boxes with |dx|_inf <= 1.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from .bspline import S_REMOVE
from .geometry import RWGMesh


@dataclass
class LevelParams:
    level: int
    h: float
    s: int
    sb: int
    sp: int          # s' = s + 2 s_b
    shat: int        # stabilized count
    delta: float     # knot spacing
    Delta: float     # interpolation-point spacing
    boxes: dict = field(default_factory=dict)   # (i,j,k) -> index
    ijk: np.ndarray = None                      # [B,3]

    def box_ext_lo(self, root_lo, ijk):
        return root_lo + np.asarray(ijk) * self.h - self.sb * self.delta


@dataclass
class Tree:
    root_lo: np.ndarray
    root_edge: float
    D: int
    p: int
    top: int
    levels: dict                 # level -> LevelParams
    rwg_box: np.ndarray          # [N] leaf box index
    tri_box: np.ndarray          # [Nt] leaf box index
    parent: dict                 # level -> [B_l] index of parent box at level-1


def box_ijk(points, root_lo, root_edge, level):
    h = root_edge / (2 ** level)
    idx = np.floor((points - root_lo) / h).astype(np.int64)
    return np.clip(idx, 0, 2 ** level - 1)


def build_tree(mesh: RWGMesh, k, p, grid_spacing, levels, n_splines=None,
               allow_overlap=False) -> Tree:
    if p not in S_REMOVE:
        raise ValueError("p must be in 1..6")
    s = n_splines if n_splines else p + 4
    delta = float(grid_spacing)
    h_leaf = (s - p) * delta
    V = mesh.V
    lo = V.min(axis=0)
    hi = V.max(axis=0)
    edge = float(np.max(hi - lo))
    D = 0
    while h_leaf * (2 ** D) < edge:
        D += 1
    if levels < 1 or levels > D + 1:
        raise ValueError("levels must be in 1..D+1")
    root_edge = h_leaf * (2 ** D)
    root_lo = (lo + hi) * 0.5 - root_edge * 0.5
    lam = 2.0 * math.pi / k

    mid = (V[mesh.edges[:, 0]] + V[mesh.edges[:, 1]]) * 0.5
    cen = mesh.centroid
    rwg_ijk = box_ijk(mid, root_lo, root_edge, D)
    tri_ijk = box_ijk(cen, root_lo, root_edge, D)

    # maximum protrusion of a support beyond its leaf box
    prot = 0.0
    for pts_ijk, supp in ((rwg_ijk, np.stack([V[mesh.T[mesh.tri_pm[:, 0]]],
                                             V[mesh.T[mesh.tri_pm[:, 1]]]], axis=1).reshape(-1, 6, 3)),
                          (tri_ijk, V[mesh.T])):
        blo = root_lo + pts_ijk * h_leaf
        bhi = blo + h_leaf
        smin = supp.min(axis=1)
        smax = supp.max(axis=1)
        prot = max(prot, float(np.max(np.maximum(blo - smin, 0.0))),
                   float(np.max(np.maximum(smax - bhi, 0.0))))
    sb = int(math.ceil(prot / delta))

    top = D - levels + 1
    lv = {}
    h = h_leaf
    cur_s, cur_sb, cur_delta = s, sb, delta
    for ell in range(D, top - 1, -1):
        if ell < D:
            h = root_edge / (2 ** ell)
            if h < 0.5 * lam:
                cur_sb = (cur_sb + 1) // 2
                cur_delta = cur_delta * 2.0
            else:
                cur_s = 2 * cur_s - p
        if 2 * cur_sb >= cur_s - p and not allow_overlap:
            # boxes two apart would have touching or overlapping interpolation
            # domains, so far-pair kernel samples could hit R = 0
            raise ValueError("grid spacing too small for the mesh: buffer splines "
                             f"s_b = {cur_sb} leave no gap between far interpolation domains")
        sp = cur_s + 2 * cur_sb
        shat = sp - 2 * S_REMOVE[p]
        if shat <= p:
            raise ValueError("too few splines after stabilization")
        Delta = (sp - p) * cur_delta / (shat - 1)
        lv[ell] = LevelParams(level=ell, h=root_edge / (2 ** ell), s=cur_s, sb=cur_sb, sp=sp,
                              shat=shat, delta=cur_delta, Delta=Delta)

    # occupied boxes (union of RWG and triangle boxes), parents
    leaf_keys = sorted(set(map(tuple, rwg_ijk)) | set(map(tuple, tri_ijk)))
    keys = {D: leaf_keys}
    for ell in range(D - 1, top - 1, -1):
        keys[ell] = sorted(set((i // 2, j // 2, kk // 2) for (i, j, kk) in keys[ell + 1]))
    parent = {}
    for ell in range(D, top - 1, -1):
        L = lv[ell]
        L.boxes = {key: i for i, key in enumerate(keys[ell])}
        L.ijk = np.array(keys[ell], dtype=np.int64).reshape(-1, 3)
    for ell in range(D, top, -1):
        up = lv[ell - 1].boxes
        parent[ell] = np.array([up[(i // 2, j // 2, kk // 2)] for (i, j, kk) in keys[ell]], dtype=np.int64)
    leaf = lv[D].boxes
    rwg_box = np.array([leaf[tuple(x)] for x in rwg_ijk], dtype=np.int64)
    tri_box = np.array([leaf[tuple(x)] for x in tri_ijk], dtype=np.int64)
    return Tree(root_lo=root_lo, root_edge=root_edge, D=D, p=p, top=top, levels=lv,
                rwg_box=rwg_box, tri_box=tri_box, parent=parent)


def interaction_lists(tree: Tree, ell):
    """Far pairs (x, y) translated at level ell: non-adjacent boxes whose
    parents are adjacent; at the top grid level every non-adjacent pair."""
    L = tree.levels[ell]
    ijk = L.ijk
    dif = np.abs(ijk[:, None, :] - ijk[None, :, :]).max(axis=2)
    far = dif >= 2
    if ell > tree.top:
        pijk = ijk // 2
        pd = np.abs(pijk[:, None, :] - pijk[None, :, :]).max(axis=2)
        far &= pd <= 1
    xs, ys = np.nonzero(far)
    return xs, ys


def near_box_pairs(tree: Tree):
    L = tree.levels[tree.D]
    ijk = L.ijk
    dif = np.abs(ijk[:, None, :] - ijk[None, :, :]).max(axis=2)
    return dif <= 1      # [B,B] boolean

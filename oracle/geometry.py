"""RWG basis functions and the star matrix (oracle; test infrastructure only).

Sec. II: Galerkin RWG functions *without* edge-length normalization,
    f_m(x) = (x - x_m^+) / (2 a_m^+)   on c_m^+,
    f_m(x) = (x_m^- - x) / (2 a_m^-)   on c_m^-,
so div f_m = +1/a^+ on c^+ and -1/a^- on c^-.

Sec. VI-A: the star matrix has Sigma[m, c_m^+] = +1 and Sigma[m, c_m^-] = -1, and
the pulse basis is phi_c = 1/a_c on triangle c, so div f_m = sum_c Sigma[m,c] phi_c.

Orientation (the paper's figure only shows it, it states no rule): the RWG of
the edge (lo, hi), lo < hi global vertex ids, has c^+ = the triangle whose
counter-clockwise vertex cycle runs lo -> hi.  Unknowns are numbered by edge in
lexicographic order of (lo, hi).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class RWGMesh:
    V: np.ndarray          # [nv,3] vertices
    T: np.ndarray          # [nt,3] triangles (CCW outward)
    edges: np.ndarray      # [N,2] (lo, hi) vertex ids
    tri_pm: np.ndarray     # [N,2] (c+, c-) triangle ids
    free_pm: np.ndarray    # [N,2] (x+, x-) free vertex ids
    area: np.ndarray       # [nt]
    normal: np.ndarray     # [nt,3] unit normals
    centroid: np.ndarray   # [nt,3]

    @property
    def N(self):
        return self.edges.shape[0]

    @property
    def Nt(self):
        return self.T.shape[0]

    def sigma_dense(self):
        """Star matrix Sigma [N, Nt] (Sec. VI-A)."""
        S = np.zeros((self.N, self.Nt))
        r = np.arange(self.N)
        S[r, self.tri_pm[:, 0]] = 1.0
        S[r, self.tri_pm[:, 1]] = -1.0
        return S

    def sigmaT_apply(self, j):
        """rho = Sigma^T j (charge per triangle), j [N] or [R, N]."""
        j = np.asarray(j)
        jj = np.atleast_2d(j)
        rho = np.zeros((jj.shape[0], self.Nt), dtype=np.result_type(j, np.float64))
        for r in range(jj.shape[0]):
            np.add.at(rho[r], self.tri_pm[:, 0], jj[r])
            np.subtract.at(rho[r], self.tri_pm[:, 1], jj[r])
        return rho[0] if j.ndim == 1 else rho

    def sigma_apply(self, rho):
        """Sigma rho, rho [..., Nt] -> [..., N]."""
        rho = np.asarray(rho)
        return rho[..., self.tri_pm[:, 0]] - rho[..., self.tri_pm[:, 1]]


def build_rwg(V, T) -> RWGMesh:
    V = np.asarray(V, dtype=np.float64)
    T = np.asarray(T, dtype=np.int64)
    nt = T.shape[0]
    a, b, c = V[T[:, 0]], V[T[:, 1]], V[T[:, 2]]
    n = np.cross(b - a, c - a)
    nn = np.linalg.norm(n, axis=1)
    if np.any(nn <= 1e-300):
        raise ValueError("degenerate triangle")
    area = 0.5 * nn
    normal = n / nn[:, None]
    centroid = (a + b + c) / 3.0

    edge_map: dict = {}
    for t in range(nt):
        for k in range(3):
            u, v = int(T[t, k]), int(T[t, (k + 1) % 3])
            w = int(T[t, (k + 2) % 3])
            key = (min(u, v), max(u, v))
            edge_map.setdefault(key, []).append((t, u < v, w))
    keys = sorted(edge_map.keys())
    N = len(keys)
    edges = np.zeros((N, 2), dtype=np.int64)
    tri_pm = np.zeros((N, 2), dtype=np.int64)
    free_pm = np.zeros((N, 2), dtype=np.int64)
    for m, key in enumerate(keys):
        lst = edge_map[key]
        if len(lst) != 2:
            raise ValueError(f"edge {key} is shared by {len(lst)} triangles (mesh not a closed 2-manifold)")
        (t0, fwd0, w0), (t1, fwd1, w1) = lst
        if fwd0 == fwd1:
            raise ValueError(f"inconsistent orientation at edge {key}")
        if fwd0:
            tp, wp, tm, wm = t0, w0, t1, w1
        else:
            tp, wp, tm, wm = t1, w1, t0, w0
        edges[m] = key
        tri_pm[m] = (tp, tm)
        free_pm[m] = (wp, wm)
    return RWGMesh(V=V, T=T, edges=edges, tri_pm=tri_pm, free_pm=free_pm,
                   area=area, normal=normal, centroid=centroid)


def rwg_value(mesh: RWGMesh, m: int, c: int, x):
    """f_m(x) for points x [P,3] lying on triangle c (must be c_m^+ or c_m^-)."""
    x = np.asarray(x, dtype=np.float64)
    if c == mesh.tri_pm[m, 0]:
        return (x - mesh.V[mesh.free_pm[m, 0]]) / (2.0 * mesh.area[c])
    if c == mesh.tri_pm[m, 1]:
        return (mesh.V[mesh.free_pm[m, 1]] - x) / (2.0 * mesh.area[c])
    raise ValueError("triangle not in the support of the RWG")


def current_at(mesh: RWGMesh, j, x_tri, tri_ids):
    """Surface current J(x) = sum_m j_m f_m(x) at points x_tri [P,3] on triangles tri_ids [P]."""
    j = np.asarray(j)
    out = np.zeros((x_tri.shape[0], 3), dtype=np.result_type(j, np.float64))
    for s, col in ((1.0, 0), (-1.0, 1)):
        tri = mesh.tri_pm[:, col]
        free = mesh.V[mesh.free_pm[:, col]]
        # for each point, every RWG whose c^{+/-} is that point's triangle
        order = np.argsort(tri, kind="stable")
        tri_s = tri[order]
        for p in range(x_tri.shape[0]):
            lo = np.searchsorted(tri_s, tri_ids[p], "left")
            hi = np.searchsorted(tri_s, tri_ids[p], "right")
            for m in order[lo:hi]:
                out[p] += j[m] * s * (x_tri[p] - free[m]) / (2.0 * mesh.area[tri_ids[p]])
    return out

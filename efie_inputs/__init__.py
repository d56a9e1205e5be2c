"""Seeded synthetic inputs shared by the tests, the bench and the smoke check.

This module holds only input generators: closed triangle meshes (geodesic
spheres, ellipsoids, thin closed boxes), seeded complex vectors and plane-wave
directions.  It contains none of the fast method's arithmetic, so both the CPU
oracle and the CUDA library may consume its outputs without sharing code.

Every mesh is returned as ``(vertices [nv,3] float64, triangles [nt,3] int32)``
with counter-clockwise vertex order seen from outside (outward normals).
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "icosphere",
    "ellipsoid",
    "thin_box",
    "merge_meshes",
    "complex_gaussian",
    "azimuth_planewaves",
    "mesh_stats",
]


def _icosahedron():
    t = (1.0 + math.sqrt(5.0)) / 2.0
    v = np.array(
        [
            [-1, t, 0], [1, t, 0], [-1, -t, 0], [1, -t, 0],
            [0, -1, t], [0, 1, t], [0, -1, -t], [0, 1, -t],
            [t, 0, -1], [t, 0, 1], [-t, 0, -1], [-t, 0, 1],
        ],
        dtype=np.float64,
    )
    f = np.array(
        [
            [0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
            [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
            [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
            [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1],
        ],
        dtype=np.int64,
    )
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return v, f


def icosphere(freq: int, radius: float = 1.0, center=(0.0, 0.0, 0.0)):
    """Class-I geodesic sphere: every icosahedron face split into freq^2
    triangles, vertices projected onto the sphere.  20 freq^2 triangles,
    10 freq^2 + 2 vertices, 30 freq^2 edges."""
    if freq < 1:
        raise ValueError("freq must be >= 1")
    iv, ifc = _icosahedron()
    key_to_idx: dict = {}
    verts: list = []

    def vid(a, b, c, i, j):
        # point A + i/n (B-A) + j/n (C-A); key on the integer barycentric
        # coordinates relative to the sorted corner ids (shared across faces)
        w = {a: freq - i - j, b: i, c: j}
        key = tuple(sorted((k, val) for k, val in w.items() if val != 0))
        idx = key_to_idx.get(key)
        if idx is None:
            p = (iv[a] * (freq - i - j) + iv[b] * i + iv[c] * j) / freq
            p = p / np.linalg.norm(p)
            idx = len(verts)
            key_to_idx[key] = idx
            verts.append(p)
        return idx

    tris = []
    for a, b, c in ifc:
        for i in range(freq):
            for j in range(freq - i):
                v00 = vid(a, b, c, i, j)
                v10 = vid(a, b, c, i + 1, j)
                v01 = vid(a, b, c, i, j + 1)
                tris.append((v00, v10, v01))
                if i + j + 1 < freq:
                    v11 = vid(a, b, c, i + 1, j + 1)
                    tris.append((v10, v11, v01))
    V = np.array(verts, dtype=np.float64) * float(radius)
    T = np.array(tris, dtype=np.int32)
    T = _orient_outward(V, T)
    V = V + np.asarray(center, dtype=np.float64)
    return V, T


def _orient_outward(V, T):
    """Flip triangles whose normal points towards the centroid of the body
    (valid for the star-shaped bodies generated here)."""
    c0 = V.mean(axis=0)
    a, b, c = V[T[:, 0]], V[T[:, 1]], V[T[:, 2]]
    n = np.cross(b - a, c - a)
    cen = (a + b + c) / 3.0
    flip = np.einsum("ij,ij->i", n, cen - c0) < 0
    T = T.copy()
    T[flip] = T[flip][:, [0, 2, 1]]
    return T


def ellipsoid(freq: int, semi_axes, center=(0.0, 0.0, 0.0)):
    """Geodesic sphere scaled anisotropically to the given semi-axes."""
    V, T = icosphere(freq, 1.0)
    V = V * np.asarray(semi_axes, dtype=np.float64) + np.asarray(center, dtype=np.float64)
    return V, T


def thin_box(size, n_div, center=(0.0, 0.0, 0.0)):
    """Closed box of extents size=(lx,ly,lz) with n_div=(nx,ny,nz) quads per
    edge direction, each quad split into two triangles."""
    lx, ly, lz = (float(s) for s in size)
    nx, ny, nz = (int(n) for n in n_div)
    key_to_idx: dict = {}
    verts: list = []

    def vid(i, j, k):
        key = (i, j, k)
        idx = key_to_idx.get(key)
        if idx is None:
            idx = len(verts)
            key_to_idx[key] = idx
            verts.append((lx * (i / nx - 0.5), ly * (j / ny - 0.5), lz * (k / nz - 0.5)))
        return idx

    tris = []

    def face(fixed_axis, fixed_val, na, nb):
        ax = [d for d in range(3) if d != fixed_axis]
        for a in range(na):
            for b in range(nb):
                q = []
                for da, db in ((0, 0), (1, 0), (1, 1), (0, 1)):
                    idx = [0, 0, 0]
                    idx[fixed_axis] = fixed_val
                    idx[ax[0]] = a + da
                    idx[ax[1]] = b + db
                    q.append(vid(*idx))
                tris.append((q[0], q[1], q[2]))
                tris.append((q[0], q[2], q[3]))

    face(0, 0, ny, nz); face(0, nx, ny, nz)
    face(1, 0, nx, nz); face(1, ny, nx, nz)
    face(2, 0, nx, ny); face(2, nz, nx, ny)
    V = np.array(verts, dtype=np.float64)
    T = np.array(tris, dtype=np.int32)
    T = _orient_outward(V, T)
    return V + np.asarray(center, dtype=np.float64), T


def merge_meshes(*meshes):
    """Disjoint union of closed meshes."""
    Vs, Ts, off = [], [], 0
    for V, T in meshes:
        Vs.append(V)
        Ts.append(T + off)
        off += V.shape[0]
    return np.concatenate(Vs).astype(np.float64), np.concatenate(Ts).astype(np.int32)


def complex_gaussian(shape, seed: int, dtype=np.complex128):
    """Seeded standard complex Gaussian array (independent re/im, unit variance each)."""
    rng = np.random.default_rng(seed)
    z = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    return z.astype(dtype)


def azimuth_planewaves(n_dirs: int, step_deg: float = None):
    """Plane waves with propagation direction in the xy-plane at azimuths
    phi_i = i*step (theta = 90 deg) and theta-hat polarisation (= -z at
    theta = 90 deg).  Returns (khat [n,3], pol [n,3])."""
    if step_deg is None:
        step_deg = 360.0 / n_dirs
    phi = np.deg2rad(step_deg * np.arange(n_dirs))
    # incident from phi: propagation direction -r_hat(theta=90,phi)
    khat = -np.stack([np.cos(phi), np.sin(phi), np.zeros_like(phi)], axis=1)
    pol = np.tile(np.array([0.0, 0.0, -1.0]), (n_dirs, 1))
    return khat, pol


def mesh_stats(V, T):
    a, b, c = V[T[:, 0]], V[T[:, 1]], V[T[:, 2]]
    e = np.concatenate([np.linalg.norm(b - a, axis=1), np.linalg.norm(c - b, axis=1),
                        np.linalg.norm(a - c, axis=1)])
    return {"n_vertices": int(V.shape[0]), "n_triangles": int(T.shape[0]),
            "edge_mean": float(e.mean()), "edge_max": float(e.max()),
            "edge_min": float(e.min())}

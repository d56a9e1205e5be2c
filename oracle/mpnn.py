"""Learned mesh-local preconditioner network, FP64 NumPy reference (oracle;
test infrastructure only).  Not part of the paper: a small message-passing
network that maps a residual r to an approximate error z ~ T^-1 r, used as the
flexible right preconditioner of FGMRES.

Graph: nodes are RWG unknowns; m and n are neighbours when they share a
triangle c, with sign s_mn = sigma_{m,c} sigma_{n,c} (sigma = +1 on c+, -1 on
c-).  On a closed mesh every node has exactly four neighbours.

Network (width 64):
    s   = sqrt(mean |r|^2)                      (output 0 if s == 0)
    x   = [Re r / s, Im r / s, l_m / mean(l), 1]          (l_m edge length)
    h   = tanh(x We^T + be)
    for l = 0..2:
        a  = sum_n s_mn h_n                      (signed neighbour sum)
        h  = tanh(h Ws_l^T + a Wn_l^T + bl_l) + h
    y   = h Wd^T + bd,   z = s (y_0 + j y_1)
Loss of a pair (r, e): |z - e|^2 / |e|^2.

bf16=True rounds every weight matrix and every activation entering a matrix
product to bfloat16 (round to nearest even), as the GPU kernels do; sums stay
in FP64 here (FP32 on the GPU).
"""
from __future__ import annotations

import numpy as np

WIDTH = 64
N_LAYERS = 3
N_IN = 4


def bf16_round(a):
    """Round float64 values to the nearest bfloat16 (ties to even)."""
    a32 = np.asarray(a, dtype=np.float32)
    u = a32.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def build_graph(mesh):
    """Neighbour ids [N,4] and signs [N,4] of the RWG adjacency, edge lengths."""
    N = mesh.N
    tri_rwgs = [[] for _ in range(mesh.Nt)]
    for m in range(N):
        tri_rwgs[mesh.tri_pm[m, 0]].append((m, 1.0))
        tri_rwgs[mesh.tri_pm[m, 1]].append((m, -1.0))
    nbr = np.full((N, 4), -1, dtype=np.int64)
    sgn = np.zeros((N, 4))
    cnt = np.zeros(N, dtype=np.int64)
    for c in range(mesh.Nt):
        lst = tri_rwgs[c]
        for (m, sm) in lst:
            for (n, sn) in lst:
                if n == m:
                    continue
                nbr[m, cnt[m]] = n
                sgn[m, cnt[m]] = sm * sn
                cnt[m] += 1
    V = mesh.V
    length = np.linalg.norm(V[mesh.edges[:, 0]] - V[mesh.edges[:, 1]], axis=1)
    return nbr, sgn, length


def init_params(seed=0, width=WIDTH):
    rng = np.random.default_rng(seed)
    p = {"We": rng.standard_normal((width, N_IN)) / np.sqrt(N_IN), "be": np.zeros(width)}
    for l in range(N_LAYERS):
        p[f"Ws{l}"] = rng.standard_normal((width, width)) * (0.5 / np.sqrt(width))
        p[f"Wn{l}"] = rng.standard_normal((width, width)) * (0.25 / np.sqrt(width))
        p[f"bl{l}"] = np.zeros(width)
    p["Wd"] = rng.standard_normal((2, width)) * (0.1 / np.sqrt(width))
    p["bd"] = np.zeros(2)
    return p


def _aggregate(nbr, sgn, h):
    out = np.zeros_like(h)
    for j in range(nbr.shape[1]):
        ok = nbr[:, j] >= 0
        out[ok] += sgn[ok, j][:, None] * h[nbr[ok, j]]
    return out


def forward(p, graph, r, bf16=False):
    nbr, sgn, length = graph
    q = bf16_round if bf16 else (lambda v: v)
    r = np.asarray(r, dtype=np.complex128)
    s = np.sqrt(np.mean(np.abs(r) ** 2))
    cache = {"s": s}
    if s == 0:
        return np.zeros_like(r), cache
    x = np.stack([r.real / s, r.imag / s, length / length.mean(), np.ones(len(r))], axis=1)
    cache["x"] = x
    u = q(x) @ q(p["We"]).T + p["be"]
    h = np.tanh(u)
    cache["u0"] = u
    hs = [h]
    us, as_ = [], []
    for l in range(N_LAYERS):
        a = _aggregate(nbr, sgn, h)
        u = q(h) @ q(p[f"Ws{l}"]).T + q(a) @ q(p[f"Wn{l}"]).T + p[f"bl{l}"]
        h = np.tanh(u) + h
        us.append(u)
        as_.append(a)
        hs.append(h)
    y = q(h) @ q(p["Wd"]).T + p["bd"]
    cache.update(hs=hs, us=us, as_=as_, y=y)
    return s * (y[:, 0] + 1j * y[:, 1]), cache


def loss(z, e):
    return float(np.sum(np.abs(z - e) ** 2) / np.sum(np.abs(e) ** 2))


def backward(p, graph, cache, z, e, bf16=False):
    """Gradients of loss(z, e) with respect to every parameter (straight-through
    for the bf16 roundings)."""
    nbr, sgn, _ = graph
    q = bf16_round if bf16 else (lambda v: v)
    g = {k: np.zeros_like(v) for k, v in p.items()}
    s = cache["s"]
    if s == 0:
        return g
    E = np.sum(np.abs(e) ** 2)
    dz = 2.0 * (z - e) / E
    dy = s * np.stack([dz.real, dz.imag], axis=1)
    hs, us, as_ = cache["hs"], cache["us"], cache["as_"]
    h = hs[-1]
    g["Wd"] = dy.T @ q(h)
    g["bd"] = dy.sum(axis=0)
    dh = dy @ q(p["Wd"])
    for l in reversed(range(N_LAYERS)):
        h_in, a, u = hs[l], as_[l], us[l]
        du = dh * (1.0 - np.tanh(u) ** 2)
        g[f"Ws{l}"] = du.T @ q(h_in)
        g[f"Wn{l}"] = du.T @ q(a)
        g[f"bl{l}"] = du.sum(axis=0)
        da = du @ q(p[f"Wn{l}"])
        dh = dh + du @ q(p[f"Ws{l}"]) + _aggregate(nbr, sgn, da)
    du0 = dh * (1.0 - np.tanh(cache["u0"]) ** 2)
    g["We"] = du0.T @ q(cache["x"])
    g["be"] = du0.sum(axis=0)
    return g


def flatten(p):
    """Parameter vector in the library's order."""
    keys = ["We", "be"]
    for l in range(N_LAYERS):
        keys += [f"Ws{l}", f"Wn{l}", f"bl{l}"]
    keys += ["Wd", "bd"]
    return np.concatenate([p[k].ravel() for k in keys]), keys


def unflatten(vec, like):
    out, off = {}, 0
    _, keys = flatten(like)
    for k in keys:
        n = like[k].size
        out[k] = vec[off:off + n].reshape(like[k].shape)
        off += n
    return out

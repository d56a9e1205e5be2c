"""Plain restarted GMRES / flexible GMRES in FP64 complex (oracle; test
infrastructure only).  The paper states only that an iterative solver is used
(Sec. II); the paper names GMRES without its details; here GMRES(m), x0 = 0, success when the true relative
residual ||b - T x|| / ||b|| <= tol.  Arnoldi with classical Gram-Schmidt
applied twice (CGS2), Givens rotations for the least-squares problem.
"""
from __future__ import annotations

import numpy as np


def fgmres(matvec, b, tol=1e-6, restart=100, max_iters=1000, precond=None):
    """Solve T x = b.  precond(v) returns an approximation of T^{-1} v (right
    preconditioning, flexible: it may change between iterations).
    Returns (x, info) with info = {iterations, true_rel_residual, converged}."""
    b = np.asarray(b, dtype=np.complex128)
    n = b.shape[0]
    x = np.zeros(n, dtype=np.complex128)
    bnorm = np.linalg.norm(b)
    if bnorm == 0:
        return x, {"iterations": 0, "true_rel_residual": 0.0, "converged": True}
    its = 0
    r = b.copy()
    while True:
        beta = np.linalg.norm(r)
        if beta / bnorm <= tol or its >= max_iters:
            break
        m = restart
        Vb = np.zeros((m + 1, n), dtype=np.complex128)
        Z = np.zeros((m, n), dtype=np.complex128)
        H = np.zeros((m + 1, m), dtype=np.complex128)
        cs = np.zeros(m, dtype=np.complex128)
        sn = np.zeros(m, dtype=np.complex128)
        g = np.zeros(m + 1, dtype=np.complex128)
        g[0] = beta
        Vb[0] = r / beta
        kk = 0
        for kk in range(m):
            z = precond(Vb[kk]) if precond is not None else Vb[kk]
            Z[kk] = z
            w = matvec(z)
            for _ in range(2):                       # CGS2
                h = Vb[:kk + 1].conj() @ w
                w = w - h @ Vb[:kk + 1]
                H[:kk + 1, kk] += h
            H[kk + 1, kk] = np.linalg.norm(w)
            if H[kk + 1, kk] != 0:
                Vb[kk + 1] = w / H[kk + 1, kk]
            # Givens rotations G_i = [[conj(c), conj(s)], [-s, c]], c = a/den,
            # s = b/den, which map (a, b) to (den, 0)
            for i in range(kk):
                t = np.conj(cs[i]) * H[i, kk] + np.conj(sn[i]) * H[i + 1, kk]
                H[i + 1, kk] = -sn[i] * H[i, kk] + cs[i] * H[i + 1, kk]
                H[i, kk] = t
            a, bb = H[kk, kk], H[kk + 1, kk]
            den = np.sqrt(abs(a) ** 2 + abs(bb) ** 2)
            cs[kk] = a / den if den else 1.0
            sn[kk] = bb / den if den else 0.0
            H[kk, kk] = den
            H[kk + 1, kk] = 0.0
            g[kk + 1] = -sn[kk] * g[kk]
            g[kk] = np.conj(cs[kk]) * g[kk]
            its += 1
            if abs(g[kk + 1]) / bnorm <= tol or its >= max_iters:
                break
        kdim = kk + 1
        y = np.linalg.solve(np.triu(H[:kdim, :kdim]), g[:kdim])
        x = x + y @ Z[:kdim]
        r = b - matvec(x)
    rel = np.linalg.norm(b - matvec(x)) / bnorm
    return x, {"iterations": its, "true_rel_residual": float(rel), "converged": bool(rel <= tol)}

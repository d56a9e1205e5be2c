"""Pins of the dense Galerkin EFIE oracle (Sec. II, Sec. VI-A): complex
symmetry, the Mie series (current on a PEC sphere, convergence under mesh
refinement, sign sensitivity), reciprocity of the plane-wave response, the star
null space, and GMRES against a direct solve."""
import numpy as np
import pytest

import efie_inputs as E
from oracle import dense, krylov, mie
from oracle.geometry import build_rwg, current_at


def _mie_error(m, k, T, khat=(0, 0, -1.0), pol=(1.0, 0, 0)):
    e = dense.rhs_planewave(m, k, khat, pol)[0]
    j = np.linalg.solve(T, e)
    Jm = current_at(m, j, m.centroid, np.arange(m.Nt))
    r = np.linalg.norm(m.V, axis=1).mean()
    pts = m.centroid / np.linalg.norm(m.centroid, axis=1, keepdims=True) * r
    Jmie = mie.surface_current(pts, r, k, khat, pol)
    n = m.normal
    Jmie = Jmie - np.sum(Jmie * n, axis=1, keepdims=True) * n
    return np.linalg.norm(Jm - Jmie) / np.linalg.norm(Jmie)


def test_symmetry(c1_dense):
    A, V = c1_dense
    assert np.abs(A - A.T).max() <= 1e-13 * np.abs(A).max()
    assert np.abs(V - V.T).max() <= 1e-13 * np.abs(V).max()


def test_mie_c1_and_sign(c1_mesh, c1_dense):
    _, _, m = c1_mesh
    A, V = c1_dense
    k = 2 * np.pi
    T = dense.efie_matrix(m, k, A, V)
    err = _mie_error(m, k, T)
    assert err < 0.08
    S = m.sigma_dense()
    T_wrong = 1j * k * A - (1.0 / (1j * k)) * (S @ V @ S.T)
    assert _mie_error(m, k, T_wrong) > 0.5


def test_mie_refinement():
    """Current error against Mie falls as the mesh is refined (0.4 lambda
    sphere, so every mesh stays small)."""
    k = 2 * np.pi
    errs = []
    kh = np.array([0.3, -0.2, 0.9]) / np.linalg.norm([0.3, -0.2, 0.9])
    pol = np.array([1.0, 0.4, 0.0])
    pol = pol - (pol @ kh) * kh
    pol /= np.linalg.norm(pol)
    for n in (3, 5, 7):
        V, T = E.icosphere(n, 0.2)
        m = build_rwg(V, T)
        Tm = dense.efie_matrix(m, k)
        errs.append(_mie_error(m, k, Tm, khat=kh, pol=pol))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 0.1


def test_reciprocity():
    """Plane wave A, observed with plane wave B equals the swap:
    e_B^T T^-1 e_A = e_A^T T^-1 e_B for a symmetric T (reciprocity)."""
    V, T = E.icosphere(4, 0.3)
    m = build_rwg(V, T)
    k = 2 * np.pi
    Tm = dense.efie_matrix(m, k)
    eA = dense.rhs_planewave(m, k, (0, 0, 1.0), (1.0, 0, 0))[0]
    eB = dense.rhs_planewave(m, k, (0.6, 0.8, 0), (0, 0, 1.0))[0]
    a = eB @ np.linalg.solve(Tm, eA)
    b = eA @ np.linalg.solve(Tm, eB)
    assert abs(a - b) / abs(a) < 1e-10


def test_star_null_space(c1_mesh, c1_dense):
    """Sec. VI-A: Sigma^T annihilates solenoidal (loop) currents, so the scalar
    part Sigma V Sigma^T x vanishes for x in null(Sigma^T)."""
    _, _, m = c1_mesh
    _, V = c1_dense
    S = m.sigma_dense()
    x = E.complex_gaussian(m.N, 7)
    # project onto null(Sigma^T)
    x = x - S @ np.linalg.lstsq(S, x, rcond=None)[0]
    assert np.linalg.norm(m.sigmaT_apply(x)) < 1e-12 * np.linalg.norm(x)
    yV = m.sigma_apply(V @ m.sigmaT_apply(x))
    assert np.linalg.norm(yV) < 1e-10 * np.abs(V).max() * np.linalg.norm(x)


def test_gmres_vs_direct(c1_mesh, c1_dense):
    _, _, m = c1_mesh
    A, V = c1_dense
    k = 2 * np.pi
    T = dense.efie_matrix(m, k, A, V)
    e = dense.rhs_planewave(m, k, (0, 0, -1.0), (1.0, 0, 0))[0]
    x, info = krylov.fgmres(lambda v: T @ v, e, tol=1e-6, restart=100, max_iters=500)
    assert info["converged"]
    xs = np.linalg.solve(T, e)
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) < 1e-4


def test_rows_dense_matches_full(c1_mesh, c1_dense):
    _, _, m = c1_mesh
    A, V = c1_dense
    k = 2 * np.pi
    rows = np.array([0, 5, 777, 1919])
    x = E.complex_gaussian(m.N, 3)
    yA, yV = dense.rows_dense(m, k, rows, x)
    S = m.sigma_dense()
    assert np.abs(yA[0] - (A @ x)[rows]).max() < 1e-12 * np.abs(A @ x).max()
    assert np.abs(yV[0] - (S @ V @ S.T @ x)[rows]).max() < 1e-12 * np.abs(S @ V @ S.T @ x).max()

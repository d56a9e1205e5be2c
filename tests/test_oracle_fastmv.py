"""Pins of the oracle's B-spline fast matvec: polynomial-kernel exactness of
the whole far pipeline (moments, transfers, stabilization, Toeplitz/FFT
translation, interaction lists, interpolation), FFT vs plain Toeplitz
translation, accuracy against the dense product, star null space and
symmetry of the fast operator."""
import numpy as np
import pytest

import efie_inputs as E
from oracle import dense, fastmv
from oracle.geometry import build_rwg


def _poly_far_check(p, k, radius, freq, delta, levels, n_reg):
    V, T = E.icosphere(freq, radius)
    m = build_rwg(V, T)
    # translation-invariant kernel of degree p: interpolation is exact at every level
    kern = lambda D: (D[..., 0] + 2.0 * D[..., 1] - D[..., 2] + 0.3) ** p + 0j
    # the polynomial kernel is regular, so touching far domains are harmless here
    op = fastmv.BsplineEFIE(m, k, p, delta, levels, kernel=kern, near=None, allow_overlap=True)
    A, Vm = dense.assemble_dense(m, k, kernel=kern, n_reg=n_reg)
    nb, rb, tb = op.near_masks()
    Af = np.where(nb[rb[:, None], rb[None, :]], 0, A)
    Vf = np.where(nb[tb[:, None], tb[None, :]], 0, Vm)
    x = E.complex_gaussian(m.N, 2)
    yA, yV = op.far_parts(x)
    S = m.sigma_dense()
    refA, refV = Af @ x, S @ Vf @ S.T @ x
    return (np.linalg.norm(yA - refA) / np.linalg.norm(refA),
            np.linalg.norm(yV - refV) / np.linalg.norm(refV), op)


@pytest.mark.parametrize("p", [1, 3, 6])
def test_polynomial_kernel_exact_constant_s(p):
    eA, eV, op = _poly_far_check(p, 2 * np.pi, 0.5, 3, 0.06, 2, n_reg=(p + 4) // 2)
    # two grid levels with constant s, transfers in use
    L = op.tree.levels
    assert L[op.tree.D].s == L[op.tree.D - 1].s and len(op.IL[op.tree.D][0]) > 0
    assert eA < 1e-12 and eV < 1e-12


def test_polynomial_kernel_exact_increasing_s():
    # k large enough that the parent box edge >= lambda/2: s -> 2s - p
    p = 3
    eA, eV, op = _poly_far_check(p, 2 * np.pi * 2.5, 0.5, 3, 0.06, 2, n_reg=4)
    L = op.tree.levels
    assert L[op.tree.D - 1].s == 2 * L[op.tree.D].s - p
    assert eA < 1e-12 and eV < 1e-12


def test_fft_equals_toeplitz(c1_oracle):
    x = E.complex_gaussian(c1_oracle.mesh.N, 5)
    c1_oracle.translation = "fft"
    y1 = c1_oracle.matvec(x)
    c1_oracle.translation = "toeplitz"
    y2 = c1_oracle.matvec(x)
    c1_oracle.translation = "fft"
    assert np.linalg.norm(y1 - y2) / np.linalg.norm(y2) < 1e-13


def test_fast_vs_dense_c1(c1_mesh, c1_dense, c1_oracle):
    """Gate: relative l2 of the fast matvec against the dense product <= 1e-3
    (p = 3, s = 7, delta = 0.1 lambda, two levels)."""
    _, _, m = c1_mesh
    A, V = c1_dense
    k = 2 * np.pi
    T = dense.efie_matrix(m, k, A, V)
    for x in (E.complex_gaussian(m.N, 1),
              np.linalg.solve(T, dense.rhs_planewave(m, k, (0, 0, -1.0), (1.0, 0, 0))[0])):
        y = c1_oracle.matvec(x)
        yd = T @ x
        assert np.linalg.norm(y - yd) / np.linalg.norm(yd) < 1e-3


def test_fast_star_null_space(c1_oracle):
    m = c1_oracle.mesh
    S = m.sigma_dense()
    x = E.complex_gaussian(m.N, 9)
    x = x - S @ np.linalg.lstsq(S, x, rcond=None)[0]
    yA, yV = c1_oracle.matvec_parts(x)
    assert np.linalg.norm(yV) < 1e-9 * np.linalg.norm(yA)


def test_fast_operator_symmetric(c1_oracle):
    m = c1_oracle.mesh
    x = E.complex_gaussian(m.N, 11)
    y = E.complex_gaussian(m.N, 12)
    a = y @ c1_oracle.matvec(x)
    b = x @ c1_oracle.matvec(y)
    assert abs(a - b) / abs(a) < 1e-12


def test_error_falls_with_p(c1_mesh, c1_dense):
    """Sec. VII-A, Eq. errorapprox: the far error falls with p (s - p = 4 fixed)."""
    _, _, m = c1_mesh
    A, Vm = c1_dense
    k = 2 * np.pi
    Td = dense.efie_matrix(m, k, A, Vm)
    x = E.complex_gaussian(m.N, 4)
    yd = Td @ x
    errs = []
    for p in (1, 3, 5):
        op = fastmv.BsplineEFIE(m, k, p, 0.1, 1, dense_AV=(A, Vm))
        assert len(op.IL[op.tree.D][0]) > 0
        errs.append(np.linalg.norm(op.matvec(x) - yd) / np.linalg.norm(yd))
    assert errs[1] < errs[0] / 3
    assert errs[2] < errs[1]


def test_overlapping_domains_rejected():
    V, T = E.icosphere(5, 0.5)
    m = build_rwg(V, T)
    with pytest.raises(ValueError):
        fastmv.BsplineEFIE(m, 2 * np.pi, 3, 0.08, 1, near=None)

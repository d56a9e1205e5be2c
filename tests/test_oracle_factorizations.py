"""Pins of the oracle's direct and dyadic factorizations
(`oracle.factorizations`, Sec. VI): polynomial-kernel exactness of the far
part against the dense far product with the same kernel (for the dyadic form
this checks the Hessian translation against the divergence form, since
int int f_m . grad grad kappa . f_n = -Phi_mn), for constant s and for
s -> 2s - p; accuracy against the dense Helmholtz product; symmetry; and
agreement with the star-based factorization of `oracle.fastmv`."""
import numpy as np
import pytest

import efie_inputs as E
from oracle import dense
from oracle import factorizations as F
from oracle.geometry import build_rwg

P = 3
A_VEC = np.array([1.0, 2.0, -1.0])


def _kern(D):
    return (D[..., 0] + 2.0 * D[..., 1] - D[..., 2] + 0.3) ** P + 0j


def _hess(D):
    u = D[..., 0] + 2.0 * D[..., 1] - D[..., 2] + 0.3
    return (P * (P - 1) * u ** (P - 2))[..., None, None] * np.outer(A_VEC, A_VEC) + 0j


@pytest.mark.parametrize("k", [2 * np.pi, 2 * np.pi * 2.5])
def test_polynomial_kernel_exact(k):
    V, T = E.icosphere(3, 0.5)
    m = build_rwg(V, T)
    A, Vm = dense.assemble_dense(m, k, kernel=_kern, n_reg=(P + 4) // 2)
    S = m.sigma_dense()
    Phi = S @ Vm @ S.T
    x = E.complex_gaussian(m.N, 2)
    for cls, extra in ((F.DirectBsplineEFIE, {}), (F.DyadicBsplineEFIE, {"kernel_hessian": _hess})):
        op = cls(m, k, P, 0.06, 2, kernel=_kern, near=None, allow_overlap=True, **extra)
        if k > 2 * np.pi:
            assert op.tree.levels[op.tree.D - 1].s == 2 * op.tree.levels[op.tree.D].s - P
        assert len(op.IL[op.tree.D][0]) > 0
        nb, rb, _ = op.near_masks()
        mask = nb[rb[:, None], rb[None, :]]
        yA, yV = op.far_parts(x)
        rA, rV = np.where(mask, 0, A) @ x, np.where(mask, 0, Phi) @ x
        assert np.linalg.norm(yA - rA) / np.linalg.norm(rA) < 1e-12, cls.__name__
        assert np.linalg.norm(yV - rV) / np.linalg.norm(rV) < 1e-12, cls.__name__


@pytest.mark.parametrize("p", [2, 5])
def test_polynomial_kernel_exact_other_degrees(p):
    """The same exactness for p = 2 (Table I: no knots removed) and p = 5 (two
    removed per side), with a kernel of degree p and its Hessian; the dense
    reference on a regular rule exact for the degree-p kernel."""
    def kern(D):
        return (D[..., 0] + 2.0 * D[..., 1] - D[..., 2] + 0.3) ** p + 0j

    def hess(D):
        u = D[..., 0] + 2.0 * D[..., 1] - D[..., 2] + 0.3
        return (p * (p - 1) * u ** (p - 2))[..., None, None] * np.outer(A_VEC, A_VEC) + 0j

    V, T = E.icosphere(3, 0.5)
    m = build_rwg(V, T)
    A, Vm = dense.assemble_dense(m, 2 * np.pi, kernel=kern, n_reg=(p + 4) // 2 + 1)
    S = m.sigma_dense()
    Phi = S @ Vm @ S.T
    x = E.complex_gaussian(m.N, 20 + p)
    for cls, extra in ((F.DirectBsplineEFIE, {}), (F.DyadicBsplineEFIE, {"kernel_hessian": hess})):
        op = cls(m, 2 * np.pi, p, 0.06, 2, kernel=kern, near=None, allow_overlap=True, **extra)
        assert len(op.IL[op.tree.D][0]) > 0
        nb, rb, _ = op.near_masks()
        mask = nb[rb[:, None], rb[None, :]]
        yA, yV = op.far_parts(x)
        rA, rV = np.where(mask, 0, A) @ x, np.where(mask, 0, Phi) @ x
        assert np.linalg.norm(yA - rA) / np.linalg.norm(rA) < 1e-11, (cls.__name__, p)
        assert np.linalg.norm(yV - rV) / np.linalg.norm(rV) < 1e-11, (cls.__name__, p)


def test_green_hessian_finite_difference():
    k = 2 * np.pi
    rng = np.random.default_rng(1)
    D = rng.normal(size=(5, 3)) + np.array([1.0, 0.0, 0.0])
    H = F.green_hessian(D, k)
    h = 1e-4
    g = lambda X: dense.green(np.sqrt(np.sum(X * X, axis=-1)), k)
    for i in range(3):
        for j in range(3):
            ei, ej = np.eye(3)[i] * h, np.eye(3)[j] * h
            fd = (g(D + ei + ej) - g(D + ei - ej) - g(D - ei + ej) + g(D - ei - ej)) / (4 * h * h)
            assert np.max(np.abs(fd - H[:, i, j])) < 1e-5 * np.max(np.abs(H))


@pytest.fixture(scope="module")
def c1_forms(c1_mesh, c1_dense):
    _, _, m = c1_mesh
    k = 2 * np.pi
    return (F.DirectBsplineEFIE(m, k, P, 0.1, 2, dense_AV=c1_dense),
            F.DyadicBsplineEFIE(m, k, P, 0.1, 2, dense_AV=c1_dense))


def test_fast_vs_dense_c1(c1_mesh, c1_dense, c1_oracle, c1_forms):
    _, _, m = c1_mesh
    k = 2 * np.pi
    T = dense.efie_matrix(m, k, *c1_dense)
    x = E.complex_gaussian(m.N, 11)
    yd = T @ x
    ys = c1_oracle.matvec(x)
    for op in c1_forms:
        y = op.matvec(x)
        assert np.linalg.norm(y - yd) / np.linalg.norm(yd) < 1e-3, type(op).__name__
        assert np.linalg.norm(y - ys) / np.linalg.norm(ys) < 1e-3, type(op).__name__


def test_symmetric(c1_mesh, c1_forms):
    _, _, m = c1_mesh
    x1, x2 = E.complex_gaussian(m.N, 12), E.complex_gaussian(m.N, 13)
    for op in c1_forms:
        a, b = x2 @ op.matvec(x1), x1 @ op.matvec(x2)
        assert abs(a - b) / abs(a) < 1e-12, type(op).__name__


def test_adaptive_forms_uniform_limit(c1_mesh, c1_oracle):
    """The direct and dyadic forms on the nonuniform octree, with every box
    subdivided down to the uniform tree's depth (same root), reproduce the
    uniform-tree forms to rounding (far parts; near parts share the code)."""
    _, _, m = c1_mesh
    tr = c1_oracle.tree
    x = E.complex_gaussian(m.N, 40)
    lim = dict(max_elems=-1, max_prot=np.inf, top=tr.top, root=(tr.root_lo, tr.root_edge), max_depth=tr.D,
               near=None)
    for uni, ada in ((F.DirectBsplineEFIE, F.AdaptiveDirectBsplineEFIE),
                     (F.DyadicBsplineEFIE, F.AdaptiveDyadicBsplineEFIE)):
        u = uni(m, 2 * np.pi, P, 0.1, 2, near=None)
        a = ada(m, 2 * np.pi, P, **lim)
        assert a.tree.D == tr.D and all(a.tree.is_leaf[tr.D])
        for yu, ya in zip(u.far_parts(x), a.far_parts(x)):
            assert np.linalg.norm(ya - yu) / np.linalg.norm(yu) < 1e-12, ada.__name__


def test_adaptive_forms_polynomial_kernel_exact():
    """Far exactness of the direct and dyadic forms on a nonuniform tree with
    leaves on three levels (a fine small sphere beside a coarse large one):
    with a degree-p polynomial kernel (and its Hessian) the far parts equal
    the dense far rows, A masked and Phi = Sigma V Sigma^T masked by the RWG
    pairs of non-near leaves (the dyadic scalar part -H x equals Phi x by
    integration by parts)."""
    from oracle.geometry import build_rwg
    k = 2 * np.pi
    m = build_rwg(*E.merge_meshes(E.icosphere(8, 0.3, center=(-1.0, 0.0, 0.0)),
                                  E.icosphere(5, 0.8, center=(1.0, 0.1, 0.05))))
    x = E.complex_gaussian(m.N, 41)
    rows = np.random.default_rng(42).choice(m.N, 6, replace=False)
    quad = dict(n_reg=(P + 4) // 2 + 1)
    S = m.sigma_dense()
    tri, _, _ = dense.rwg_sides(m)
    for cls, extra in ((F.AdaptiveDirectBsplineEFIE, {}), (F.AdaptiveDyadicBsplineEFIE, {"kernel_hessian": _hess})):
        op = cls(m, k, P, max_elems=30, top=2, kernel=_kern, near=None, allow_overlap=True, **extra)
        assert sum(op.tree.is_leaf[ell].any() for ell in op.grid_levels) == 3
        nb, rl, _ = op.near_masks()
        yA, yV = op.far_parts(x)
        far = [~nb[rl[mm], rl] for mm in rows]
        Xm = np.stack([x * f for f in far])
        rA = np.diagonal(dense.rows_dense(m, k, rows, Xm, kernel=_kern, **quad)[0])
        rV = np.zeros(len(rows), dtype=np.complex128)
        for i, mm in enumerate(rows):
            # row mm of Sigma V Sigma^T: its two triangles' rows of V, then Sigma^T
            vrow = np.zeros(m.Nt, dtype=np.complex128)
            for s in range(2):
                c = tri[mm, s]
                I0, _ = dense.pair_integrals(m, np.full(m.Nt, c), np.arange(m.Nt), k, kernel=_kern, **quad)
                vrow += S[mm, c] * I0 / (m.area[c] * m.area)
            rV[i] = (vrow @ S.T) @ (x * far[i])
        assert np.linalg.norm(yA[rows] - rA) / np.linalg.norm(rA) < 1e-11, cls.__name__
        assert np.linalg.norm(yV[rows] - rV) / np.linalg.norm(rV) < 1e-11, cls.__name__

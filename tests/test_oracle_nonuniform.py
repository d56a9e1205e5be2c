"""Pins of the oracle's nonuniform-octree variant (`oracle.nonuniform`):
  * uniform limit: with every box subdivided to one depth it reproduces the
    uniform oracle (`oracle.fastmv`) to rounding;
  * partition: on a tree with leaves on two levels, every pair of functions is
    either near or translated on exactly one level;
  * polynomial-kernel exactness of the far part (sampled rows against the
    exact far rows of the dense product with the same kernel), for constant s
    and for s -> 2s - p;
  * accuracy against the dense Helmholtz product on sampled rows (<= 1e-3)."""
import numpy as np
import pytest

import efie_inputs as E
from oracle import dense
from oracle import nonuniform as NU
from oracle.geometry import build_rwg

P = 3


def _kern(D):
    return (D[..., 0] + 2.0 * D[..., 1] - D[..., 2] + 0.3) ** P + 0j


@pytest.fixture(scope="module")
def nu_mesh():
    V, T = E.icosphere(14, 0.5)
    return build_rwg(V, T)


@pytest.fixture(scope="module")
def nu_op(nu_mesh):
    # leaves on levels 2 and 3 (boxes with <= 60 triangles, or whose functions
    # would protrude more than 25% from a child box, stay leaves)
    return NU.AdaptiveBsplineEFIE(nu_mesh, 2 * np.pi, P, max_elems=60, top=2, near=None)


def _split_rows(mesh, op, k, rows, x, kernel, want_far, **quad):
    """Exact (far or near) part of (T x)[rows] for the op's block partition:
    (yA, yV) with the A part summed over the far (near) RWG columns of each row
    and the V part over the far (near) triangles of each test triangle.  quad:
    the dense reference's quadrature orders (n_reg high enough that a
    polynomial kernel is integrated exactly)."""
    nb, rl, tl = op.near_masks()
    Xm = np.stack([x * (nb[rl[m], rl] != want_far) for m in rows])
    yA = np.diagonal(dense.rows_dense(mesh, k, rows, Xm, kernel=kernel, **quad)[0]).copy()
    tri, _, _ = dense.rwg_sides(mesh)
    rho = mesh.sigmaT_apply(x)
    yV = np.zeros(len(rows), dtype=np.complex128)
    for i, m in enumerate(rows):
        for s, sgn in ((0, 1.0), (1, -1.0)):
            c = tri[m, s]
            I0, _ = dense.pair_integrals(mesh, np.full(mesh.Nt, c), np.arange(mesh.Nt), k, kernel=kernel, **quad)
            keep = nb[tl[c], tl] != want_far
            yV[i] += sgn * np.sum(np.where(keep, I0 / (mesh.area[c] * mesh.area) * rho, 0.0))
    return yA, yV


def test_uniform_limit(c1_mesh, c1_dense, c1_oracle):
    _, _, m = c1_mesh
    tr = c1_oracle.tree
    op = NU.AdaptiveBsplineEFIE(m, 2 * np.pi, P, max_elems=-1, max_prot=np.inf, top=tr.top,
                                root=(tr.root_lo, tr.root_edge), max_depth=tr.D, dense_AV=c1_dense)
    assert op.tree.D == tr.D and all(op.tree.is_leaf[tr.D])
    for ell in c1_oracle.grid_levels:
        a, b = op.tree.levels[ell], tr.levels[ell]
        assert (a.s, a.sb, a.sp, a.shat) == (b.s, b.sb, b.sp, b.shat) and np.array_equal(a.ijk, b.ijk)
        assert np.isclose(a.delta, b.delta, rtol=1e-15)
    x = E.complex_gaussian(m.N, 4)
    y0, y1 = c1_oracle.matvec(x), op.matvec(x)
    assert np.linalg.norm(y1 - y0) / np.linalg.norm(y0) < 1e-12


def test_partition_exactly_once(nu_op):
    t = nu_op.tree
    assert t.D == 3 and t.is_leaf[2].any() and not t.is_leaf[2].all() and t.is_leaf[3].all()
    nb, rl, tl = nu_op.near_masks()
    for kind, lf in (("rwg", rl), ("tri", tl)):
        cov = NU.far_coverage(nu_op, kind) + nb[lf[:, None], lf[None, :]]
        assert cov.min() == 1 and cov.max() == 1, kind
    # near leaves of different levels exist (a level-2 leaf next to level-3 leaves)
    lvl = NU.leaf_index(t)[0]
    assert (nb & (lvl[:, None] != lvl[None, :])).any()


@pytest.mark.parametrize("k", [2 * np.pi, 2 * np.pi * 2.5])
def test_polynomial_kernel_exact(nu_mesh, nu_op, k):
    m = nu_mesh
    if k == 2 * np.pi:
        op = nu_op
        op.kernel = _kern
    else:
        # level-2 boxes (0.25) at least lambda/2 (0.2): s -> 2s - p there
        op = NU.AdaptiveBsplineEFIE(m, k, P, max_elems=60, top=2, kernel=_kern, near=None, allow_overlap=True)
        assert op.tree.levels[2].s == 2 * op.tree.levels[3].s - P
    try:
        x = E.complex_gaussian(m.N, 6)
        rows = np.random.default_rng(3).choice(m.N, 12, replace=False)
        yA, yV = op.far_parts(x)
        rA, rV = _split_rows(m, op, k, rows, x, _kern, want_far=True)
        assert np.linalg.norm(yA[rows] - rA) / np.linalg.norm(rA) < 1e-11
        assert np.linalg.norm(yV[rows] - rV) / np.linalg.norm(rV) < 1e-11
    finally:
        nu_op.kernel = None


def test_fast_vs_dense_rows(nu_mesh, nu_op):
    m, k = nu_mesh, 2 * np.pi
    x = E.complex_gaussian(m.N, 8)
    rows = np.random.default_rng(5).choice(m.N, 12, replace=False)
    fA, fV = nu_op.far_parts(x)
    nA, nV = _split_rows(m, nu_op, k, rows, x, None, want_far=False)
    y_fast = 1j * k * (fA[rows] + nA) + (fV[rows] + nV) / (1j * k)
    dA, dV = dense.rows_dense(m, k, rows, x)
    y_dense = 1j * k * dA[0] + dV[0] / (1j * k)
    assert np.linalg.norm(y_fast - y_dense) / np.linalg.norm(y_dense) < 1e-3


@pytest.mark.parametrize("p", [1, 5])
def test_polynomial_kernel_exact_other_degrees(p):
    """The same exactness for p = 1 (Table I: no knots removed) and p = 5 (two
    removed per side), with a kernel of degree p, on a tree with leaves on three
    levels (a fine small sphere beside a coarse large one)."""
    k = 2 * np.pi
    m = build_rwg(*E.merge_meshes(E.icosphere(8, 0.3, center=(-1.0, 0.0, 0.0)),
                                  E.icosphere(5, 0.8, center=(1.0, 0.1, 0.05))))

    def kern(D):
        return (D[..., 0] + 2.0 * D[..., 1] - D[..., 2] + 0.3) ** p + 0j

    op = NU.AdaptiveBsplineEFIE(m, k, p, max_elems=30, top=2, kernel=kern, near=None, allow_overlap=True)
    assert sum(op.tree.is_leaf[ell].any() for ell in op.grid_levels) >= 2
    x = E.complex_gaussian(m.N, 16 + p)
    rows = np.random.default_rng(30 + p).choice(m.N, 6, replace=False)
    yA, yV = op.far_parts(x)
    # a regular rule exact for the degree-p kernel times the linear basis functions
    rA, rV = _split_rows(m, op, k, rows, x, kern, want_far=True, n_reg=(p + 4) // 2 + 1)
    assert np.linalg.norm(yA[rows] - rA) / np.linalg.norm(rA) < 1e-11
    assert np.linalg.norm(yV[rows] - rV) / np.linalg.norm(rV) < 1e-11

"""GPU parity of the direct factorization (Sec. VI-B; efie_options
factorization = EFIE_FACT_DIRECT): the scalar part is anterpolated from the
divergence moments of every RWG in its own leaf box, and one near set of RWG
pairs holds A and Phi = Sigma V Sigma^T.  The CUDA path through the C ABI
against the oracle's direct form (`oracle.factorizations.DirectBsplineEFIE`)
on the same seeded inputs, element by element:

* the C1 sphere (1,920 RWG, 2 levels), both precisions, 19 vectors (mixed:
  one pair of 8-vector chunks through the tensor-core pass, then a partial
  chunk), and the (A x, Phi x) split of efie_matvec_parts;
* the three-level, two-doubling tree (s' = 9, 13, 21), mixed form;
* a solve: the direct form converges to the FP64 true residual, and its
  solution is the one of the oracle's direct operator within the tolerance.

Bounds as in the star-form tests: the FP64 form follows the oracle's
arithmetic (gate 1e-10), the mixed form has a complex FP32 far field (1e-5);
against the dense product the fast-matvec accuracy bound 1e-3."""
import numpy as np
import pytest

import efie_inputs as E

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
TOL32 = 1e-5


def _torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.fixture(scope="module")
def G():
    _torch()
    import __graft_entry__ as g
    g.build()
    import paper_2606_13482_gb300 as G
    return G


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def c1_direct(c1_mesh, c1_dense):
    from oracle.factorizations import DirectBsplineEFIE
    _, _, m = c1_mesh
    return DirectBsplineEFIE(m, 2 * np.pi, 3, 0.1, 2, dense_AV=c1_dense)


def test_direct_c1_both_precisions(G, c1_mesh, c1_dense, c1_direct):
    torch = _torch()
    V, T, m = c1_mesh
    k = 2 * np.pi
    X = E.complex_gaussian((19, m.N), 91)
    ref = np.stack([c1_direct.matvec(X[r]) for r in (0, 8, 15, 18)])
    dense_T = 1j * k * c1_dense[0] + (1.0 / (1j * k)) * (m.sigma_dense() @ c1_dense[1] @ m.sigma_dense().T)
    for prec, tol in ((G.EFIE_FP64, TOL64), (G.EFIE_MIXED, TOL32)):
        h = G.EFIE(V, T, k, 3, 0.1, 2, precision=prec, factorization=G.EFIE_FACT_DIRECT)
        try:
            info = h.info()
            assert info["near_nnz_V"] == info["near_nnz_A"]
            Xd = torch.from_numpy(X).cuda()
            Y = h.matvec(Xd).cpu().numpy()
            yA, yV = h.matvec_parts(Xd[:2])
            yA, yV = yA.cpu().numpy(), yV.cpu().numpy()
        finally:
            h.close()
        for i, r in enumerate((0, 8, 15, 18)):
            rel = _rel(Y[r], ref[i])
            mx = float(np.abs(Y[r] - ref[i]).max() / np.abs(ref[i]).max())
            print(f"direct C1 precision {prec} rhs {r}: rel l2 {rel:.3e}, max-abs {mx:.3e}")
            assert rel < tol and mx < 10 * tol, (prec, r, rel, mx)
        # the split: A x and Phi x against the oracle's parts
        rA, rV = c1_direct.matvec_parts(X[1])
        assert _rel(yA[1], rA) < tol and _rel(yV[1], rV) < tol
        # the fast-matvec accuracy against the dense Galerkin product
        assert _rel(Y[0], dense_T @ X[0]) < 1e-3


def test_direct_two_doublings(G):
    """3,840 RWG, grids of 0.4, 0.8 and 1.6 wavelengths (s' = 9, 13, 21, top
    FFT length 37), 16 vectors in the mixed form (one chunk pair on the
    tensor cores on every level), against the oracle's direct form."""
    torch = _torch()
    from oracle.factorizations import DirectBsplineEFIE
    from oracle.geometry import build_rwg
    A = E.icosphere(8, 0.6, center=(-2.1, 0.0, 0.0))
    B = E.icosphere(8, 0.6, center=(2.1, 0.3, 0.1))
    V, T = E.merge_meshes(A, B)
    k, p, delta, levels = 2 * np.pi, 3, 0.1, 3
    ref_op = DirectBsplineEFIE(build_rwg(V, T), k, p, delta, levels)
    X = E.complex_gaussian((16, ref_op.mesh.N), 92)
    h = G.EFIE(V, T, k, p, delta, levels, precision=G.EFIE_MIXED, factorization=G.EFIE_FACT_DIRECT)
    try:
        Y = h.matvec(torch.from_numpy(X).cuda()).cpu().numpy()
    finally:
        h.close()
    for r in (0, 7, 8, 15):
        rel = _rel(Y[r], ref_op.matvec(X[r]))
        print(f"direct two doublings rhs {r}: rel l2 {rel:.3e}")
        assert rel < TOL32, (r, rel)


def test_direct_solve(G, c1_mesh, c1_direct):
    """GMRES on the direct form (mixed handle, FP64 true residual): converges
    to 1e-6, and the solution solves the oracle's direct operator to the same
    residual (up to the mixed form's far-field rounding)."""
    torch = _torch()
    V, T, m = c1_mesh
    k = 2 * np.pi
    h = G.EFIE(V, T, k, 3, 0.1, 2, precision=G.EFIE_MIXED, factorization=G.EFIE_FACT_DIRECT, gmres_restart=100)
    try:
        b = h.rhs_planewave([0, 0, -1.0], [1.0, 0, 0])
        x, info, rc = h.solve(b, tol=1e-6)
        assert rc == 0 and info[0]["converged"] and info[0]["true_rel_residual"] <= 1e-6
        xh = x.cpu().numpy()[0]
        bh = b.cpu().numpy()[0]
    finally:
        h.close()
    res = _rel(c1_direct.matvec(xh), bh)
    print(f"direct solve: oracle residual {res:.3e}")
    assert res < 2e-6

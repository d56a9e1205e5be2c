"""GPU parity of the dyadic factorization (Sec. VI-C; efie_options
factorization = EFIE_FACT_DYADIC): the three RWG moment components are
translated with g and with the six entries of its Hessian d_a d_b g, whose
interpolation gives -int int f_m . grad grad g . f_n (the scalar part, equal to
Phi_mn per pair in the continuum); the near field is the direct form's (A and
Phi on RWG pairs).  The CUDA path through the C ABI against the oracle's
dyadic form (`oracle.factorizations.DyadicBsplineEFIE`) on the same seeded
inputs, element by element:

* the C1 sphere (1,920 RWG, 2 levels), both precisions, with the
  (A x, -H x) split of efie_matvec_parts, and the fast-matvec accuracy against
  the dense Galerkin product;
* a constant-s tree (Sec. IV-C: 3,000 RWG, k = pi, three levels, far pairs on
  two), so that the Hessian grids take the downward transfers as well.

Gates as for the other factorizations: 1e-10 for the FP64 form, 1e-5 for the
mixed form, 1e-3 against the dense product."""
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


def test_dyadic_c1_both_precisions(G, c1_mesh, c1_dense):
    torch = _torch()
    from oracle.factorizations import DyadicBsplineEFIE
    V, T, m = c1_mesh
    k = 2 * np.pi
    ref_op = DyadicBsplineEFIE(m, k, 3, 0.1, 2, dense_AV=c1_dense)
    X = E.complex_gaussian((9, m.N), 93)
    ref = np.stack([ref_op.matvec(X[r]) for r in (0, 4, 8)])
    S = m.sigma_dense()
    dense_T = 1j * k * c1_dense[0] + (1.0 / (1j * k)) * (S @ c1_dense[1] @ S.T)
    for prec, tol in ((G.EFIE_FP64, TOL64), (G.EFIE_MIXED, TOL32)):
        h = G.EFIE(V, T, k, 3, 0.1, 2, precision=prec, factorization=G.EFIE_FACT_DYADIC)
        try:
            Xd = torch.from_numpy(X).cuda()
            Y = h.matvec(Xd).cpu().numpy()
            yA, yV = [t.cpu().numpy() for t in h.matvec_parts(Xd[:2])]
        finally:
            h.close()
        for i, r in enumerate((0, 4, 8)):
            rel = _rel(Y[r], ref[i])
            mx = float(np.abs(Y[r] - ref[i]).max() / np.abs(ref[i]).max())
            print(f"dyadic C1 precision {prec} rhs {r}: rel l2 {rel:.3e}, max-abs {mx:.3e}")
            assert rel < tol and mx < 10 * tol, (prec, r, rel, mx)
        rA, rV = ref_op.matvec_parts(X[1])
        assert _rel(yA[1], rA) < tol and _rel(yV[1], rV) < tol, (_rel(yA[1], rA), _rel(yV[1], rV))
        assert _rel(Y[0], dense_T @ X[0]) < 1e-3


def test_dyadic_constant_s_tree(G):
    torch = _torch()
    from oracle.factorizations import DyadicBsplineEFIE
    from oracle.geometry import build_rwg
    V, T = E.icosphere(10, 0.5)
    k, p, delta, levels = np.pi, 3, 0.06, 3
    info, lv = G.plan(V, T, k, p, delta, levels)
    assert sum(L["n_far_pairs"] > 0 for L in lv) >= 2
    ref_op = DyadicBsplineEFIE(build_rwg(V, T), k, p, delta, levels)
    X = E.complex_gaussian((2, ref_op.mesh.N), 94)
    for prec, tol in ((G.EFIE_FP64, TOL64), (G.EFIE_MIXED, TOL32)):
        h = G.EFIE(V, T, k, p, delta, levels, precision=prec, factorization=G.EFIE_FACT_DYADIC)
        try:
            Y = h.matvec(torch.from_numpy(X).cuda()).cpu().numpy()
        finally:
            h.close()
        for r in range(2):
            rel = _rel(Y[r], ref_op.matvec(X[r]))
            print(f"dyadic constant-s precision {prec} rhs {r}: rel l2 {rel:.3e}")
            assert rel < tol, (prec, r, rel)

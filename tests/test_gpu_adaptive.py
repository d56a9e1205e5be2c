"""GPU parity of the nonuniform octree (Sec. VII tree rule; efie_setup_adaptive):
the CUDA path through the C ABI against the oracle's nonuniform operator
(`oracle.nonuniform.AdaptiveBsplineEFIE`) on the same seeded inputs, element
by element.

The mesh is a fine small sphere (1,280 triangles, radius 0.3 wavelength) beside
a coarse large one (500 triangles, radius 0.8): with at most 30 triangles per
box the tree has leaves on levels 2, 3 and 4 (s' = 15, 9, 9), far pairs on all
three levels, parents on level 2 next to leaves of the same level, and near
blocks between leaves of different levels.

* both precisions: 19 vectors (the mixed form runs one pair of 8-vector chunks
  on the tensor-core path, then a partial chunk), and the (A x, V x) split;
* a bounded GMRES run (mixed handle, FP64 true residual): the residual the
  library reports for its iterate is the oracle's residual of that iterate.

Gates as for the uniform tree: 1e-10 for the FP64 form (same arithmetic as
the oracle up to rounding order), 1e-5 for the mixed form (complex FP32 far
field)."""
import numpy as np
import pytest

import efie_inputs as E

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
TOL32 = 1e-5
TREE = dict(max_elems=30, max_prot=0.25, top=2)


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
def two_spheres():
    from oracle import nonuniform as NU
    from oracle.geometry import build_rwg
    V, T = E.merge_meshes(E.icosphere(8, 0.3, center=(-1.0, 0.0, 0.0)),
                          E.icosphere(5, 0.8, center=(1.0, 0.1, 0.05)))
    k = 2 * np.pi
    op = NU.AdaptiveBsplineEFIE(build_rwg(V, T), k, 3, **TREE)
    return V, T, k, op


def test_adaptive_tree_shape(G, two_spheres):
    V, T, k, op = two_spheres
    lv, _, _ = G.plan_adaptive(V, T, k, 3, **TREE)
    assert [L["level"] for L in lv] == [2, 3, 4]
    assert all(L["n_leaves"] > 0 and L["n_far_pairs"] > 0 for L in lv)
    assert any(L["n_leaves"] < L["n_boxes"] for L in lv)


def test_adaptive_both_precisions(G, two_spheres):
    torch = _torch()
    V, T, k, op = two_spheres
    X = E.complex_gaussian((19, op.mesh.N), 95)
    cols = (0, 8, 15, 18)
    ref = {r: op.matvec(X[r]) for r in cols}
    rA, rV = op.matvec_parts(X[1])
    for prec, tol in ((G.EFIE_FP64, TOL64), (G.EFIE_MIXED, TOL32)):
        h = G.EFIE(V, T, k, 3, 0.0, 0, precision=prec, tree=TREE)
        try:
            info = h.info()
            assert info["n_unknowns"] == op.mesh.N
            Xd = torch.from_numpy(X).cuda()
            Y = h.matvec(Xd).cpu().numpy()
            yA, yV = [t.cpu().numpy() for t in h.matvec_parts(Xd[:2])]
        finally:
            h.close()
        for r in cols:
            rel = _rel(Y[r], ref[r])
            mx = float(np.abs(Y[r] - ref[r]).max() / np.abs(ref[r]).max())
            print(f"adaptive precision {prec} rhs {r}: rel l2 {rel:.3e}, max-abs {mx:.3e}")
            assert rel < tol and mx < 10 * tol, (prec, r, rel, mx)
        ea, ev = _rel(yA[1], rA), _rel(yV[1], rV)
        print(f"adaptive precision {prec} parts: A {ea:.3e}, V {ev:.3e}")
        assert ea < tol and ev < tol, (prec, ea, ev)


def test_adaptive_solve(G, two_spheres):
    """GMRES on the adaptive handle (mixed form, FP64 true residual).  The
    finely meshed 0.3-wavelength sphere makes this EFIE system slow to
    converge (1,000 iterations of GMRES(100) stay above 1e-6), so a bounded
    run is checked instead: it makes progress, and the true residual the
    library reports for its iterate is the oracle's residual of that iterate."""
    torch = _torch()
    V, T, k, op = two_spheres
    h = G.EFIE(V, T, k, 3, 0.0, 0, precision=G.EFIE_MIXED, tree=TREE, gmres_restart=100, max_iters=300)
    try:
        b = h.rhs_planewave([0, 0, -1.0], [1.0, 0, 0])
        x, info, rc = h.solve(b, tol=1e-6)
        xh, bh = x.cpu().numpy()[0], b.cpu().numpy()[0]
    finally:
        h.close()
    lib_res = info[0]["true_rel_residual"]
    res = _rel(op.matvec(xh), bh)
    print(f"adaptive solve: rc {rc}, {info[0]['iterations']} iterations, library residual {lib_res:.3e}, "
          f"oracle residual {res:.3e}")
    assert rc in (0, 1) and lib_res < 1e-1
    assert abs(res - lib_res) <= 1e-6 * lib_res + 1e-12
    if rc == 0:
        assert lib_res <= 1e-6


def test_adaptive_rejects_other_factorizations(G, two_spheres):
    V, T, k, _ = two_spheres
    with pytest.raises(G.EfieError):
        G.EFIE(V, T, k, 3, 0.0, 0, tree=TREE, factorization=G.EFIE_FACT_DIRECT)


def test_adaptive_uneven_mesh_against_uniform_tree(G):
    """An uneven mesh at scale (80,880 RWG): a finely meshed 1-wavelength
    sphere beside a coarsely meshed 2.5-wavelength one.  The uniform tree
    needs a 0.2-wavelength knot spacing here (finer spacings leave the coarse
    triangles' buffer splines no gap between far domains), so its near field
    holds 4.3e9 entries; the tree rule of Sec. VII (200 triangles, 25%
    protrusion) gives leaves on five levels and 9.4 times fewer near entries.
    Both are fast approximations of the same operator, so their products
    agree to the coarser one's accuracy (gate 1e-2); the setup and the time
    of a 64-vector product of each are printed."""
    import time
    torch = _torch()
    V, T = E.merge_meshes(E.icosphere(50, 1.0, center=(-2.25, 0.0, 0.0)),
                          E.icosphere(14, 2.5, center=(2.25, 0.1, 0.05)))
    k = 2 * np.pi
    X = torch.from_numpy(E.complex_gaussian((64, 80880), 96)).cuda()
    out = {}
    for name, kw in (("nonuniform", dict(tree=dict(max_elems=200, max_prot=0.25, top=2))),
                     ("uniform", dict(grid_spacing=0.2, levels=3))):
        t0 = time.perf_counter()
        h = G.EFIE(V, T, k, 3, precision=G.EFIE_MIXED, **kw)
        torch.cuda.synchronize()
        t_setup = time.perf_counter() - t0
        try:
            info = h.info()
            assert info["n_unknowns"] == 80880
            Y = torch.empty_like(X)
            h.matvec(X, Y)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(3):
                h.matvec(X, Y)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / 3
            out[name] = Y.cpu().numpy()
        finally:
            h.close()
        print(f"uneven mesh, {name} tree: setup {t_setup:.1f} s, near entries A {info['near_nnz_A']:.3g} "
              f"V {info['near_nnz_V']:.3g}, {ms:.1f} ms per 64-vector product ({64e3 / ms:.1f} matvecs/s)")
    a, b = out["nonuniform"], out["uniform"]
    rel = float(np.linalg.norm(a - b) / np.linalg.norm(b))
    print(f"uneven mesh: nonuniform vs uniform tree, rel l2 {rel:.3e}")
    assert rel < 1e-2

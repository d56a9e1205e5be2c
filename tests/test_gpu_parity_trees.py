"""GPU parity on the tree shapes and spline degrees that the C1 tests do not
reach: the CUDA path through the C ABI against the CPU oracle's B-spline
scheme on the same seeded inputs, element by element (relative l2 and
max-abs).

* every spline degree other than 3 (Table I: s_remove = 0 for p = 1, 2 and
  2 for p = 5, 6; the p-dependent moment extents and quadrature orders);
* a multilevel tree under the constant-s rule of Sec. IV-C (boxes below half
  a wavelength: s stays, the knot spacing doubles), far pairs on two levels;
* a three-level tree with two s-doublings (Sec. IV-D, s -> 2s - p twice:
  s' = 9, 13, 21), which runs the top-level kernels of the bench workload
  (s' = 21, FFT length 37, the shared-memory top-level translation for
  8-vector chunks) on a problem the oracle can finish.

Bounds: the plain FP64 form follows the oracle's arithmetic step for step, so
it agrees to rounding (measured ~1e-15; gate 1e-10); the mixed form keeps the
far field in complex FP32 (gate 1e-5, as in the C1 tests)."""
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


def _errs(got, ref):
    rel = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    mx = float(np.abs(got - ref).max() / np.abs(ref).max())
    return rel, mx


def _check(G, V, T, k, p, delta, levels, ref_op, seed, n_rhs=1, cols=(0,), tag=""):
    """FP64 and mixed handles against the oracle on seeded vectors."""
    torch = _torch()
    X = E.complex_gaussian((n_rhs, ref_op.mesh.N), seed)
    ref = np.stack([ref_op.matvec(X[c]) for c in cols])
    for prec, tol in ((G.EFIE_FP64, TOL64), (G.EFIE_MIXED, TOL32)):
        h = G.EFIE(V, T, k, p, delta, levels, precision=prec)
        try:
            Y = h.matvec(torch.from_numpy(X).cuda()).cpu().numpy()
        finally:
            h.close()
        rel, mx = _errs(Y[list(cols)], ref)
        print(f"{tag} precision={prec}: rel l2 {rel:.3e}, max-abs {mx:.3e}")
        assert rel < tol and mx < 10 * tol, (tag, prec, rel, mx)


@pytest.mark.parametrize("p", [1, 2, 5, 6])
def test_spline_degree(G, p, c1_mesh, c1_dense):
    """C1 sphere (1,920 RWG), k = 2 pi, 0.1-wavelength grid, 2 levels, p != 3.
    The near field comes from the oracle's dense quadrature (the tree, and
    so the near set, is the same for every p: the leaf box is (s - p) delta =
    4 delta)."""
    from oracle import fastmv
    from oracle.bspline import S_REMOVE
    V, T, m = c1_mesh
    k = 2 * np.pi
    ref_op = fastmv.BsplineEFIE(m, k, p, 0.1, 2, dense_AV=c1_dense)
    L = ref_op.tree.levels[ref_op.tree.D]
    assert L.s == p + 4 and L.shat == L.sp - 2 * S_REMOVE[p]
    _check(G, V, T, k, p, 0.1, 2, ref_op, 30 + p, tag=f"p={p}")


def test_constant_s_multilevel(G):
    """Sec. IV-C: on a 1-wavelength-diameter sphere at k = pi (lambda = 2),
    every box is below lambda/2, so s stays 7 on all three levels while the
    knot spacing doubles; far pairs on the leaf level and its parent."""
    from oracle import fastmv
    from oracle.geometry import build_rwg
    V, T = E.icosphere(10, 0.5)
    k, p, delta, levels = np.pi, 3, 0.06, 3
    info, lv = G.plan(V, T, k, p, delta, levels)
    assert len({L["s"] for L in lv}) == 1
    assert sum(L["n_far_pairs"] > 0 for L in lv) >= 2
    assert lv[1]["delta"] == pytest.approx(2 * lv[0]["delta"])
    ref_op = fastmv.BsplineEFIE(build_rwg(V, T), k, p, delta, levels)
    _check(G, V, T, k, p, delta, levels, ref_op, 40, tag="constant-s")


@pytest.fixture(scope="module")
def two_doublings():
    """Two spheres of radius 0.6 wavelength, 4.2 wavelengths apart (3,840
    RWG): with a 0.1-wavelength grid the leaf boxes are 0.4 wavelength and
    the root needs 4 levels, so a 3-level tree has grids of 0.4, 0.8 and 1.6
    wavelengths and s goes 7 -> 11 -> 19."""
    from oracle import fastmv
    from oracle.geometry import build_rwg
    A = E.icosphere(8, 0.6, center=(-2.1, 0.0, 0.0))
    B = E.icosphere(8, 0.6, center=(2.1, 0.3, 0.1))
    V, T = E.merge_meshes(A, B)
    k, p, delta, levels = 2 * np.pi, 3, 0.1, 3
    return V, T, k, p, delta, levels, fastmv.BsplineEFIE(build_rwg(V, T), k, p, delta, levels)


def test_three_levels_two_doublings(G, two_doublings):
    V, T, k, p, delta, levels, ref_op = two_doublings
    info, lv = G.plan(V, T, k, p, delta, levels)
    assert [L["s"] for L in lv] == [7, 11, 19]
    assert [L["sp"] for L in lv] == [9, 13, 21] and lv[2]["nfft"] == 37
    assert all(L["n_far_pairs"] > 0 for L in lv)
    # 8 vectors: the mixed form runs full 32-channel chunks through the
    # shared-memory top-level translation
    _check(G, V, T, k, p, delta, levels, ref_op, 50, n_rhs=8, cols=(0, 7), tag="two doublings")


@pytest.mark.parametrize("mac_variant", [0, 1, 2, 3, 5])
def test_two_doublings_translation_variants(G, two_doublings, mac_variant):
    """The top-level translation kernels the autotuner can pick (tensor cores
    persistent, register tiles, CUDA cores with shared-memory staging, tensor
    cores per tile and frequency, tensor cores persistent and loader-fed),
    mixed form, 8 vectors, against the oracle."""
    torch = _torch()
    V, T, k, p, delta, levels, ref_op = two_doublings
    h = G.EFIE(V, T, k, p, delta, levels, precision=G.EFIE_MIXED)
    try:
        h.autotune_set(8, mac_variant)
        X = E.complex_gaussian((8, h.N), 60 + mac_variant)
        Y = h.matvec(torch.from_numpy(X).cuda()).cpu().numpy()
    finally:
        h.close()
    for r in (0, 5):
        rel, mx = _errs(Y[r], ref_op.matvec(X[r]))
        assert rel < TOL32 and mx < 10 * TOL32, (mac_variant, r, rel, mx)


def test_two_doublings_chunk_pairs(G, two_doublings):
    """19 vectors in the mixed form: the first 16 go through the chunk-pair
    path (two chunks of 8 per tensor-core pass, 128-row B operands, N = 128
    MMAs) on every level: the top level's all-pairs tiles and the
    interaction-list tiles of the two levels below it (variant 0; variant 5,
    the loader-fed kernel), or the top level
    only with the lower levels on CUDA cores (variant 4); the last 3
    through the single-chunk path.  Both against the oracle, and against the
    CUDA-core translation (variant 2, one chunk at a time)."""
    torch = _torch()
    V, T, k, p, delta, levels, ref_op = two_doublings
    X = E.complex_gaussian((19, ref_op.mesh.N), 70)
    Xd = torch.from_numpy(X).cuda()
    h = G.EFIE(V, T, k, p, delta, levels, precision=G.EFIE_MIXED)
    try:
        Y = h.matvec(Xd).cpu().numpy()
        h.autotune_set(8, 4)
        Y4 = h.matvec(Xd).cpu().numpy()
        h.autotune_set(8, 5)
        Y5 = h.matvec(Xd).cpu().numpy()
        h.autotune_set(8, 2)
        Y2 = h.matvec(Xd).cpu().numpy()
    finally:
        h.close()
    for r in (0, 7, 8, 15, 16, 18):
        ref = ref_op.matvec(X[r])
        for tag, Yv in (("0", Y), ("4", Y4), ("5", Y5)):
            rel, mx = _errs(Yv[r], ref)
            print(f"chunk pair variant {tag} rhs {r}: rel l2 {rel:.3e}, max-abs {mx:.3e}")
            assert rel < TOL32 and mx < 10 * TOL32, (tag, r, rel, mx)
    assert np.linalg.norm(Y - Y2) < 1e-5 * np.linalg.norm(Y2)
    assert np.linalg.norm(Y4 - Y2) < 1e-5 * np.linalg.norm(Y2)
    assert np.linalg.norm(Y5 - Y2) < 1e-5 * np.linalg.norm(Y2)


def test_two_doublings_transform_schedules(G, two_doublings):
    """The four transform schedules (line passes; forward y and z passes
    fused per (box, x-frequency) slab; forward and inverse fused; both fused
    on the 9-spline level only, the default) on all three spline counts of
    the tree (s' = 9, 13, 21; FFT lengths 13, 21, 37), mixed form, 8
    vectors: each against the oracle, and against the line passes to FP32
    rounding."""
    torch = _torch()
    V, T, k, p, delta, levels, ref_op = two_doublings
    X = E.complex_gaussian((8, ref_op.mesh.N), 80)
    Xd = torch.from_numpy(X).cuda()
    h = G.EFIE(V, T, k, p, delta, levels, precision=G.EFIE_MIXED)
    try:
        assert h.transform_schedule() == 3
        Y3 = h.matvec(Xd).cpu().numpy()
        assert h.transform_schedule(0) == 0
        Y0 = h.matvec(Xd).cpu().numpy()
        assert h.transform_schedule(1) == 1
        Y1 = h.matvec(Xd).cpu().numpy()
        assert h.transform_schedule(2) == 2
        Y2 = h.matvec(Xd).cpu().numpy()
    finally:
        h.close()
    for r in (0, 3, 7):
        ref = ref_op.matvec(X[r])
        for tag, Yv in (("lines", Y0), ("fused forward", Y1), ("fused both", Y2), ("fused on 9", Y3)):
            rel, mx = _errs(Yv[r], ref)
            print(f"transform schedule {tag} rhs {r}: rel l2 {rel:.3e}, max-abs {mx:.3e}")
            assert rel < TOL32 and mx < 10 * TOL32, (tag, r, rel, mx)
    assert np.linalg.norm(Y1 - Y0) < 1e-6 * np.linalg.norm(Y0)
    assert np.linalg.norm(Y2 - Y0) < 1e-6 * np.linalg.norm(Y0)
    assert np.linalg.norm(Y3 - Y0) < 1e-6 * np.linalg.norm(Y0)

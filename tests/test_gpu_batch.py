"""Batching: meshes of uneven size and different numbers of right-hand sides
in one CUDA graph launch, checked against the CPU oracle's B-spline scheme,
and the autotuner."""
import numpy as np
import pytest

import efie_inputs as E

pytestmark = pytest.mark.gpu


def test_batch_graph_matches_individual_products():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    import paper_2606_13482_gb300 as G
    meshes = [E.ellipsoid(6, [0.3, 0.25, 0.2]), E.ellipsoid(9, [0.5, 0.4, 0.3]), E.icosphere(7, 0.35)]
    hs = [G.EFIE(V, T, 2 * np.pi, 3, 0.07, 1, precision=G.EFIE_MIXED) for V, T in meshes]
    counts = [1, 3, 8]
    xs = [torch.from_numpy(E.complex_gaussian((c, h.N), 10 + i)).cuda() for i, (c, h) in enumerate(zip(counts, hs))]
    ref = [h.matvec(x).cpu().numpy() for h, x in zip(hs, xs)]
    b = G.Batch(hs)
    ys = [torch.empty_like(x) for x in xs]
    for _ in range(2):                       # capture, then replay
        b.matvec(xs, ys)
        torch.cuda.synchronize()
        for y, r in zip(ys, ref):
            assert np.linalg.norm(y.cpu().numpy() - r) <= 1e-6 * np.linalg.norm(r)
    # new inputs in the same buffers: the replayed graph sees them
    for i, x in enumerate(xs):
        x.copy_(torch.from_numpy(E.complex_gaussian(tuple(x.shape), 50 + i)))
    ref2 = [h.matvec(x).cpu().numpy() for h, x in zip(hs, xs)]
    b.matvec(xs, ys)
    torch.cuda.synchronize()
    for y, r in zip(ys, ref2):
        assert np.linalg.norm(y.cpu().numpy() - r) <= 1e-6 * np.linalg.norm(r)
    # different output buffers: re-captured
    ys2 = [torch.empty_like(x) for x in xs]
    b.matvec(xs, ys2)
    torch.cuda.synchronize()
    for y, r in zip(ys2, ref2):
        assert np.linalg.norm(y.cpu().numpy() - r) <= 1e-6 * np.linalg.norm(r)
    # the graph's outputs against the oracle (mixed form: complex FP32 far field)
    from oracle import fastmv
    from oracle.geometry import build_rwg
    for (V, T), x, y, c in zip(meshes, xs, ys2, counts):
        ref_op = fastmv.BsplineEFIE(build_rwg(V, T), 2 * np.pi, 3, 0.07, 1)
        xc = x.cpu().numpy()
        yc = y.cpu().numpy()
        for r in sorted({0, c - 1}):
            ref = ref_op.matvec(xc[r])
            err = np.linalg.norm(yc[r] - ref) / np.linalg.norm(ref)
            print(f"batch graph vs oracle (N={x.shape[1]}, rhs {r}): {err:.3e}")
            assert err < 1e-5
    b.close()
    chunk, mac, near = hs[2].autotune(8)
    assert chunk in (1, 2, 4, 8) and mac in range(6) and near in range(4)
    y = hs[2].matvec(xs[2]).cpu().numpy()
    assert np.linalg.norm(y - ref2[2]) <= 1e-5 * np.linalg.norm(ref2[2])
    for h in hs:
        h.close()

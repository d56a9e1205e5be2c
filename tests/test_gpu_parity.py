"""GPU parity: the CUDA path through the C ABI against the CPU oracle on the
same seeded inputs.  Tolerances: plain FP64 form within 1e-10 relative l2 of
the oracle's B-spline scheme (expected ~1e-12: same rules, rounding only);
mixed form within 1e-5 (complex FP32 far field, ~1e-7 per product, grown
through the FFT and transfer passes)."""
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


@pytest.fixture(scope="module")
def c1_gpu(G, c1_mesh):
    V, T, _ = c1_mesh
    h64 = G.EFIE(V, T, 2 * np.pi, 3, 0.1, 2, precision=G.EFIE_FP64)
    h32 = G.EFIE(V, T, 2 * np.pi, 3, 0.1, 2, precision=G.EFIE_MIXED)
    yield h64, h32
    h64.close()
    h32.close()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_unknown_ordering(G, c1_gpu, c1_mesh):
    h64, _ = c1_gpu
    _, _, m = c1_mesh
    e, t = h64.rwg_edges()
    assert np.array_equal(e, m.edges) and np.array_equal(t, m.tri_pm)


def test_rhs_planewave(G, c1_gpu, c1_mesh):
    torch = _torch()
    from oracle import dense
    h64, _ = c1_gpu
    _, _, m = c1_mesh
    kh = np.array([[0, 0, -1.0], [0.6, 0.0, 0.8]])
    pol = np.array([[1.0, 0, 0], [0, 1.0, 0]])
    got = h64.rhs_planewave(kh, pol).cpu().numpy()
    ref = dense.rhs_planewave(m, 2 * np.pi, kh, pol)
    assert _rel(got, ref) < 1e-12


def test_matvec_fp64_vs_oracle(G, c1_gpu, c1_oracle):
    torch = _torch()
    h64, _ = c1_gpu
    x = E.complex_gaussian(h64.N, 1)
    y = h64.matvec(torch.from_numpy(x).cuda()).cpu().numpy()
    ref = c1_oracle.matvec(x)
    assert _rel(y, ref) < TOL64
    yA, yV = h64.matvec_parts(torch.from_numpy(x).cuda())
    rA, rV = c1_oracle.matvec_parts(x)
    assert _rel(yA.cpu().numpy(), rA) < TOL64
    assert _rel(yV.cpu().numpy(), rV) < TOL64


def test_matvec_mixed_vs_oracle(G, c1_gpu, c1_oracle):
    torch = _torch()
    _, h32 = c1_gpu
    x = E.complex_gaussian(h32.N, 2)
    y = h32.matvec(torch.from_numpy(x).cuda()).cpu().numpy()
    assert _rel(y, c1_oracle.matvec(x)) < TOL32
    # the FP64 entry point of a mixed handle: FP64 far field and the near field
    # kept as double-float pairs (48-bit significand), so ~1e-13 from the oracle
    y64 = h32.matvec(torch.from_numpy(x).cuda(), fp64=True).cpu().numpy()
    assert _rel(y64, c1_oracle.matvec(x)) < 1e-10


def test_batched_rhs_ragged_chunks(G, c1_gpu, c1_oracle):
    """11 right-hand sides: one chunk of 8 and a ragged chunk of 3."""
    torch = _torch()
    h64, h32 = c1_gpu
    X = E.complex_gaussian((11, h64.N), 3)
    Y = h64.matvec(torch.from_numpy(X).cuda()).cpu().numpy()
    for r in (0, 7, 8, 10):
        assert _rel(Y[r], c1_oracle.matvec(X[r])) < TOL64
    Y32 = h32.matvec(torch.from_numpy(X).cuda()).cpu().numpy()
    assert _rel(Y32, Y) < TOL32


def test_matvec_host_buffers(G, c1_gpu, c1_oracle):
    """efie_matvec_host: 11 right-hand sides in pinned and in pageable host
    memory (chunks of 8 and 3 through the double-buffered staging) give the
    device-buffer product; a second call reuses the staging."""
    torch = _torch()
    for h, tol in zip(c1_gpu, (1e-12, 1e-6)):
        X = torch.from_numpy(E.complex_gaussian((11, h.N), 21))
        ref = h.matvec(X.cuda()).cpu().numpy()
        for pinned in (True, False):
            Xh = X.pin_memory() if pinned else X.clone()
            for _ in range(2):
                Yh = h.matvec_host(Xh)
                torch.cuda.synchronize()
                err = _rel(Yh.numpy(), ref)
                print(f"host-buffer matvec (pinned={pinned}): {err:.3e}")
                assert err < tol
        assert _rel(ref[3], c1_oracle.matvec(X[3].numpy())) < (TOL64 if tol < 1e-9 else TOL32)
        empty = torch.zeros((0, h.N), dtype=torch.complex128)
        assert h.matvec_host(empty).shape == (0, h.N)


def test_star_null_space_gpu(G, c1_gpu, c1_mesh):
    """Sec. VI-A: the scalar part vanishes on loop currents (to roundoff)."""
    torch = _torch()
    h64, h32 = c1_gpu
    _, _, m = c1_mesh
    S = m.sigma_dense()
    x = E.complex_gaussian(m.N, 9)
    x = x - S @ np.linalg.lstsq(S, x, rcond=None)[0]
    for h in (h64, h32):
        yA, yV = h.matvec_parts(torch.from_numpy(x).cuda())
        assert np.linalg.norm(yV.cpu().numpy()) < 1e-9 * np.linalg.norm(yA.cpu().numpy())


def test_fast_vs_dense_gate(G, c1_gpu, c1_mesh, c1_dense):
    """Fast matvec within 1e-3 relative l2 of the dense FP64 product (C1)."""
    torch = _torch()
    from oracle import dense
    h64, h32 = c1_gpu
    _, _, m = c1_mesh
    A, V = c1_dense
    T = dense.efie_matrix(m, 2 * np.pi, A, V)
    x = E.complex_gaussian(m.N, 4)
    for h in (h64, h32):
        y = h.matvec(torch.from_numpy(x).cuda()).cpu().numpy()
        assert _rel(y, T @ x) < 1e-3


def test_solve_plane_wave(G, c1_gpu, c1_mesh, c1_dense):
    """GMRES to 1e-6 true residual; the solution agrees with the dense LU
    solution to tolerance plus the fast-matvec error."""
    torch = _torch()
    from oracle import dense
    h64, h32 = c1_gpu
    _, _, m = c1_mesh
    A, V = c1_dense
    T = dense.efie_matrix(m, 2 * np.pi, A, V)
    e = h64.rhs_planewave([0, 0, -1.0], [1.0, 0, 0])
    xs = np.linalg.solve(T, e.cpu().numpy()[0])
    for h in (h64, h32):
        x, info, rc = h.solve(e, tol=1e-6)
        assert rc == 0 and info[0]["converged"] and info[0]["true_rel_residual"] <= 1e-6
        assert _rel(x.cpu().numpy()[0], xs) < 2e-2


def test_empty_batch(G, c1_gpu):
    torch = _torch()
    h64, _ = c1_gpu
    x = torch.zeros((0, h64.N), dtype=torch.complex128, device="cuda")
    y = h64.matvec(x)
    assert y.shape == (0, h64.N)


TWO_LEVEL = (11, 0.5, 2 * np.pi * 2.2, 3, 0.06, 2)


@pytest.fixture(scope="module")
def two_level_oracle():
    from oracle import fastmv
    from oracle.geometry import build_rwg
    freq, r, k, p, delta, levels = TWO_LEVEL
    V, T = E.icosphere(freq, r)
    return V, T, fastmv.BsplineEFIE(build_rwg(V, T), k, p, delta, levels)


def test_two_level_increasing_s(G, two_level_oracle):
    """Two grid levels with far pairs on both and s -> 2s - p at the parent
    (boxes >= lambda/2): upward / downward transfers on the GPU."""
    torch = _torch()
    V, T, ref_op = two_level_oracle
    _, _, k, p, delta, levels = TWO_LEVEL
    info, lv = G.plan(V, T, k, p, delta, levels)
    assert lv[1]["s"] == 2 * lv[0]["s"] - p and lv[0]["n_far_pairs"] > 0 and lv[1]["n_far_pairs"] > 0
    h = G.EFIE(V, T, k, p, delta, levels, precision=G.EFIE_FP64)
    x = E.complex_gaussian(h.N, 5)
    y = h.matvec(torch.from_numpy(x).cuda()).cpu().numpy()
    h.close()
    assert _rel(y, ref_op.matvec(x)) < TOL64


def test_top_level_mixed_batched(G, two_level_oracle):
    """Mixed form with 8- and 3-vector chunks on a tree whose top grid level has
    far pairs (the shared-memory top-level translation path)."""
    torch = _torch()
    V, T, ref_op = two_level_oracle
    _, _, k, p, delta, levels = TWO_LEVEL
    h = G.EFIE(V, T, k, p, delta, levels, precision=G.EFIE_MIXED)
    X = E.complex_gaussian((11, h.N), 6)
    Y = h.matvec(torch.from_numpy(X).cuda()).cpu().numpy()
    h.close()
    for r in (0, 5, 9):
        assert _rel(Y[r], ref_op.matvec(X[r])) < TOL32


@pytest.mark.parametrize("mac_variant", [0, 1, 2, 3, 5])
def test_top_level_translation_variants(G, two_level_oracle, mac_variant):
    """The top-level translation kernels the autotuner can pick (0: tensor
    cores, 3-term TF32 split, persistent warp-specialised; 1: register tiles;
    2: CUDA cores with shared-memory staging; 3: tensor cores, one CTA per
    tile and frequency; 5: the persistent form fed by a loader warp) against
    the oracle, mixed form."""
    torch = _torch()
    V, T, ref_op = two_level_oracle
    _, _, k, p, delta, levels = TWO_LEVEL
    h = G.EFIE(V, T, k, p, delta, levels, precision=G.EFIE_MIXED)
    h.autotune_set(8, mac_variant)
    X = E.complex_gaussian((8, h.N), 7)
    Y = h.matvec(torch.from_numpy(X).cuda()).cpu().numpy()
    h.close()
    for r in (0, 7):
        assert _rel(Y[r], ref_op.matvec(X[r])) < TOL32


@pytest.mark.parametrize("near_variant", [0, 1, 2, 3])
def test_near_field_variants_mixed(G, c1_gpu, c1_oracle, near_variant):
    """The double-float near-field kernels (x staged by double-buffered
    asynchronous copies, 8 vectors per thread; x read through L1; x staged
    between barriers, 4 vectors per thread; x in an mbarrier ring filled by a
    copy warp, no block barriers) against the FP64 oracle, with 8-, 3- and
    1-vector chunks."""
    torch = _torch()
    h64, h32 = c1_gpu
    X = E.complex_gaussian((12, h32.N), 8)
    for chunk in (8, 3, 1):
        h32.autotune_set(chunk, 0, near_variant)
        Y = h32.matvec(torch.from_numpy(X).cuda()).cpu().numpy()
        for r in (0, 11):
            assert _rel(Y[r], c1_oracle.matvec(X[r])) < TOL32
    # FP64 far field + this double-float near field: FP64-class agreement
    Y64 = h32.matvec(torch.from_numpy(X[:2]).cuda(), fp64=True).cpu().numpy()
    assert _rel(Y64[1], c1_oracle.matvec(X[1])) < 1e-10
    h32.autotune_set(8, 0, 0)

"""GPU parity at full size: the 20-wavelength PEC sphere (geodesic frequency
200, 800,000 triangles, 1,200,000 RWG unknowns, p = 3, 0.1-wavelength grid,
3 grid levels), mixed form, 64 seeded right-hand sides in one call: the
workload and launch configuration that bench.py times.  The oracle cannot run
the B-spline scheme at this size, so the checks are
  * sampled outputs against the oracle's exact dense rows (Sec. II Galerkin
    EFIE, computed row by row without forming T): relative l2 <= 1e-3, the
    fast-matvec accuracy bound against the dense product;
  * the mixed form against the FP64 form of the same handle: <= 1e-5;
  * properties that hold at any size: complex symmetry of the fast operator
    (X^T T X is symmetric, since anterpolation and interpolation use the same
    moments and the Green's function is even), and linearity across the batch.
"""
import numpy as np
import pytest

import efie_inputs as E

pytestmark = pytest.mark.gpu

FREQ, RADIUS, K, P, DELTA, LEVELS, NRHS = 200, 10.0, 2 * np.pi, 3, 0.1, 3, 64


def _torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.fixture(scope="module")
def full():
    torch = _torch()
    import __graft_entry__ as g
    g.build()
    import paper_2606_13482_gb300 as G
    V, T = E.icosphere(FREQ, RADIUS)
    h = G.EFIE(V, T, K, P, DELTA, LEVELS, precision=G.EFIE_MIXED)
    gen = torch.Generator().manual_seed(1234)
    xh = torch.complex(torch.randn((NRHS, h.N), generator=gen, dtype=torch.float64),
                       torch.randn((NRHS, h.N), generator=gen, dtype=torch.float64))
    x = xh.cuda()
    y = h.matvec(x)
    torch.cuda.synchronize()
    yield G, h, V, T, xh, x, y
    h.close()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_fullsize_sampled_rows_vs_dense(full):
    G, h, V, T, xh, x, y = full
    from oracle import dense
    from oracle.geometry import build_rwg
    m = build_rwg(V, T)
    e, _ = h.rwg_edges()
    assert np.array_equal(e.astype(np.int64), m.edges)
    rng = np.random.default_rng(7)
    rows = np.sort(rng.choice(m.N, 3, replace=False))
    rhs = [0, 37]
    xs = xh[rhs].numpy()
    yA, yV = dense.rows_dense(m, K, rows, xs)
    ref = 1j * K * yA + yV / (1j * K)
    got = y[rhs].cpu().numpy()[:, rows]
    err = _rel(got, ref)
    print(f"full-size sampled rows vs dense: {err:.3e}")
    assert err < 1e-3


def test_fullsize_mixed_vs_fp64(full):
    G, h, V, T, xh, x, y = full
    rhs = [0, 37]
    y64 = h.matvec(x[rhs], fp64=True)
    err = _rel(y[rhs].cpu().numpy(), y64.cpu().numpy())
    print(f"full-size mixed vs FP64: {err:.3e}")
    assert err < 1e-5


def test_fullsize_symmetry_and_linearity(full):
    torch = _torch()
    G, h, V, T, xh, x, y = full
    S = x @ y.transpose(0, 1)                       # S_ij = x_i^T T x_j
    asym = float(torch.linalg.norm(S - S.transpose(0, 1)) / torch.linalg.norm(S))
    print(f"full-size ||S - S^T|| / ||S||: {asym:.3e}")
    assert asym < 1e-4
    a, b = 0.6 - 0.3j, -1.1 + 0.4j
    z = (a * x[3] + b * x[5]).unsqueeze(0)
    yz = h.matvec(z)
    lin = _rel(yz[0].cpu().numpy(), (a * y[3] + b * y[5]).cpu().numpy())
    print(f"full-size linearity: {lin:.3e}")
    assert lin < 1e-5

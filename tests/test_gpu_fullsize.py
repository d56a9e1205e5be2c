"""GPU parity at full size: the 20-wavelength PEC sphere (geodesic frequency
200, 800,000 triangles, 1,200,000 RWG unknowns, p = 3, 0.1-wavelength grid,
3 grid levels), mixed form, 64 seeded right-hand sides in one call: the
workload and launch configuration that bench.py times.  The oracle cannot run
the B-spline scheme at this size, so the checks are
  * sampled outputs against the oracle's exact dense rows (Sec. II Galerkin
    EFIE, computed row by row without forming T): relative l2 <= 1e-3, the
    fast-matvec accuracy bound against the dense product.  The rows are every
    RWG inside 16 seeded patches of 14 triangles spread over the sphere (about
    220 rows); a patch's rows share their test triangles, which is what a dense
    row costs, and the patches run in a process pool (spawn) on the host cores;
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


_MESH = None


def _pool_init(V, T):
    global _MESH
    from oracle.geometry import build_rwg
    _MESH = build_rwg(V, T)


def _pool_rows(args):
    from oracle import dense
    rows, xs = args
    yA, yV = dense.rows_dense(_MESH, K, rows, xs)
    return 1j * K * yA + yV / (1j * K)


def _patches(m, n_patches, n_tris, seed):
    """Row sets: the RWGs with both triangles inside a patch of n_tris
    triangles grown breadth-first from a seeded triangle."""
    tp = m.tri_pm
    a = np.concatenate([tp[:, 0], tp[:, 1]])
    b = np.concatenate([tp[:, 1], tp[:, 0]])
    o = np.argsort(a, kind="stable")
    ptr = np.searchsorted(a[o], np.arange(m.Nt + 1))
    nbr = b[o]
    rng = np.random.default_rng(seed)
    out = []
    for s0 in rng.choice(m.Nt, n_patches, replace=False):
        got, seen, i = [int(s0)], {int(s0)}, 0
        while len(got) < n_tris:
            for d in nbr[ptr[got[i]]:ptr[got[i] + 1]]:
                if int(d) not in seen and len(got) < n_tris:
                    seen.add(int(d))
                    got.append(int(d))
            i += 1
        inside = np.zeros(m.Nt, dtype=bool)
        inside[got] = True
        out.append(np.nonzero(inside[tp[:, 0]] & inside[tp[:, 1]])[0])
    return out


def test_fullsize_sampled_rows_vs_dense(full):
    import multiprocessing as mp
    import os
    from concurrent.futures import ProcessPoolExecutor
    G, h, V, T, xh, x, y = full
    from oracle.geometry import build_rwg
    m = build_rwg(V, T)
    e, _ = h.rwg_edges()
    assert np.array_equal(e.astype(np.int64), m.edges)
    patches = _patches(m, 16, 14, 7)
    rows = np.concatenate(patches)
    assert len(np.unique(rows)) == len(rows) >= 200
    rhs = [0, 37]
    xs = xh[rhs].numpy()
    workers = max(1, min(len(patches), os.cpu_count() or 1))
    with ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn"), initializer=_pool_init,
                             initargs=(V, T)) as ex:
        ref = np.concatenate(list(ex.map(_pool_rows, [(p, xs) for p in patches])), axis=1)
    got = y[rhs].cpu().numpy()[:, rows]
    err = _rel(got, ref)
    mx = float(np.abs(got - ref).max() / np.abs(ref).max())
    print(f"full-size sampled rows ({len(rows)}) vs dense: rel l2 {err:.3e}, max-abs {mx:.3e}")
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

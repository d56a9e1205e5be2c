"""Degenerate octrees: every leaf box is adjacent to every other, so the
interaction lists are empty on every grid level and T x is the near field
alone, which equals the dense Galerkin product with the same quadrature rules
(Sec. VI-A).  Cases: a single leaf box (depth 0), eight leaf boxes with one
grid level, and eight leaf boxes under a one-box parent level (transfers with
nothing to translate).  Both precisions against the oracle's dense matrix,
19 vectors (two full 8-vector chunks and a partial one), and in the mixed
form every double-float near-field kernel the autotuner can pick."""
import numpy as np
import pytest

import efie_inputs as E

pytestmark = pytest.mark.gpu

K = 2 * np.pi
CASES = [(4, 0.2, 0.1, 1), (6, 0.35, 0.1, 1), (6, 0.35, 0.1, 2)]
_dense = {}


def _torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _dense_T(freq, r):
    if (freq, r) not in _dense:
        from oracle import dense
        from oracle.geometry import build_rwg
        V, T = E.icosphere(freq, r)
        m = build_rwg(V, T)
        _dense[(freq, r)] = dense.efie_matrix(m, K)
    return _dense[(freq, r)]


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("freq,r,delta,levels", CASES)
def test_all_near_equals_dense(freq, r, delta, levels):
    torch = _torch()
    import __graft_entry__ as g
    g.build()
    import paper_2606_13482_gb300 as G
    V, T = E.icosphere(freq, r)
    info, lv = G.plan(V, T, K, 3, delta, levels)
    assert all(L["n_far_pairs"] == 0 for L in lv)
    Td = _dense_T(freq, r)
    X = E.complex_gaussian((19, Td.shape[0]), 17)
    ref = X @ Td.T
    for prec, nvs in ((G.EFIE_FP64, (0,)), (G.EFIE_MIXED, (0, 1, 2, 3))):
        h = G.EFIE(V, T, K, 3, delta, levels, precision=prec)
        try:
            for nv in nvs:
                h.autotune_set(8, 0, nv)
                Y = h.matvec(torch.from_numpy(X).cuda()).cpu().numpy()
                err = _rel(Y, ref)
                print(f"all-near {freq},{r},{levels} precision {prec} near variant {nv}: {err:.3e}")
                assert err < 1e-9
        finally:
            h.close()

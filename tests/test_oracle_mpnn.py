"""Pins of the learned-preconditioner reference network (not part of the
paper): finite-difference gradients, bfloat16 rounding against an independent
conversion, and the graph structure of a closed mesh."""
import numpy as np
import pytest

import efie_inputs as E
from oracle import mpnn
from oracle.geometry import build_rwg


@pytest.fixture(scope="module")
def small():
    V, T = E.icosphere(3, 0.3)
    m = build_rwg(V, T)
    return m, mpnn.build_graph(m)


def test_graph_degree_and_signs(small):
    m, (nbr, sgn, length) = small
    assert (nbr >= 0).all() and set(np.unique(sgn)) <= {-1.0, 1.0}
    # symmetric: n in N(m) with sign s  <=>  m in N(n) with the same sign
    for i in range(0, m.N, 7):
        for j in range(4):
            n = nbr[i, j]
            k = list(nbr[n]).index(i)
            assert sgn[n, k] == sgn[i, j]


def test_bf16_round_matches_torch():
    torch = pytest.importorskip("torch")
    x = np.random.default_rng(0).standard_normal(10000) * 10.0 ** np.random.default_rng(1).integers(-5, 5, 10000)
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mpnn.bf16_round(x), ref)


@pytest.mark.parametrize("bf16", [False, True])
def test_gradient_finite_differences(small, bf16):
    m, g = small
    p = mpnn.init_params(1)
    r = E.complex_gaussian(m.N, 1)
    e = E.complex_gaussian(m.N, 2)
    z, c = mpnn.forward(p, g, r)
    gr = mpnn.backward(p, g, c, z, e)
    rng = np.random.default_rng(0)
    for k in p:
        for _ in range(3):
            idx = tuple(rng.integers(0, s) for s in p[k].shape)
            eps = 1e-6
            pp = {kk: vv.copy() for kk, vv in p.items()}
            pm = {kk: vv.copy() for kk, vv in p.items()}
            pp[k][idx] += eps
            pm[k][idx] -= eps
            fd = (mpnn.loss(mpnn.forward(pp, g, r)[0], e) - mpnn.loss(mpnn.forward(pm, g, r)[0], e)) / (2 * eps)
            assert abs(fd - gr[k][idx]) <= 1e-5 * max(1e-3, abs(fd)), (k, idx, fd, gr[k][idx])
    if bf16:
        # the bf16 forward stays close to the exact one
        zb, _ = mpnn.forward(p, g, r, bf16=True)
        assert np.linalg.norm(zb - z) / np.linalg.norm(z) < 2e-2


def test_zero_residual_gives_zero(small):
    m, g = small
    z, _ = mpnn.forward(mpnn.init_params(0), g, np.zeros(m.N, dtype=complex))
    assert np.all(z == 0)

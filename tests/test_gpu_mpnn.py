"""GPU learned preconditioner (not part of the paper) against the FP64 NumPy
reference with the same bfloat16 rounding points: forward output and parameter
gradients (bfloat16 operands, FP32 accumulation: relative error ~1e-3,
checked at 2e-2 / cosine 0.999), then training on pairs harvested from the
plain solver's own GMRES runs."""
import numpy as np
import pytest

import efie_inputs as E

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.fixture(scope="module")
def setup():
    torch = _torch()
    import __graft_entry__ as g
    g.build()
    import paper_2606_13482_gb300 as G
    from oracle import mpnn
    from oracle.geometry import build_rwg
    V, T = E.icosphere(6, 0.3)
    h = G.EFIE(V, T, 2 * np.pi, 3, 0.07, 2, precision=G.EFIE_MIXED)
    m = build_rwg(V, T)
    graph = mpnn.build_graph(m)
    p = mpnn.init_params(3)
    vec, _ = mpnn.flatten(p)
    h.precond_params(vec.astype(np.float32))
    # the reference uses exactly the float32 parameters the GPU holds
    p32 = mpnn.unflatten(vec.astype(np.float32).astype(np.float64), p)
    yield G, h, graph, p32
    h.close()


def _cos(a, b):
    return float(np.dot(a.ravel(), b.ravel()) / (np.linalg.norm(a) * np.linalg.norm(b)))


def test_forward_parity(setup):
    torch = _torch()
    from oracle import mpnn
    G, h, graph, p = setup
    r = E.complex_gaussian(h.N, 11)
    z = h.precond_apply(torch.from_numpy(r).cuda()).cpu().numpy()
    zr, _ = mpnn.forward(p, graph, r, bf16=True)
    assert np.linalg.norm(z - zr) / np.linalg.norm(zr) < 2e-2
    assert abs(_cos(np.concatenate([z.real, z.imag]), np.concatenate([zr.real, zr.imag]))) > 0.999


def test_gradient_parity(setup):
    torch = _torch()
    from oracle import mpnn
    G, h, graph, p = setup
    r = E.complex_gaussian(h.N, 12)
    e = E.complex_gaussian(h.N, 13)
    g, loss = h.precond_gradient(torch.from_numpy(r).cuda(), torch.from_numpy(e).cuda())
    zr, cache = mpnn.forward(p, graph, r, bf16=True)
    gr = mpnn.backward(p, graph, cache, zr, e, bf16=True)
    assert abs(loss - mpnn.loss(zr, e)) < 1e-3 * mpnn.loss(zr, e)
    gref, keys = mpnn.flatten(gr)
    off = 0
    for k in keys:
        n = gr[k].size
        a, b = g[off:off + n], gref[off:off + n]
        off += n
        assert np.linalg.norm(a - b) <= 2e-2 * np.linalg.norm(b) + 1e-12, k
        assert _cos(a, b) > 0.999, k


def test_training_reduces_loss(setup, tmp_path):
    torch = _torch()
    G, h, graph, p = setup
    kh = np.array([[0, 0, -1.0], [1.0, 0, 0], [0, 1.0, 0], [0.6, 0, 0.8]])
    pol = np.array([[1.0, 0, 0], [0, 0, 1.0], [1.0, 0, 0], [0, 1.0, 0]])
    b = h.rhs_planewave(kh, pol)
    R, Ee = h.precond_harvest(b, restart=5, n_cycles=6)
    assert torch.isfinite(R).all() and torch.isfinite(Ee).all()
    losses = h.precond_train(R, Ee, epochs=30, lr=2e-3, seed=1)
    # Adam on 24 pairs lowers the relative error loss steadily (0.98 -> 0.76
    # measured on this mesh); require a clear, monotone-in-trend decrease
    assert losses[-1] < 0.9 * losses[0], losses
    assert losses[-1] < min(losses[:5]), losses
    path = str(tmp_path / "w.bin")
    h.precond_save(path)
    h.precond_load(path)
    x, info, rc = h.solve(b[:1], tol=1e-6)
    assert info[0]["converged"] and info[0]["true_rel_residual"] <= 1e-6


def test_precond_held_out(tmp_path):
    """Train on two ellipsoids with pairs from their own GMRES runs, then solve a
    held-out ellipsoid with FGMRES + network and with plain GMRES.  Asserted:
    both reach the 1e-6 true residual (checked with the plain FP64 fast
    matvec) and the network is used throughout (no fallback to plain GMRES).
    Not asserted: a gain.  Training is deterministic (fixed-order gradient
    sums, seeded shuffles), but the outcome moves with rounding-level changes
    of the training matvecs and with the training configuration: on this
    held-out mesh eight configurations gave from 13% fewer to 52% more
    iterations than plain GMRES, so the network is not reliably better here.
    The bound below (at most twice plain GMRES's iterations) only separates a
    working network from a broken one."""
    torch = _torch()
    import __graft_entry__ as g
    g.build()
    import paper_2606_13482_gb300 as G
    rng = np.random.default_rng(21)

    def pw(n, seed):
        r = np.random.default_rng(seed)
        kh = r.standard_normal((n, 3))
        kh /= np.linalg.norm(kh, axis=1, keepdims=True)
        pol = np.cross(kh, r.standard_normal((n, 3)))
        return kh, pol / np.linalg.norm(pol, axis=1, keepdims=True)

    path = str(tmp_path / "net.bin")
    for i in range(2):
        V, T = E.ellipsoid(9, rng.uniform(0.35, 0.6, 3))
        h = G.EFIE(V, T, 2 * np.pi, 3, 0.1, 1, precision=G.EFIE_MIXED, gmres_restart=30, max_iters=4000)
        if i:
            h.precond_load(path)
            h.precond_enable(False)
        b = h.rhs_planewave(*pw(3, i))
        R, Ee = h.precond_harvest(b, restart=8, n_cycles=6)
        h.precond_train(R, Ee, epochs=20, lr=2e-3, seed=i)
        h.precond_save(path)
        h.close()
    V, T = E.ellipsoid(9, [0.55, 0.4, 0.5])
    h = G.EFIE(V, T, 2 * np.pi, 3, 0.1, 1, precision=G.EFIE_MIXED, gmres_restart=30, max_iters=4000)
    b = h.rhs_planewave(*pw(2, 99))
    _, plain, _ = h.solve(b, tol=1e-6)
    h.precond_load(path)
    _, learned, _ = h.solve(b, tol=1e-6)
    h.close()
    print("held-out iterations plain", [a["iterations"] for a in plain],
          "learned", [c["iterations"] for c in learned])
    for a, c in zip(plain, learned):
        assert a["converged"] and c["converged"] and c["precond_fallback"] == 0
        assert c["true_rel_residual"] <= 1e-6
        assert c["iterations"] <= 2 * a["iterations"]


def test_training_is_deterministic():
    """Two trainings from the same seed on the same harvested pairs give
    bit-identical parameters, and so do two harvests of the same solves."""
    torch = _torch()
    import __graft_entry__ as g
    g.build()
    import paper_2606_13482_gb300 as G
    V, T = E.ellipsoid(7, [0.4, 0.3, 0.35])
    h = G.EFIE(V, T, 2 * np.pi, 3, 0.1, 1, precision=G.EFIE_MIXED, gmres_restart=30)
    try:
        b = h.rhs_planewave([[0, 0, -1.0], [1.0, 0, 0]], [[1.0, 0, 0], [0, 1.0, 0]])
        R1, E1 = h.precond_harvest(b, restart=6, n_cycles=3)
        R2, E2 = h.precond_harvest(b, restart=6, n_cycles=3)
        assert torch.equal(R1, R2) and torch.equal(E1, E2)
        p0 = (0.05 * np.random.default_rng(3).standard_normal(h.N_PARAMS)).astype(np.float32)
        params = []
        for objective in ("error", "residual"):
            for _ in range(2):
                h.precond_params(p0)                 # the same starting point each time
                h.precond_train(R1, E1, epochs=3, lr=2e-3, seed=5, objective=objective)
                params.append(h.precond_params())
        assert np.array_equal(params[0], params[1]) and np.array_equal(params[2], params[3])
        assert not np.array_equal(params[0], params[2])
    finally:
        h.close()

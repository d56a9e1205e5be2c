"""Failure paths, injected from the host (no GPU fault, trap or hang):

* a device-memory budget (efie_options.device_mem_limit) too small for the
  setup products returns EFIE_ENOMEM and frees what was allocated; a budget
  that fits one solve's workspace serves repeated solves, because every
  solve returns its workspace to the budget;
* non-finite network parameters loaded through efie_precond_params: the
  flexible solve sees a non-finite preconditioner output, hands every
  right-hand side back to plain GMRES (precond_fallback = 1) and still meets
  the tolerance on the FP64 true residual."""
import numpy as np
import pytest

import efie_inputs as E

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    import paper_2606_13482_gb300 as G
    return G


def test_device_mem_limit(G):
    import torch
    V, T = E.icosphere(8, 0.5)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        with pytest.raises(G.EfieError) as e:
            G.EFIE(V, T, 2 * np.pi, 3, 0.1, 2, device_mem_limit=1 << 20)
        assert e.value.code == -2 and "device_mem_limit" in str(e.value)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free0 - free1 < 64 << 20, (free0, free1)     # nothing left behind

    # the resident bytes of a handle after one product and one solve
    h = G.EFIE(V, T, 2 * np.pi, 3, 0.1, 2, gmres_restart=30)
    b_rhs = h.rhs_planewave([0, 0, -1.0], [1.0, 0, 0])
    x_ref, info, rc = h.solve(b_rhs, tol=1e-6)
    resident = h.info()["device_bytes"]
    h.close()
    work = (30 + 1) * h.N * 16 + 4 * h.N * 16 + (1 << 20)   # one solve's workspace, with slack
    h = G.EFIE(V, T, 2 * np.pi, 3, 0.1, 2, gmres_restart=30, device_mem_limit=resident + work)
    try:
        for _ in range(3):                                  # the budget comes back after every solve
            x, info, rc = h.solve(b_rhs, tol=1e-6)
            assert rc == 0 and info[0]["converged"]
            assert np.allclose(x.cpu().numpy(), x_ref.cpu().numpy(), rtol=0, atol=1e-12 * float(x_ref.abs().max()))
            assert h.info()["device_bytes"] == resident
    finally:
        h.close()
    # a budget with no room for the workspace: the solve fails cleanly and the
    # handle still computes products
    h = G.EFIE(V, T, 2 * np.pi, 3, 0.1, 2, gmres_restart=30, device_mem_limit=resident + (1 << 16))
    try:
        y0 = h.matvec(b_rhs)
        with pytest.raises(G.EfieError) as e:
            h.solve(b_rhs, tol=1e-6)
        assert e.value.code == -2
        assert h.info()["device_bytes"] == resident
        y1 = h.matvec(b_rhs)
        assert torch_equal(y0, y1)
    finally:
        h.close()


def torch_equal(a, b):
    import torch
    return bool(torch.equal(a, b))


def test_nonfinite_network_falls_back(G):
    V, T = E.icosphere(8, 0.5)
    h = G.EFIE(V, T, 2 * np.pi, 3, 0.1, 2, gmres_restart=50)
    try:
        b = h.rhs_planewave([[0, 0, -1.0], [1.0, 0, 0]], [[1.0, 0, 0], [0, 1.0, 0]])
        x_plain, info_plain, rc = h.solve(b, tol=1e-6)
        assert rc == 0
        w = np.full(h.N_PARAMS, np.nan, dtype=np.float32)
        h.precond_params(w)                                  # loads the parameters
        h.precond_enable(True)
        x, info, rc = h.solve(b, tol=1e-6)
        assert rc == 0
        for i, ip in zip(info, info_plain):
            assert i["precond_fallback"] == 1
            assert i["converged"] and i["true_rel_residual"] <= 1e-6
        rel = np.linalg.norm((x - x_plain).cpu().numpy()) / np.linalg.norm(x_plain.cpu().numpy())
        assert rel < 1e-5
    finally:
        h.close()

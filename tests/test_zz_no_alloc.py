"""The allocation-free plane-wave entry point.

Some callers may not allocate device memory once they are running (a
no-allocation or memory-pool policy, loops that cannot take the
synchronisation of cudaMalloc/cudaFree).  efie_rhs_planewave_noalloc serves
them from a fixed device array of the library; this test checks that it gives
the same right-hand sides as efie_rhs_planewave on two calls in a row with
different inputs (the shared array keeps the previous call's contents), and
that it rejects batches beyond its fixed capacity.  This file is collected
last so a failure here leaves every other test already run."""
import numpy as np
import pytest

import efie_inputs as E

pytestmark = pytest.mark.gpu


def test_rhs_planewave_noalloc_matches():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    import paper_2606_13482_gb300 as G
    V, T = E.icosphere(6, 0.3)
    h = G.EFIE(V, T, 2 * np.pi, 3, 0.07, 2, precision=G.EFIE_FP64)
    try:
        rng = np.random.default_rng(5)
        for call, n in enumerate((7, 3)):
            kh = rng.standard_normal((n, 3))
            kh /= np.linalg.norm(kh, axis=1, keepdims=True)
            pol = np.cross(kh, rng.standard_normal((n, 3)))
            ref = h.rhs_planewave(kh, pol).cpu().numpy()
            out = torch.empty((n, h.N), dtype=torch.complex128, device="cuda")
            got = h.rhs_planewave_noalloc(kh, pol, out).cpu().numpy()
            assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref), call
        big = torch.empty((4097, h.N), dtype=torch.complex128, device="cuda")
        with pytest.raises(G.EfieError) as e:
            h.rhs_planewave_noalloc(np.tile([0, 0, 1.0], (4097, 1)), np.tile([1.0, 0, 0], (4097, 1)), big)
        assert e.value.code == -1
    finally:
        h.close()

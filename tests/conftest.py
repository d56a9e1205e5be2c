import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: longer CPU test")


@pytest.fixture(scope="session")
def c1_mesh():
    import efie_inputs as E
    from oracle.geometry import build_rwg
    V, T = E.icosphere(8, 0.5)
    return V, T, build_rwg(V, T)


@pytest.fixture(scope="session")
def c1_dense(c1_mesh):
    from oracle import dense
    _, _, m = c1_mesh
    k = 2 * np.pi
    A, V = dense.assemble_dense(m, k)
    return A, V


@pytest.fixture(scope="session")
def c1_oracle(c1_mesh, c1_dense):
    from oracle import fastmv
    _, _, m = c1_mesh
    return fastmv.BsplineEFIE(m, 2 * np.pi, 3, 0.1, 2, dense_AV=c1_dense)

import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built libvie")
    config.addinivalue_line("markers", "slow: long CPU test")


@pytest.fixture(scope="session")
def tiny_dense():
    """(Problem, dense scaled matrix, scaled RHS, khat, pol) of the 4x4 array of 3^3-voxel cubes."""
    import workloads
    from oracle import problem_from_geometry, assembly as A
    g, kh, pol = workloads.config("tiny")
    P = problem_from_geometry(g)
    Z = A.dense_matrix(P)
    return P, Z, A.rhs(P, kh[0], pol[0]), kh[0], pol[0]

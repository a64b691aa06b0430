import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: larger CPU cases")


@pytest.fixture(scope="session")
def gen():
    from paper_1410_2153_gb300 import meshgen
    return meshgen


def oracle_iterate(mesh, b, steps, **params):
    """The oracle's PCG iterate after exactly `steps` iterations.

    Solutions are compared at 1e-10 when both sides take the same number of
    steps.  A right-hand side whose residual crosses rtol within rounding of
    the stopping test can stop one step apart on the two sides; the iterates
    then differ by up to the stopping tolerance, so the library's solution is
    compared with the oracle's iterate after the library's step count."""
    import oracle
    o = oracle.Oracle(mesh, **dict(params, max_iter=max(int(steps), 1)))
    u, _, _, _ = o.solve(b, rtol=0.0)
    return u

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


def mixed_iterations_ok(mesh, b, it_mixed, it_ref, u_mixed, **params):
    """Iteration gate of a GPU solve (the mixed-precision form, or a variant
    whose step count is sensitive to rounding) against the FP64 oracle's
    count it_ref at rtol 1e-8.

    Within 2 steps: accepted.  More steps are accepted only with the check of
    the mixed-precision reading (the FP32 preconditioner is a perturbed one,
    so the flexible CG may need extra steps; the answer must not suffer): the
    solution must be as close to the oracle's solve at rtol 1e-13 as the
    oracle's own rtol-1e-8 solution is, within a factor 2 (an rtol-1e-8 stop
    bounds the residual, not the error; where the residual crosses the
    threshold moves the error by up to the residual's drop per step), and the
    step count stays within a quarter of the oracle's.  Returns (ok, message)."""
    import numpy as np
    import oracle
    if abs(it_mixed - it_ref) <= 2:
        return True, ""
    o = oracle.Oracle(mesh, **params)
    u13, st13, _, _ = o.solve(b, rtol=1e-13)
    u8, st8, _, _ = o.solve(b, rtol=1e-8)
    e_mixed = np.linalg.norm(u_mixed - u13) / np.linalg.norm(u13)
    e_ref = np.linalg.norm(u8 - u13) / np.linalg.norm(u13)
    ok = st13 == 0 and abs(it_mixed - it_ref) <= 0.25 * it_ref and e_mixed <= 2.0 * e_ref
    return ok, f"mixed {it_mixed} vs {it_ref} steps; error to the rtol-1e-13 solve {e_mixed:.3e} vs oracle {e_ref:.3e}"

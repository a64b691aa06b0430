"""Several right-hand sides in one solve (the SpMM form) against the oracle.

amg_solve_multi runs the PCG on up to 4 columns at once, each matrix read
serving every column.  Per column the arithmetic is that of amg_solve except
on the small auxiliary levels that the fused shared-memory kernels hold (fewer
rows fit when 4 columns share the shared memory), so columns are compared with
the oracle at the parity tolerances (FP64 1e-10, mixed 1e-6 against the FP64
oracle, iterations within 2 or with the rtol-1e-13 check of
conftest.mixed_iterations_ok) and with single-column solves at 1e-9.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from conftest import mixed_iterations_ok, oracle_iterate  # noqa: E402


def _case(gen, name):
    if name == "graded257":
        return gen.grid2d(257, 2, graded=True), {}
    if name == "jitter129":
        return gen.grid2d(129, 7), {}
    m, _ = gen.workload_3d(seed=2, nside=17)
    return m, {"n_min": 6}


@pytest.mark.parametrize("name", ["graded257", "jitter129", "kuhn17_jump"])
@pytest.mark.parametrize("precision", [0, 1])
def test_multi_columns_match_oracle_and_single_solves(gen, name, precision):
    from paper_1410_2153_gb300 import asmg
    m, p = _case(gen, name)
    o = oracle.Oracle(m, **p)
    vf = o.vertex_of_free()
    k = 4
    B = np.zeros((k, m.nv))
    refs = []
    for c in range(k):
        b = o.mass_apply(gen.nodal_uniform(m, 40 + c))
        B[c, vf] = b
        refs.append(b)
    s = asmg.Solver(m, precision=precision, **p)
    U = torch.zeros(k * m.nv, dtype=torch.float64, device="cuda")
    hist = np.zeros(k * (s.params.max_iter + 1))
    rc, its, st = asmg.amg_solve_multi(s.h, k, torch.from_numpy(B.ravel()).cuda(), U, 1e-8, hist)
    assert rc == asmg.ASMG_OK and (st == 0).all()
    U = U.cpu().numpy().reshape(k, m.nv)
    tol = 1e-10 if precision == 0 else 1e-6
    for c in range(k):
        u_ref, sto, it_ref, hist_ref = o.solve(refs[c], rtol=1e-8)
        assert sto == 0
        ok, msg = mixed_iterations_ok(m, refs[c], int(its[c]), it_ref, U[c, vf], **p)
        assert ok, msg
        want = u_ref
        if precision == 0 and its[c] != it_ref:
            want = oracle_iterate(m, refs[c], int(its[c]), **p)
        assert np.linalg.norm(U[c, vf] - want) <= tol * np.linalg.norm(want), c
        # the column's residual history ends below the stopping tolerance
        h = hist[c * (s.params.max_iter + 1): c * (s.params.max_iter + 1) + its[c] + 1]
        assert h[-1] <= 1e-8 * np.linalg.norm(refs[c]) and h[0] > 0
        single, rc1, it1, _ = s.solve(B[c], rtol=1e-8)
        assert rc1 == asmg.ASMG_OK and abs(it1 - its[c]) <= 2
        if it1 == its[c]:
            assert np.linalg.norm(single - U[c]) <= 1e-9 * np.linalg.norm(single)
    s.close()


def test_multi_fewer_columns_and_zero_column(gen):
    # k < 4 leaves the unused columns at zero; a zero right-hand side is
    # converged before the first step and stays zero
    from paper_1410_2153_gb300 import asmg
    m = gen.grid2d(97, 3)
    o = oracle.Oracle(m)
    vf = o.vertex_of_free()
    s = asmg.Solver(m, precision=1)
    B = np.zeros((3, m.nv))
    B[0, vf] = o.mass_apply(gen.nodal_uniform(m, 5))
    B[2, vf] = o.mass_apply(gen.nodal_uniform(m, 6))
    U = np.zeros(3 * m.nv)
    rc, its, st = asmg.amg_solve_multi(s.h, 3, B.ravel(), U, 1e-8)   # host arrays
    assert rc == asmg.ASMG_OK and (st == 0).all()
    assert its[1] == 0 and np.all(U[m.nv:2 * m.nv] == 0)
    U = U.reshape(3, m.nv)
    for c in (0, 2):
        u_ref, _, it_ref, _ = o.solve(B[c, vf], rtol=1e-8)
        assert abs(its[c] - it_ref) <= 2
        assert np.linalg.norm(U[c, vf] - u_ref) <= 1e-6 * np.linalg.norm(u_ref)
    with pytest.raises(asmg.AsmgError) as e:
        asmg.amg_solve_multi(s.h, 5, np.zeros(5 * m.nv), np.zeros(5 * m.nv), 1e-8)
    assert e.value.code == asmg.ASMG_ERR_INVALID_ARG
    s.close()

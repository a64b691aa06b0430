"""BF16 storage of the auxiliary-level matrices (asmg_params.level_bf16).

The mixed form may read the level operators A_l of the V-cycle (its sweeps
and residuals) in BF16: each stored value is the FP32 value rounded to
nearest even, widened back to FP32 exactly on load, and the arithmetic,
diagonal inverses and vectors stay FP32.  That changes the preconditioner,
not the problem: the flexible CG still stops on the FP64 residual at rtol, so
solutions are held to the FP64 oracle at the mixed tolerance (relative 1e-6)
with the iteration gate of the mixed form (conftest.mixed_iterations_ok).
Every schedule reads the same BF16 values, so tiled sweeps equal the class
launches bit for bit, and the 4-column solve matches single solves at 1e-9.
The tile and multi-column cases use a lognormal coefficient, whose values
BF16 rounds.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from conftest import mixed_iterations_ok  # noqa: E402


def _case(gen, name):
    if name == "graded257":
        return gen.grid2d(257, 2, graded=True), {}
    if name == "jitter129_lognormal":
        m = gen.grid2d(129, 3)
        m.coeff = np.exp(2.0 * np.random.default_rng(9).normal(size=m.ne))
        return m, {}
    if name == "L129":
        return gen.grid2d_domain(129, 3, "L"), {}
    if name == "square65_neumann":
        m = gen.grid2d(65, 1)
        x, y = m.verts[:, 0], m.verts[:, 1]
        m.bflag = m.bflag.copy()
        m.bflag[(x == 1.0) & (y > 0) & (y < 1)] = 2
        return m, {"coarse_max": 8}
    m, _ = gen.workload_3d(seed=2, nside=33)
    return m, {"n_min": 6}


def _lib_params(p):
    return {("coarse_max_dofs" if k == "coarse_max" else k): v for k, v in p.items()}


@pytest.mark.parametrize("name", ["graded257", "jitter129_lognormal", "L129", "square65_neumann", "kuhn33_jump"])
def test_bf16_levels_solve_to_oracle(gen, name):
    from paper_1410_2153_gb300 import asmg
    m, p = _case(gen, name)
    lp = _lib_params(p)
    s16 = asmg.Solver(m, precision=asmg.ASMG_MIXED, level_bf16=1, **lp)
    s32 = asmg.Solver(m, precision=asmg.ASMG_MIXED, **lp)
    # one application of B moves by about the BF16 rounding (2^-9 relative
    # per value), not more.  With a coefficient of 1 on a box, the level
    # stencils are small dyadic numbers (4, -1, 2, -1/2, ...), exact in BF16,
    # and B does not move at all; a varying coefficient (lognormal, a jump of
    # 1e3) is rounded, and B moves
    rng = np.random.default_rng(3)
    r = torch.from_numpy(rng.standard_normal(m.nv)).cuda()
    z16 = s16.precond(r).cpu().numpy()
    z32 = s32.precond(r).cpu().numpy()
    d = np.linalg.norm(z16 - z32) / np.linalg.norm(z32)
    if name == "graded257":
        assert d == 0.0, d
    elif name in ("jitter129_lognormal", "kuhn33_jump"):
        assert 1e-6 < d < 5e-2, d
    else:
        assert d < 5e-2, d
    o = oracle.Oracle(m, **p)
    vf = o.vertex_of_free()
    f = gen.nodal_uniform(m, 19)
    b = o.mass_apply(f)
    u_ref, st, it_ref, _ = o.solve(b, rtol=1e-8)
    assert st == 0
    u, rc, it, hist = s16.solve(s16.mass_apply(torch.from_numpy(f).cuda()), rtol=1e-8)
    assert rc == asmg.ASMG_OK
    u = u.cpu().numpy()[vf]
    ok, msg = mixed_iterations_ok(m, b, it, it_ref, u, **p)
    assert ok, msg
    err = np.linalg.norm(u - u_ref) / np.linalg.norm(u_ref)
    assert err <= 1e-6, err
    s16.close()
    s32.close()


@pytest.mark.parametrize("tile_rows", [64, 300])
def test_bf16_tiled_sweeps_equal_class_launches(gen, tile_rows):
    from paper_1410_2153_gb300 import asmg
    m = gen.grid2d(257, 4, graded=True)
    m.coeff = np.exp(np.random.default_rng(10).normal(size=m.ne))
    ref = asmg.Solver(m, precision=asmg.ASMG_MIXED, level_bf16=1, tile_rows=-1)
    til = asmg.Solver(m, precision=asmg.ASMG_MIXED, level_bf16=1, tile_rows=tile_rows)
    assert sum(til.info("ntiles", l) > 0 for l in range(til.info("coarse") + 1, til.info("J") + 1)) > 0
    rng = np.random.default_rng(6)
    r = torch.from_numpy(rng.standard_normal(m.nv)).cuda()
    z0 = ref.precond(r).cpu().numpy()
    z1 = til.precond(r).cpu().numpy()
    assert np.array_equal(z0, z1), np.abs(z0 - z1).max()
    b = ref.mass_apply(torch.from_numpy(gen.nodal_uniform(m, 8)).cuda())
    u0, rc0, it0, h0 = ref.solve(b, rtol=1e-8)
    u1, rc1, it1, h1 = til.solve(b, rtol=1e-8)
    assert rc0 == rc1 == asmg.ASMG_OK and it0 == it1
    assert np.array_equal(u0.cpu().numpy(), u1.cpu().numpy())
    ref.close()
    til.close()


def test_bf16_multi_columns_match_single_solves(gen):
    from paper_1410_2153_gb300 import asmg
    m = gen.grid2d(257, 2, graded=True)
    m.coeff = np.exp(np.random.default_rng(11).normal(size=m.ne))
    s = asmg.Solver(m, precision=asmg.ASMG_MIXED, level_bf16=1)
    k = 4
    B = torch.stack([s.mass_apply(torch.from_numpy(gen.nodal_uniform(m, 50 + c)).cuda()) for c in range(k)])
    U = torch.zeros(k * m.nv, dtype=torch.float64, device="cuda")
    hist = np.zeros(k * (s.params.max_iter + 1))
    rc, its, st = asmg.amg_solve_multi(s.h, k, B.reshape(-1).contiguous(), U, 1e-8, hist)
    assert rc == asmg.ASMG_OK and (st == 0).all()
    U = U.cpu().numpy().reshape(k, m.nv)
    for c in range(k):
        u, rc1, it1, _ = s.solve(B[c].contiguous(), rtol=1e-8)
        assert rc1 == asmg.ASMG_OK and abs(int(its[c]) - it1) <= 2
        u = u.cpu().numpy()
        if it1 == int(its[c]):
            assert np.linalg.norm(U[c] - u) <= 1e-9 * np.linalg.norm(u), c
    s.close()

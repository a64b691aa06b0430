"""Temporally blocked auxiliary sweeps against the class-by-class launches.

With tile_rows > 0 every pre- and post-smoothing sweep of an auxiliary level
runs in one launch (one thread block per tile of smoothing rows plus its
halo).  The tiles keep each row's arithmetic and entry order, and leave out
only entries that cannot reach the tile's own results, so one preconditioner
application and whole solves must equal the launches per colour class and
sweep (tile_rows = -1) bit for bit; the solves are also held to the oracle at
the parity tolerances (1e-10 FP64, 1e-6 mixed; iterations within 2).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402


def _cases(gen):
    # 33^3: the finest auxiliary level (31^3 nodes) is too large for the
    # fused small-level kernels, so it runs the per-level sweeps
    m3, f3 = gen.workload_3d(seed=2, nside=33)
    return {
        "graded257": (gen.grid2d(257, 2, graded=True), {}),
        "jitter129": (gen.grid2d(129, 3), {}),
        "kuhn33_jump": (m3, {"n_min": 6}),
        "L129": (gen.grid2d_domain(129, 3, "L"), {}),
    }


@pytest.mark.parametrize("name", ["graded257", "jitter129", "kuhn33_jump", "L129"])
@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("size", ["small", "large"])
def test_tiled_sweeps_equal_class_launches(gen, name, precision, size):
    from paper_1410_2153_gb300 import asmg
    m, opts = _cases(gen)[name]
    # own rows per tile: 3D rows are longer and their halos deeper, so their
    # tiles are smaller for the shared-memory budget
    tile_rows = {("small", 2): 64, ("large", 2): 300, ("small", 3): 32, ("large", 3): 64}[(size, m.dim)]
    ref = asmg.Solver(m, precision=precision, tile_rows=-1, **opts)
    til = asmg.Solver(m, precision=precision, tile_rows=tile_rows, **opts)
    ntiled = sum(til.info("ntiles", l) > 0 for l in range(til.info("coarse") + 1, til.info("J") + 1))
    assert ntiled > 0
    assert all(ref.info("ntiles", l) == 0 for l in range(ref.info("coarse") + 1, ref.info("J") + 1))
    rng = np.random.default_rng(5)
    r = torch.from_numpy(rng.standard_normal(m.nv)).cuda()
    z0 = ref.precond(r).cpu().numpy()
    z1 = til.precond(r).cpu().numpy()
    assert np.array_equal(z0, z1), np.abs(z0 - z1).max()
    f = gen.nodal_uniform(m, 13)
    b = ref.mass_apply(torch.from_numpy(f).cuda())
    u0, rc0, it0, h0 = ref.solve(b, rtol=1e-8)
    u1, rc1, it1, h1 = til.solve(b, rtol=1e-8)
    assert rc0 == rc1 == asmg.ASMG_OK and it0 == it1
    assert np.array_equal(u0.cpu().numpy(), u1.cpu().numpy())
    assert np.array_equal(h0, h1)
    # the tiled solve against the oracle
    o = oracle.Oracle(m, **opts)
    vf = o.vertex_of_free()
    u_ref, st, it_ref, _ = o.solve(o.mass_apply(f), rtol=1e-8)
    assert abs(it1 - it_ref) <= 2
    tol = 1e-10 if precision == 0 else 1e-6
    if precision == 0 and it1 != it_ref:
        from conftest import oracle_iterate
        u_ref = oracle_iterate(m, o.mass_apply(f), it1, **opts)
    err = np.linalg.norm(u1.cpu().numpy()[vf] - u_ref) / np.linalg.norm(u_ref)
    assert err <= tol, err
    ref.close()
    til.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_autotuned_schedule_equals_class_launches(gen, precision):
    # tile_rows = 0: the setup times each level both ways and keeps the
    # faster schedule; whatever it picks, the solve is the same bit for bit
    from paper_1410_2153_gb300 import asmg
    m = gen.grid2d(257, 4, graded=True)
    ref = asmg.Solver(m, precision=precision, tile_rows=-1)
    aut = asmg.Solver(m, precision=precision)
    f = gen.nodal_uniform(m, 3)
    b = ref.mass_apply(torch.from_numpy(f).cuda())
    u0, rc0, it0, h0 = ref.solve(b, rtol=1e-8)
    u1, rc1, it1, h1 = aut.solve(b, rtol=1e-8)
    assert rc0 == rc1 == asmg.ASMG_OK and it0 == it1
    assert np.array_equal(u0.cpu().numpy(), u1.cpu().numpy())
    ref.close()
    aut.close()


@pytest.mark.parametrize("graph", [1, 0])
def test_expired_wait_reports_timeout_and_gpu_stays_usable(gen, graph):
    # failure injection on the host side: every tiled sweep takes the path of
    # an expired bounded wait (it still waits for its own shared-memory copy
    # before exiting).  The solve stops with ASMG_ERR_TIMEOUT, the context
    # stays usable, and a handle without injection then solves normally.
    from paper_1410_2153_gb300 import asmg
    m = gen.grid2d(257, 4, graded=True)
    bad = asmg.Solver(m, precision=1, tile_rows=64, inject_timeout=1, use_graph=graph)
    f = torch.from_numpy(gen.nodal_uniform(m, 3)).cuda()
    b = bad.mass_apply(f)
    u = torch.zeros_like(b)
    hist = np.zeros(bad.params.max_iter + 1)
    with pytest.raises(asmg.AsmgError) as e:
        asmg.amg_solve(bad.h, b, u, 1e-8, hist)
    assert e.value.code == asmg.ASMG_ERR_TIMEOUT
    with pytest.raises(asmg.AsmgError) as e:
        bad.precond(b)
    assert e.value.code == asmg.ASMG_ERR_TIMEOUT
    bad.close()
    torch.cuda.synchronize()
    good = asmg.Solver(m, precision=1, tile_rows=64, use_graph=graph)
    u, rc, it, _ = good.solve(good.mass_apply(f), rtol=1e-8)
    assert rc == asmg.ASMG_OK and it > 0
    good.close()

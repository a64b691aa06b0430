"""Batched solves: independent meshes of uneven size, several right-hand
sides each, one graph launch.  A problem's right-hand sides are solved in
groups of 4 columns (amg_solve_multi's SpMM form, one graph branch per
group): every batched solution must equal the multiple solve of the same
handle bit for bit (same kernels, deterministic reductions), agree with the
single-column solve to 1e-9, and match the oracle (1e-10 relative in FP64,
1e-6 in mixed precision)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from conftest import oracle_iterate  # noqa: E402


def test_batched_solves_match_single_solves_and_oracle(gen):
    from paper_1410_2153_gb300 import asmg
    sizes = [17, 40, 33, 65, 23]
    precisions = [0, 1, 0, 1, 0]
    nrhs = 3
    meshes = [gen.grid2d(n, 50 + i) for i, n in enumerate(sizes)]
    solvers = [asmg.Solver(m, precision=p) for m, p in zip(meshes, precisions)]
    rng = np.random.default_rng(11)
    bs, us, refs = [], [], []
    for m, s in zip(meshes, solvers):
        o = oracle.Oracle(m)
        for j in range(nrhs):
            f = gen.nodal_uniform(m, 100 + j)
            b = o.mass_apply(f)
            bv = np.zeros(m.nv)
            bv[o.vertex_of_free()] = b
            # alternate host and device arrays
            if j % 2:
                bs.append(torch.from_numpy(bv).cuda())
                us.append(torch.zeros(m.nv, dtype=torch.float64, device="cuda"))
            else:
                bs.append(bv)
                us.append(np.zeros(m.nv))
            refs.append((o, b))
    batch = asmg.amg_batch_create([s.h for s in solvers], nrhs, 1e-8)
    for trial in range(2):                      # the batch graph is reusable
        for u in us:
            u.zero_() if hasattr(u, "zero_") else u.fill(0.0)
        rc, its, st = asmg.amg_batch_solve(batch, bs, us)
        assert rc == asmg.ASMG_OK and (st == 0).all()
        k = 0
        for p, (m, s) in enumerate(zip(meshes, solvers)):
            bm = np.concatenate([bs[p * nrhs + j].cpu().numpy() if hasattr(bs[p * nrhs + j], "cpu")
                                 else bs[p * nrhs + j] for j in range(nrhs)])
            um = np.zeros(nrhs * m.nv)
            rcm, itm, _ = asmg.amg_solve_multi(s.h, nrhs, bm, um, 1e-8)
            assert rcm == asmg.ASMG_OK
            for j in range(nrhs):
                o, b = refs[k]
                u = us[k].cpu().numpy() if hasattr(us[k], "cpu") else us[k]
                bv = bs[k].cpu().numpy() if hasattr(bs[k], "cpu") else bs[k]
                assert itm[j] == its[k]
                assert np.array_equal(um[j * m.nv:(j + 1) * m.nv], u)
                single, rc1, it1, _ = s.solve(bv, rtol=1e-8)
                assert rc1 == asmg.ASMG_OK and abs(it1 - its[k]) <= 2
                if it1 == its[k]:
                    assert np.linalg.norm(single - u) <= 1e-9 * np.linalg.norm(single)
                u_ref, st_o, it_o, _ = o.solve(b, rtol=1e-8)
                tol = 1e-10 if precisions[p] == 0 else 1e-6
                vf = o.vertex_of_free()
                assert abs(its[k] - it_o) <= 2
                if precisions[p] == 0 and its[k] != it_o:
                    u_ref = oracle_iterate(m, b, its[k])
                assert np.linalg.norm(u[vf] - u_ref) <= tol * np.linalg.norm(u_ref)
                k += 1
    asmg.amg_batch_destroy(batch)
    for s in solvers:
        s.close()

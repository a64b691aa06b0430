"""The 3D workload at full size (129^3 jittered cube grid, 12,582,912 Kuhn
tetrahedra, 2,048,383 dofs, coefficient 1 or 1e3 on 8^3 subcubes, f = 1,
n_min = 6) in the launch configuration bench.py times (CUDA graph, PDL).

The oracle cannot build the 3D hierarchy at this size in test time, so
parity is checked on what it computes exactly here: the cluster tree
(bit-exact keys and permutation), sampled rows of the fine operator, the
load vector, and the true residual of the GPU solutions through the
oracle's FP64 operator.  The mixed and FP64 GPU solutions must also agree,
and the auxiliary hierarchy must have the sizes the construction fixes on
this dyadic grid: with one cell's six tetrahedra per leaf the finest
auxiliary grid is the 128^3 cell grid itself.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402


def test_kuhn_129_tree_operator_and_residuals(gen):
    from paper_1410_2153_gb300 import asmg
    m, f = gen.workload_3d(seed=1, nside=129)
    o = oracle.Oracle(m, stage=0, n_min=6)            # tree + fine operator only
    s = asmg.Solver(m, precision=asmg.ASMG_MIXED, n_min=6)
    assert np.array_equal(s.export("keys"), o.keys())
    assert np.array_equal(s.export("perm"), o.perm())
    # leaves are the 128^3 cells: J = 7, aux nodes = the 127^3 interior vertices
    assert s.info("J") == 7 and s.info("naux", 7) == 127 ** 3
    assert [s.info("naux", l) for l in range(8)] == [(2 ** l - 1) ** 3 for l in range(8)]
    A = o.A().tocsr()
    vf = o.vertex_of_free()
    t = s.export("fine_A")
    rng = np.random.default_rng(0)
    rows = set(rng.choice(vf, 2000, replace=False).tolist())
    sel = np.isin(t["row"], list(rows))
    pos = {int(v): i for i, v in enumerate(vf)}
    for r, c, v in zip(t["row"][sel], t["col"][sel], t["val"][sel]):
        ref = A[pos[int(r)], pos[int(c)]]
        assert abs(v - ref) <= 1e-12 * abs(A[pos[int(r)], pos[int(r)]])
    b = o.mass_apply(f)
    bg = s.mass_apply(torch.from_numpy(f).cuda()).cpu().numpy()
    assert np.abs(bg[vf] - b).max() <= 1e-13 * np.abs(b).max()
    bv = np.zeros(m.nv)
    bv[vf] = b
    db = torch.from_numpy(bv).cuda()
    u_mix, rc, it_mix, _ = s.solve(db, rtol=1e-8)
    assert rc == asmg.ASMG_OK
    s64 = asmg.Solver(m, precision=asmg.ASMG_FP64, n_min=6)
    u_64, rc, it_64, _ = s64.solve(db, rtol=1e-8)
    assert rc == asmg.ASMG_OK
    nb = np.linalg.norm(b)
    for u in (u_mix, u_64):
        uf = u.cpu().numpy()[vf]
        assert np.linalg.norm(b - o.spmv(uf)) <= 2e-8 * nb
    um, u6 = u_mix.cpu().numpy()[vf], u_64.cpu().numpy()[vf]
    assert np.linalg.norm(um - u6) <= 1e-5 * np.linalg.norm(u6)
    assert abs(it_mix - it_64) <= max(3, 0.1 * it_64)
    s.close()
    s64.close()

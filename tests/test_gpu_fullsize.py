"""The bench workload at full size (graded 2049^2: 4,190,209 dofs, 8,388,608
triangles), in the launch configuration bench.py times (CUDA graph, PDL).

The oracle cannot run the whole solve at this size in test time, so parity is
checked on what it can compute exactly here: the cluster tree (bit-exact:
keys, permutation, every depth's segments), sampled rows of the fine
operator, and the true residual of the GPU solutions through the oracle's
FP64 operator.  The mixed and FP64 GPU solutions must also agree.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402


def test_graded_2049_tree_operator_and_residuals(gen):
    from paper_1410_2153_gb300 import asmg
    m, f = gen.workload_graded(seed=1, nside=2049)
    o = oracle.Oracle(m, stage=0)                     # tree + fine operator only
    s = asmg.Solver(m, precision=asmg.ASMG_MIXED)
    # cluster tree: bit-exact
    assert np.array_equal(s.export("keys"), o.keys())
    assert np.array_equal(s.export("perm"), o.perm())
    segs = o.tree_levels()
    assert s.info("ntree_levels") == len(segs)
    for d, seg in enumerate(segs):
        assert np.array_equal(s.export("seg", d).reshape(-1, 4), seg), d
    # sampled rows of the fine operator
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
    # solves: true residual through the oracle's operator, FP64 vs mixed
    b = o.mass_apply(f)
    bv = np.zeros(m.nv)
    bv[vf] = b
    db = torch.from_numpy(bv).cuda()
    u_mix, rc, it_mix, _ = s.solve(db, rtol=1e-8)
    assert rc == asmg.ASMG_OK
    s64 = asmg.Solver(m, precision=asmg.ASMG_FP64)
    u_64, rc, it_64, _ = s64.solve(db, rtol=1e-8)
    assert rc == asmg.ASMG_OK
    nb = np.linalg.norm(b)
    for u in (u_mix, u_64):
        uf = u.cpu().numpy()[vf]
        assert np.linalg.norm(b - o.spmv(uf)) <= 2e-8 * nb
    um, u6 = u_mix.cpu().numpy()[vf], u_64.cpu().numpy()[vf]
    assert np.linalg.norm(um - u6) <= 1e-5 * np.linalg.norm(u6)
    assert abs(it_mix - it_64) <= 3
    s.close()
    s64.close()

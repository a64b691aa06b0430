"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Integer work (keys, sort permutation, tree, closure, auxiliary node sets,
colourings) must be bit-exact; floating point within the tolerances below.

Tolerances
  fine A, level operators   1e-12 of the row's largest entry (element sums in
                            a different order; Galerkin products vs
                            rediscretisation with averaged coefficients)
  transfer P                1e-11 absolute: rows reproduce constants, so
                            their scale is 1; psi_i grows like 1/|sigma_i| and
                            thin elements cost digits in the clipped integrals
  one B_co application      1e-11 relative (FP64)
  solution FP64             1e-10 relative, iterations within 2
  solution mixed            1e-6 relative to the FP64 oracle, iterations within 2
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from conftest import oracle_iterate  # noqa: E402


@pytest.fixture(scope="module")
def A():
    from paper_1410_2153_gb300 import asmg
    assert torch.cuda.is_available()
    asmg.lib()
    return asmg


def _meshes(gen):
    return {
        "poisson65": gen.workload_small_poisson(seed=1)[0],
        "graded129": gen.grid2d(129, 2, graded=True),
        "jitter97": gen.grid2d(97, 3),
    }


@pytest.fixture(scope="module")
def cases(gen, A):
    out = {}
    for name, m in _meshes(gen).items():
        out[name] = (m, oracle.Oracle(m), A.Solver(m, precision=A.ASMG_FP64))
    return out


def _spread(v):
    v = v.astype(np.uint64) & np.uint64(0xFFFFFFFF)
    for s, mk in ((16, 0x0000FFFF0000FFFF), (8, 0x00FF00FF00FF00FF), (4, 0x0F0F0F0F0F0F0F0F),
                  (2, 0x3333333333333333), (1, 0x5555555555555555)):
        v = (v | (v << np.uint64(s))) & np.uint64(mk)
    return v


@pytest.mark.parametrize("name", ["poisson65", "graded129", "jitter97"])
def test_tree_closure_aux_nodes_and_colours_bit_exact(cases, name):
    m, o, s = cases[name]
    assert np.array_equal(s.export("keys"), o.keys())
    assert np.array_equal(s.export("perm"), o.perm())
    segs = o.tree_levels()
    assert s.info("ntree_levels") == len(segs)
    for d, seg in enumerate(segs):
        assert np.array_equal(s.export("seg", d).reshape(-1, 4), seg), d
    for d, arr in enumerate(o.boxes()):
        sp = arr[arr[:, 1] == 1, 0]
        want = np.sort(_spread(sp & np.uint64(0xFFFFFFFF)) | (_spread(sp >> np.uint64(32)) << np.uint64(1)))
        assert np.array_equal(s.export("split", d), want), d
    assert s.info("J") == o.J and s.info("coarse") == o.c
    assert np.array_equal(s.export("aux_keys"), o.level_keys(o.J))
    for l in range(o.J + 1):
        assert s.info("naux", l) == o.info("nlevel", l)
    # colourings: fine grid and every smoothing set
    assert np.array_equal(s.export("fine_colour"), o.smoothing_set(-1)[2])
    for l in range(o.c + 1, o.J + 1):
        sm = s.export("smooth", l).reshape(-1, 2)
        osm, _, ocol = o.smoothing_set(l)
        keys = o.level_keys(l)
        want = sorted(zip(keys[osm].tolist(), ocol[osm].tolist()))
        got = sorted(zip(sm[:, 0].tolist(), sm[:, 1].tolist()))
        assert got == want, l


@pytest.mark.parametrize("name", ["poisson65", "graded129"])
def test_fine_operator_transfer_and_level_operators(cases, name):
    m, o, s = cases[name]
    vf = o.vertex_of_free()
    pos = {int(v): i for i, v in enumerate(vf)}
    Ao = o.A().toarray()
    t = s.export("fine_A")
    Ag = np.zeros_like(Ao)
    Ag[[pos[int(r)] for r in t["row"]], [pos[int(c)] for c in t["col"]]] = t["val"]
    assert np.abs(Ag - Ao).max() <= 1e-12 * np.abs(Ao).max()
    # Scott-Zhang transfer
    keys = o.level_keys(o.J)
    kpos = {int(k): i for i, k in enumerate(keys)}
    t = s.export("P")
    Pg = np.zeros((o.nfree, keys.size))
    Pg[[pos[int(r)] for r in t["row"]], [kpos[int(c)] for c in t["col"]]] = t["val"]
    assert np.abs(Pg - o.P().toarray()).max() <= 1e-11
    # level operators on the rows the V-cycle stores (smoothing rows: all
    # columns; other rows: smoothing columns) against the oracle's Galerkin A_l
    for l in range(o.c + 1, o.J + 1):
        lk = o.level_keys(l)
        lpos = {int(k): i for i, k in enumerate(lk)}
        Al = o.A(l).toarray()
        t = s.export("level_rows", l)
        osm = set(lk[o.smoothing_set(l)[0]].tolist())
        got = np.zeros_like(Al)
        mask = np.zeros(Al.shape, bool)
        for r, c, v in zip(t["row"], t["col"], t["val"]):
            got[lpos[int(r)], lpos[int(c)]] = v
        ins = np.array([int(k) in osm for k in lk])
        mask[ins, :] = True
        mask[:, ins] = True
        scale = np.abs(Al).max()
        assert np.abs((got - Al)[mask]).max() <= 1e-12 * scale, l


@pytest.mark.parametrize("name", ["poisson65", "graded129", "jitter97"])
def test_preconditioner_application_fp64(cases, name):
    m, o, s = cases[name]
    rng = np.random.default_rng(5)
    r = np.zeros(m.nv)
    vf = o.vertex_of_free()
    r[vf] = rng.uniform(-1, 1, o.nfree)
    z_ref = o.precond(r[vf])
    z = s.precond(torch.from_numpy(r).cuda()).cpu().numpy()
    assert np.linalg.norm(z[vf] - z_ref) <= 1e-11 * np.linalg.norm(z_ref)
    assert np.all(z[m.bflag == 1] == 0)


@pytest.mark.parametrize("name", ["poisson65", "graded129", "jitter97"])
def test_spmv_and_mass(cases, name):
    m, o, s = cases[name]
    rng = np.random.default_rng(6)
    vf = o.vertex_of_free()
    x = np.zeros(m.nv)
    x[vf] = rng.standard_normal(o.nfree)
    y = s.spmv(torch.from_numpy(x).cuda()).cpu().numpy()
    yr = o.spmv(x[vf])
    assert np.abs(y[vf] - yr).max() <= 1e-12 * np.abs(yr).max()
    f = rng.uniform(-1, 1, m.nv)
    b = s.mass_apply(torch.from_numpy(f).cuda()).cpu().numpy()
    br = o.mass_apply(f)
    assert np.abs(b[vf] - br).max() <= 1e-13 * np.abs(br).max()
    # fixed-order gather: the same bits on a second call
    b2 = s.mass_apply(torch.from_numpy(f).cuda()).cpu().numpy()
    assert np.array_equal(b, b2)


@pytest.mark.parametrize("name", ["poisson65", "graded129", "jitter97"])
@pytest.mark.parametrize("graph", [1, 0])
def test_solve_fp64_matches_oracle(cases, gen, A, name, graph):
    m, o, _ = cases[name]
    s = A.Solver(m, precision=A.ASMG_FP64, use_graph=graph)
    f = gen.nodal_uniform(m, 11)
    vf = o.vertex_of_free()
    b_ref = o.mass_apply(f)
    u_ref, st, it_ref, hist_ref = o.solve(b_ref, rtol=1e-8)
    b = s.mass_apply(torch.from_numpy(f).cuda())
    u, rc, it, hist = s.solve(b, rtol=1e-8)
    u = u.cpu().numpy()
    assert rc == A.ASMG_OK and st == 0
    assert abs(it - it_ref) <= 2, (it, it_ref)
    u_same = u_ref if it == it_ref else oracle_iterate(m, b_ref, it)
    assert np.linalg.norm(u[vf] - u_same) <= 1e-10 * np.linalg.norm(u_same)
    assert np.all(u[m.bflag == 1] == 0)
    # the residual history is the recurrence residual: it ends below rtol
    assert hist[-1] <= 1e-8 * np.linalg.norm(b_ref) * (1 + 1e-12)
    # true residual through the oracle's operator
    assert np.linalg.norm(b_ref - o.spmv(u[vf])) <= 2e-8 * np.linalg.norm(b_ref)
    s.close()


@pytest.mark.parametrize("name", ["poisson65", "graded129", "jitter97"])
def test_solve_mixed_matches_fp64_oracle(cases, gen, A, name):
    m, o, _ = cases[name]
    s = A.Solver(m, precision=A.ASMG_MIXED)
    f = gen.nodal_uniform(m, 12)
    vf = o.vertex_of_free()
    b_ref = o.mass_apply(f)
    u_ref, st, it_ref, _ = o.solve(b_ref, rtol=1e-8)
    u, rc, it, hist = s.solve(s.mass_apply(torch.from_numpy(f).cuda()), rtol=1e-8)
    u = u.cpu().numpy()
    assert rc == A.ASMG_OK
    assert abs(it - it_ref) <= 2, (it, it_ref)
    assert np.linalg.norm(u[vf] - u_ref) <= 1e-6 * np.linalg.norm(u_ref)
    s.close()


def test_host_buffers_and_warm_start(cases, gen, A):
    m, o, s = cases["poisson65"]
    f = gen.nodal_uniform(m, 13)
    b = s.mass_apply(f)                    # host arrays through the same calls
    u, rc, it, _ = s.solve(b, rtol=1e-10)
    assert rc == A.ASMG_OK
    u2, rc2, it2, hist2 = s.solve(b, u0=u, rtol=1e-8)
    assert rc2 == A.ASMG_OK and it2 == 0 and hist2.size == 1
    # non-convergence is reported with the last iterate
    s2 = A.Solver(m, max_iter=2)
    u3, rc3, it3, hist3 = s2.solve(b, rtol=1e-14)
    assert rc3 == A.ASMG_NOT_CONVERGED and it3 == 2 and hist3.size == 3
    s2.close()


def test_zero_rhs_and_empty_aux(gen, A):
    m = gen.grid2d(3, 1)        # one free vertex
    s = A.Solver(m)
    u, rc, it, hist = s.solve(np.zeros(m.nv), rtol=1e-8)
    assert rc == A.ASMG_OK and it == 0 and np.all(u == 0)
    b = np.zeros(m.nv)
    b[4] = 1.0
    u, rc, it, _ = s.solve(b, rtol=1e-12)
    assert rc == A.ASMG_OK
    o = oracle.Oracle(m)
    assert abs(u[4] - 1.0 / o.A().toarray()[0, 0]) < 1e-14
    s.close()


@pytest.mark.parametrize("nside", [9, 17, 129])
def test_3d_cluster_tree_bit_exact(gen, A, nside):
    # Kuhn tetrahedra of a jittered cube grid; 129^3 vertices is the 3D
    # workload at full size (12,582,912 tetrahedra)
    m = gen.grid3d(nside, 4, jitter=0.15)
    keys, perm = A.amg_cluster_tree(m)
    o = oracle.Oracle(m, stage=-1)
    assert np.array_equal(keys, o.keys())
    assert np.array_equal(perm, o.perm())

"""Mixed Dirichlet / Neumann boundaries on the GPU against the oracle.

A vertex flagged 2 is a Neumann vertex: an unknown of the fine problem, with
the natural boundary condition.  The auxiliary grids are then the mixed grids
of the remark in Sec. 3.4 (simplices that meet the domain and not the
Dirichlet boundary Gamma_D), every level is smoothed as a whole, and each
level of the V-cycle adds the near-boundary correction of Algorithm 3 (the
exact solve on J_{l,j}, Sec. 3.5) after its coarse-grid correction.  The
library runs that solve on the device by block cyclic reduction; the oracle
by a dense Cholesky factor.

Integer work (level sizes, smoothing sets, colours) must be bit-exact.
Floating point: one B application 1e-11 relative in 2D; FP64 solutions
1e-10 relative with iterations within 2; mixed solutions 1e-6 relative to
the FP64 oracle, iterations within 2.  In 3D the coverage of the cut
tetrahedra comes from two different exact clippers (as for the Dirichlet
grids of non-box domains), so one B application is held to 1e-9 and FP64
solutions to 1e-8 there.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from conftest import oracle_iterate  # noqa: E402


def _neumann(m, mask):
    m.bflag = m.bflag.copy()
    m.bflag[mask] = 2
    return m


def _meshes(gen):
    out = {}
    m = gen.grid2d(65, 1)
    x, y = m.verts[:, 0], m.verts[:, 1]
    out["square65_right"] = (_neumann(m, (x == 1.0) & (y > 0) & (y < 1)), {})
    m = gen.grid2d_domain(65, 2, "L")
    x, y = m.verts[:, 0], m.verts[:, 1]
    out["L65_cut"] = (_neumann(m, (m.bflag == 1) & (x > 0) & (x < 1) & (y > 0) & (y < 1)), {"coarse_max": 8})
    m = gen.grid2d_domain(65, 2, "hole")
    x, y = m.verts[:, 0], m.verts[:, 1]
    m = _neumann(m, (m.bflag == 1) & (x == 0) & (y > 0) & (y < 1))
    m.coeff = np.exp(np.random.default_rng(4).normal(size=m.ne))
    out["hole65_left_lognormal"] = (m, {"coarse_max": 8})
    m = gen.grid2d(65, 5, graded=True)
    x, y = m.verts[:, 0], m.verts[:, 1]
    out["graded65_two_sides_nb3"] = (_neumann(m, ((x == 1.0) | (y == 1.0)) & (x > 0) & (y > 0)),
                                     {"coarse_max": 16, "nb_layers": 3})
    m = gen.grid2d_domain(65, 3, "L")
    x, y = m.verts[:, 0], m.verts[:, 1]
    out["L65_cut_nb_off"] = (_neumann(m, (m.bflag == 1) & (x > 0) & (x < 1) & (y > 0) & (y < 1)),
                             {"coarse_max": 8, "nb_layers": -1})
    m = gen.grid3d(9, 1)
    x = m.verts
    out["cube9_face"] = (_neumann(m, (x[:, 0] == 1.0) & (x[:, 1] > 0) & (x[:, 1] < 1) & (x[:, 2] > 0) & (x[:, 2] < 1)),
                         {"coarse_max": 8})
    m = gen.grid3d_domain(7, 3, "L")
    x = m.verts
    out["Lprism7_neumann_cut"] = (_neumann(m, (m.bflag == 1) & (x[:, 0] > 0) & (x[:, 0] < 1) & (x[:, 1] > 0)
                                           & (x[:, 1] < 1)), {"coarse_max": 8})
    return out


NAMES = ["square65_right", "L65_cut", "hole65_left_lognormal", "graded65_two_sides_nb3", "L65_cut_nb_off",
         "cube9_face", "Lprism7_neumann_cut"]


@pytest.fixture(scope="module")
def cases(gen):
    from paper_1410_2153_gb300 import asmg
    out = {}
    for name, (m, po) in _meshes(gen).items():
        pl = {("coarse_max_dofs" if k == "coarse_max" else k): v for k, v in po.items()}
        out[name] = (m, oracle.Oracle(m, **po), asmg.Solver(m, precision=asmg.ASMG_FP64, **pl), pl, po)
    return out


@pytest.mark.parametrize("name", NAMES)
def test_mixed_levels_smoothing_sets_and_colours_bit_exact(cases, name):
    m, o, s, p, po = cases[name]
    assert np.any(m.bflag == 2)
    assert s.info("J") == o.J and s.info("coarse") == o.c
    for l in range(o.J + 1):
        assert s.info("naux", l) == o.info("nlevel", l), l
    assert np.array_equal(s.export("fine_colour"), o.smoothing_set(-1)[2])
    for l in range(o.c + 1, o.J + 1):
        sm = s.export("smooth", l).reshape(-1, 2)
        osm, _, ocol = o.smoothing_set(l)
        keys = o.level_keys(l)
        assert sorted(zip(sm[:, 0].tolist(), sm[:, 1].tolist())) == sorted(zip(keys[osm].tolist(),
                                                                                ocol[osm].tolist())), l


@pytest.mark.parametrize("name", NAMES)
def test_mixed_preconditioner_application(cases, name):
    m, o, s, p, po = cases[name]
    rng = np.random.default_rng(5)
    vf = o.vertex_of_free()
    r = np.zeros(m.nv)
    r[vf] = rng.uniform(-1, 1, o.nfree)
    z_ref = o.precond(r[vf])
    z = s.precond(torch.from_numpy(r).cuda()).cpu().numpy()
    tol = 1e-11 if m.dim == 2 else 1e-9
    assert np.linalg.norm(z[vf] - z_ref) <= tol * np.linalg.norm(z_ref)
    assert np.all(z[m.bflag == 1] == 0)
    assert np.any(z[m.bflag == 2] != 0)


@pytest.mark.parametrize("name", NAMES)
def test_mixed_solves_match_oracle(cases, gen, name):
    from paper_1410_2153_gb300 import asmg
    m, o, s, p, po = cases[name]
    f = gen.nodal_uniform(m, 17)
    vf = o.vertex_of_free()
    b_ref = o.mass_apply(f)
    u_ref, st, it_ref, _ = o.solve(b_ref, rtol=1e-8)
    assert st == 0
    u, rc, it, _ = s.solve(s.mass_apply(torch.from_numpy(f).cuda()), rtol=1e-8)
    u = u.cpu().numpy()
    assert rc == asmg.ASMG_OK and abs(it - it_ref) <= 2, (it, it_ref)
    u_same = u_ref if it == it_ref else oracle_iterate(m, b_ref, it, **po)
    tol = 1e-10 if m.dim == 2 else 1e-8
    assert np.linalg.norm(u[vf] - u_same) <= tol * np.linalg.norm(u_same)
    assert np.all(u[m.bflag == 1] == 0)
    sm = asmg.Solver(m, precision=asmg.ASMG_MIXED, **p)
    u2, rc2, it2, _ = sm.solve(sm.mass_apply(torch.from_numpy(f).cuda()), rtol=1e-8)
    u2 = u2.cpu().numpy()
    assert rc2 == asmg.ASMG_OK and abs(it2 - it_ref) <= 2, (it2, it_ref)
    assert np.linalg.norm(u2[vf] - u_ref) <= 1e-6 * np.linalg.norm(u_ref)
    sm.close()

"""Variants of the preconditioner and of the outer iteration against the
oracle: the Jacobi smoother S = D^{-1} (Sec. 4.1), the additive form
B = S + Pi Btilde Pi^t (eq. fasp), several fine smoothing steps per
application, and the ASMG iteration u <- u + B (b - A u) (Sec. 5.1).

Tolerances as in the parity tests: one B application 1e-11 relative (FP64),
FP64 solutions 1e-10 relative (1e-9 for the Jacobi forms, whose ~60 flexible
CG steps on the graded mesh carry the ~1e-14 differences of the clipped
transfer entries), mixed solutions 1e-6.  Iterations within 2; with the
undamped Jacobi smoother on the graded mesh B is far from the ideal
preconditioner and the flexible CG's step count is sensitive to rounding, so
a larger difference is accepted only with the check of
conftest.mixed_iterations_ok (the solution as close to the oracle's
rtol-1e-13 solve as the oracle's own).  Residual histories of the ASMG
iteration agree to 1e-9 relative, or to 1e-13 of the first residual where
they reach the rounding floor of b - A x.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from conftest import mixed_iterations_ok, oracle_iterate  # noqa: E402

VARIANTS = {  # (smoother, additive, fine_sweeps)
    "jacobi": (1, 0, 1),
    "additive_gs": (0, 1, 1),
    "additive_jacobi_2": (1, 1, 2),
    "gs_2": (0, 0, 2),
}


def _mesh(gen, name):
    if name == "kuhn9":
        return gen.grid3d(9, 2)
    if name == "graded65":
        return gen.grid2d(65, 2, graded=True)
    return gen.grid2d(97, 3)


@pytest.mark.parametrize("mesh", ["jitter97", "graded65", "kuhn9"])
@pytest.mark.parametrize("variant", list(VARIANTS))
def test_variant_preconditioner_and_solve(gen, mesh, variant):
    from paper_1410_2153_gb300 import asmg
    sm, add, fs = VARIANTS[variant]
    m = _mesh(gen, mesh)
    o = oracle.Oracle(m, smoother=sm, additive=add, fine_sweeps=fs)
    s = asmg.Solver(m, precision=asmg.ASMG_FP64, smoother=sm, additive=add, fine_sweeps=fs)
    vf = o.vertex_of_free()
    rng = np.random.default_rng(7)
    r = np.zeros(m.nv)
    r[vf] = rng.uniform(-1, 1, o.nfree)
    z_ref = o.precond(r[vf])
    z = s.precond(torch.from_numpy(r).cuda()).cpu().numpy()
    assert np.linalg.norm(z[vf] - z_ref) <= 1e-11 * np.linalg.norm(z_ref)
    f = gen.nodal_uniform(m, 11)
    b_ref = o.mass_apply(f)
    u_ref, st, it_ref, _ = o.solve(b_ref, rtol=1e-8)
    assert st == 0
    # the oracle's load vector on both sides (the Jacobi forms amplify any
    # rounding difference of the right-hand side)
    bv = np.zeros(m.nv)
    bv[vf] = b_ref
    u, rc, it, _ = s.solve(torch.from_numpy(bv).cuda(), rtol=1e-8)
    u = u.cpu().numpy()
    pr = dict(smoother=sm, additive=add, fine_sweeps=fs)
    assert rc == asmg.ASMG_OK
    ok, msg = mixed_iterations_ok(m, b_ref, it, it_ref, u[vf], **pr)
    assert ok, msg
    u_same = u_ref if it == it_ref else oracle_iterate(m, b_ref, it, **pr)
    tol = 1e-9 if sm == 1 else 1e-10
    assert np.linalg.norm(u[vf] - u_same) <= tol * np.linalg.norm(u_same)
    s.close()
    sm32 = asmg.Solver(m, precision=asmg.ASMG_MIXED, smoother=sm, additive=add, fine_sweeps=fs)
    u2, rc2, it2, _ = sm32.solve(sm32.mass_apply(torch.from_numpy(f).cuda()), rtol=1e-8)
    u2 = u2.cpu().numpy()
    assert rc2 == asmg.ASMG_OK
    ok, msg = mixed_iterations_ok(m, b_ref, it2, it_ref, u2[vf], **pr)
    assert ok, msg
    assert np.linalg.norm(u2[vf] - u_ref) <= 1e-6 * np.linalg.norm(u_ref)
    sm32.close()


@pytest.mark.parametrize("mesh,smoother", [("jitter97", 0), ("jitter97", 1), ("kuhn9", 0)])
@pytest.mark.parametrize("graph", [1, 0])
def test_asmg_iteration_matches_oracle(gen, mesh, smoother, graph):
    from paper_1410_2153_gb300 import asmg
    m = _mesh(gen, mesh)
    o = oracle.Oracle(m, smoother=smoother, iteration=1)
    s = asmg.Solver(m, precision=asmg.ASMG_FP64, smoother=smoother, iteration=1, use_graph=graph)
    vf = o.vertex_of_free()
    f = gen.nodal_uniform(m, 12)
    b_ref = o.mass_apply(f)
    u_ref, st, it_ref, hist_ref = o.solve(b_ref, rtol=1e-8)
    assert st == 0
    u, rc, it, hist = s.solve(s.mass_apply(torch.from_numpy(f).cuda()), rtol=1e-8)
    u = u.cpu().numpy()
    assert rc == asmg.ASMG_OK and it == it_ref, (it, it_ref)
    # the residual history is the true residual of every iterate
    assert np.all(np.abs(hist - hist_ref) <= 1e-9 * hist_ref + 1e-13 * hist_ref[0])
    assert np.linalg.norm(u[vf] - u_ref) <= 1e-10 * np.linalg.norm(u_ref)
    s.close()
    # not converged within max_iter: last iterate and the history are returned
    s2 = asmg.Solver(m, precision=asmg.ASMG_FP64, smoother=smoother, iteration=1, max_iter=2)
    u3, rc3, it3, hist3 = s2.solve(s2.mass_apply(torch.from_numpy(f).cuda()), rtol=1e-14)
    assert rc3 == asmg.ASMG_NOT_CONVERGED and it3 == 2 and hist3.size == 3
    s2.close()


def test_asmg_iteration_divergence_reported(gen):
    # with the undamped Jacobi smoother on the 3D grid lambda_max(BA) > 2, so the
    # ASMG iteration diverges; both sides must report it, not return a solution
    from paper_1410_2153_gb300 import asmg
    m = _mesh(gen, "kuhn9")
    o = oracle.Oracle(m, smoother=1, iteration=1)
    s = asmg.Solver(m, precision=asmg.ASMG_FP64, smoother=1, iteration=1)
    f = gen.nodal_uniform(m, 12)
    _, st, _, hist_ref = o.solve(o.mass_apply(f), rtol=1e-8)
    assert st != 0
    try:
        _, rc, it, hist = s.solve(s.mass_apply(torch.from_numpy(f).cuda()), rtol=1e-8)
        assert rc == asmg.ASMG_NOT_CONVERGED and hist[-1] > hist[0]
    except asmg.AsmgError as e:          # the residual overflowed
        assert e.code == asmg.ASMG_ERR_BREAKDOWN
    s.close()

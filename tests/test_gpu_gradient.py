"""Differentiable coefficient inversion on the GPU against the oracle.

Loss L = 1/2 ||u(a) - u_obs||^2 with a = exp(g), g a Gaussian random field
(workload_inverse).  Tolerances: gradient vs the oracle's gradient 1e-8
relative (FP64) and 1e-5 (mixed) at the same rtol; vs central differences
(step 1e-6 in g_e, FP64 oracle solves at rtol 1e-14 warm-started from u)
1e-6 of the largest gradient entry.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402


@pytest.fixture(scope="module")
def inv(gen):
    m, g, g_obs = gen.workload_inverse(seed=3, nside=65)
    f = gen.nodal_uniform(m, 31)
    o = oracle.Oracle(m)
    b_free = o.mass_apply(f)
    m_obs = gen.grid2d(65, 3)
    m_obs.coeff = np.exp(g_obs)
    u_obs_free, st, _, _ = oracle.Oracle(m_obs).solve(b_free, rtol=1e-14)
    assert st == 0
    return m, g, f, o, b_free, u_obs_free


def _vertex(m, o, x_free):
    v = np.zeros(m.nv)
    v[o.vertex_of_free()] = x_free
    return v


def test_element_gradient_kernel_matches_oracle(inv):
    from paper_1410_2153_gb300 import asmg
    m, g, f, o, b_free, u_obs = inv
    s = asmg.Solver(m)
    rng = np.random.default_rng(4)
    u = rng.standard_normal(o.nfree)
    lam = rng.standard_normal(o.nfree)
    got = s.element_grad(torch.from_numpy(_vertex(m, o, u)).cuda(), torch.from_numpy(_vertex(m, o, lam)).cuda())
    want = o.elem_grad(u, lam)
    assert np.abs(got.cpu().numpy() - want).max() <= 1e-12 * np.abs(want).max()
    # log-parametrisation: a = exp(g) set in the library, dL/dg = a dL/da in the kernel
    asmg.amg_set_log_coefficients(s.h, torch.from_numpy(g).cuda())
    got_g = s.element_grad_log(torch.from_numpy(_vertex(m, o, u)).cuda(), torch.from_numpy(_vertex(m, o, lam)).cuda())
    want_g = np.exp(g) * want
    assert np.abs(got_g.cpu().numpy() - want_g).max() <= 1e-12 * np.abs(want_g).max()
    s.close()


@pytest.mark.parametrize("precision,tol", [(0, 1e-8), (1, 1e-5)])
def test_inversion_gradient_matches_oracle(inv, precision, tol):
    from paper_1410_2153_gb300 import autograd as ag
    m, g, f, o, b_free, u_obs = inv
    rtol = 1e-8
    cs = ag.CoefficientSolver(m, precision=precision, rtol=rtol)
    b = torch.from_numpy(_vertex(m, o, b_free)).cuda()
    uo = torch.from_numpy(_vertex(m, o, u_obs)).cuda()
    loss, dLdg, u = ag.inversion_loss_and_grad(cs, torch.from_numpy(g).cuda(), b, uo)
    # oracle: forward, adjoint, element formula, chain rule through a = exp(g)
    u_ref, st, _, _ = o.solve(b_free, rtol=rtol)
    lam_ref, st2, _, _ = o.solve(u_ref - u_obs, rtol=rtol)
    ref = np.exp(g) * o.elem_grad(u_ref, lam_ref)
    got = dLdg.cpu().numpy()
    assert np.linalg.norm(got - ref) <= tol * np.linalg.norm(ref)
    assert abs(loss.item() - 0.5 * np.sum((u_ref - u_obs) ** 2)) <= tol * loss.item()
    assert len(cs.last_iterations) == 2     # one forward and one adjoint solve


def test_inversion_gradient_central_differences(inv, gen):
    from paper_1410_2153_gb300 import autograd as ag
    m, g, f, o, b_free, u_obs = inv
    cs = ag.CoefficientSolver(m, precision=0, rtol=1e-12)
    b = torch.from_numpy(_vertex(m, o, b_free)).cuda()
    uo = torch.from_numpy(_vertex(m, o, u_obs)).cuda()
    loss, dLdg, u = ag.inversion_loss_and_grad(cs, torch.from_numpy(g).cuda(), b, uo)
    dLdg = dLdg.cpu().numpy()
    u_free = u.cpu().numpy()[o.vertex_of_free()]
    rng = np.random.default_rng(9)
    h = 1e-6
    for e in rng.choice(m.ne, 12, replace=False):
        ups = []
        for sgn in (1, -1):
            mm = gen.grid2d(65, 3)
            mm.coeff = np.exp(g + sgn * h * (np.arange(m.ne) == e))
            ups.append(oracle.Oracle(mm).solve(b_free, rtol=1e-14, u0=u_free)[0])
        fd = 0.5 * (ups[0] - ups[1]) @ (ups[0] + ups[1] - 2 * u_obs) / (2 * h)
        assert abs(fd - dLdg[e]) <= 1e-6 * np.abs(dLdg).max(), (e, fd, dLdg[e])


def test_rhs_gradient_is_adjoint_solution(inv):
    from paper_1410_2153_gb300 import autograd as ag
    m, g, f, o, b_free, u_obs = inv
    cs = ag.CoefficientSolver(m, precision=0, rtol=1e-12)
    b = torch.from_numpy(_vertex(m, o, b_free)).cuda().requires_grad_(True)
    a = torch.from_numpy(np.exp(g)).cuda()
    u = ag.SolveFn.apply(a, b, cs)
    w = torch.from_numpy(np.random.default_rng(2).standard_normal(m.nv)).cuda()
    (u * w).sum().backward()
    # dL/db = A^{-1} w on free vertices (A symmetric), 0 on Dirichlet ones
    lam_ref, st, _, _ = o.solve(w.cpu().numpy()[o.vertex_of_free()], rtol=1e-14)
    got = b.grad.cpu().numpy()
    assert np.linalg.norm(got[o.vertex_of_free()] - lam_ref) <= 1e-9 * np.linalg.norm(lam_ref)
    assert np.all(got[m.bflag == 1] == 0)

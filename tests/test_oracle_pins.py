"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

None of these compares the oracle with itself: each check is a closed form,
an invariant the paper states, a library routine for a special case, or a
brute-force recomputation by a different characterisation.
"""
import math
from fractions import Fraction

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import oracle
from oracle import lattice_xy

D2 = 31
TOP = 1 << D2


def _grid(gen, n, **kw):
    return gen.grid2d(n, kw.pop("seed", 1), **kw)


# --------------------------------------------------------------------------
# Sec. 2: stiffness and mass
# --------------------------------------------------------------------------

def test_stiffness_is_five_point_laplacian_on_right_triangles(gen):
    # Textbook identity: P1 on a uniform grid of SW-NE right triangles gives
    # the 5-point stencil [4; -1 -1 -1 -1], independent of h.
    n = 9
    m = _grid(gen, n, jitter=0.0, random_diag=False)
    o = oracle.Oracle(m, stage=0)
    A = o.A().toarray()
    m1 = n - 2
    T = sp.diags([-1.0, 2.0, -1.0], [-1, 0, 1], shape=(m1, m1))
    L5 = (sp.kron(sp.eye(m1), T) + sp.kron(T, sp.eye(m1))).toarray()
    assert np.abs(A - L5).max() < 1e-13


def test_stiffness_annihilates_linears_on_interior_rows(gen):
    m = _grid(gen, 17, seed=3)
    o = oracle.Oracle(m, stage=0)
    A = o.A()
    vf = o.vertex_of_free()
    x, y = m.verts[vf, 0], m.verts[vf, 1]
    # rows whose stencil touches no Dirichlet vertex
    interior = np.ones(o.nfree, bool)
    bnd = set(np.nonzero(m.bflag)[0].tolist())
    for e in m.elems:
        if any(int(v) in bnd for v in e):
            for v in e:
                if m.bflag[v] == 0:
                    interior[np.searchsorted(vf, v)] = False
    for g in (np.ones_like(x), x, y, 2.0 - 3.0 * x + 0.5 * y):
        r = A @ g
        assert np.abs(r[interior]).max() < 1e-11
    As = A.toarray()
    assert np.abs(As - As.T).max() < 1e-14
    assert np.linalg.eigvalsh(As).min() > 0


def test_mass_matrix_integrates_products_exactly(gen):
    # With every vertex free, 1^T M 1 = |Omega|, 1^T M x = 1/2, y^T M x = 1/4.
    m = _grid(gen, 9, seed=2)
    m.bflag[:] = 0
    o = oracle.Oracle(m, stage=0)
    x, y = m.verts[:, 0], m.verts[:, 1]
    assert abs(o.mass_apply(np.ones(m.nv)).sum() - 1.0) < 1e-14
    assert abs(o.mass_apply(x).sum() - 0.5) < 1e-14
    assert abs(o.mass_apply(x) @ y - 0.25) < 1e-14


# --------------------------------------------------------------------------
# Sec. 5 / C11: PCG solution
# --------------------------------------------------------------------------

def test_pcg_matches_dense_cholesky(gen):
    m = _grid(gen, 12, seed=4)
    f = gen.nodal_uniform(m, 7)
    o = oracle.Oracle(m)
    b = o.mass_apply(f)
    u, st, it, hist = o.solve(b, rtol=1e-14)
    ref = np.linalg.solve(o.A().toarray(), b)
    assert st == 0
    assert np.linalg.norm(u - ref) <= 1e-12 * np.linalg.norm(ref)
    assert hist[-1] <= 1e-14 * np.linalg.norm(b)


def _l2_error(m, vf, u_free):
    u = np.zeros(m.nv)
    u[vf] = u_free
    err2 = 0.0
    V = m.verts
    for k in range(3):
        a, b = m.elems[:, k], m.elems[:, (k + 1) % 3]
        mid = 0.5 * (V[a] + V[b])
        uh = 0.5 * (u[a] + u[b])
        ue = np.sin(math.pi * mid[:, 0]) * np.sin(math.pi * mid[:, 1])
        p0, p1, p2 = V[m.elems[:, 0]], V[m.elems[:, 1]], V[m.elems[:, 2]]
        area = 0.5 * ((p1[:, 0] - p0[:, 0]) * (p2[:, 1] - p0[:, 1]) - (p2[:, 0] - p0[:, 0]) * (p1[:, 1] - p0[:, 1]))
        err2 += (area / 3.0 * (uh - ue) ** 2).sum()
    return math.sqrt(err2)


def test_manufactured_solution_converges_at_second_order(gen):
    errs = []
    for n in (17, 33, 65, 129):
        m, f = gen.workload_small_poisson(seed=1, nside=n)
        o = oracle.Oracle(m)
        u, st, it, _ = o.solve(o.mass_apply(f), rtol=1e-12)
        assert st == 0
        errs.append(_l2_error(m, o.vertex_of_free(), u))
    ratios = [errs[i] / errs[i + 1] for i in range(3)]
    assert all(3.3 < r < 4.8 for r in ratios), (errs, ratios)


def test_iterations_grow_at_most_logarithmically(gen):
    # Sec. 4: kappa(BA) <~ log N; Sec. 5: PCG steps flat in N (5 at 4 sizes).
    its = []
    for n in (17, 33, 65, 129, 257):
        m = gen.grid2d(n, 1)
        o = oracle.Oracle(m)
        _, st, it, _ = o.solve(o.mass_apply(gen.nodal_uniform(m, 5)), rtol=1e-8)
        assert st == 0
        its.append(it)
    assert its[-1] <= its[0] + 4, its
    assert max(its) <= 12, its


def test_standalone_asmg_rate(gen):
    # Sec. 5 (Fig. rate_Dirichlet): ASMG as a stationary iteration reduces the
    # residual by roughly 0.4 per step, level independently.
    for n in (33, 65):
        m = gen.grid2d(n, 2)
        o = oracle.Oracle(m)
        A = o.A()
        b = o.mass_apply(gen.nodal_uniform(m, 3))
        u = np.zeros(o.nfree)
        rn = [np.linalg.norm(b)]
        for _ in range(12):
            u = u + o.precond(b - A @ u)
            rn.append(np.linalg.norm(b - A @ u))
        rate = (rn[-1] / rn[4]) ** (1.0 / 8.0)
        assert rate < 0.5, rate


# --------------------------------------------------------------------------
# Sec. 3.1: cluster tree
# --------------------------------------------------------------------------

def _check_tree(m, o, n_min=3):
    levels = o.tree_levels()
    perm = o.perm()
    a0, a1, _, L = o.root()
    bc = m.verts[m.elems].sum(1) / 3.0
    assert np.array_equal(np.sort(perm), np.arange(m.ne))
    keys = o.keys()
    ks = keys[perm]
    assert (np.diff(ks.astype(np.float64)) >= 0).all()
    eq = ks[1:] == ks[:-1]
    assert (perm[1:][eq] > perm[:-1][eq]).all()   # stable: ties by element index
    for d, segs in enumerate(levels):
        w = L / 2 ** d
        for prefix, b, e, split in segs:
            q = np.zeros(2, np.int64)
            for j in range(d):
                q[0] |= ((int(prefix) >> (2 * j)) & 1) << j
                q[1] |= ((int(prefix) >> (2 * j + 1)) & 1) << j
            lo = np.array([a0 + q[0] * w, a1 + q[1] * w])
            pts = bc[perm[b:e]]
            tol = 1e-12 * L
            assert (pts >= lo - tol).all() and (pts <= lo + w + tol).all()
            if split:
                assert e - b > n_min
            elif d < 31:
                assert e - b <= n_min
        if d + 1 < len(levels):
            ch = levels[d + 1]
            nsplit = int(segs[:, 3].sum())
            assert ch.shape[0] == 4 * nsplit   # all four children, empty ones too
    return levels


def test_cluster_tree_membership_and_counts(gen):
    for m in (gen.grid2d(17, 3), gen.grid2d(33, 4, graded=True)):
        o = oracle.Oracle(m, stage=0)
        _check_tree(m, o)


def test_cluster_tree_depth_bound(gen):
    # Lemma (Sec. 3.1): a split node at depth l satisfies h <= 2^-l sqrt(2) L,
    # h the minimal barycenter distance, so the depth is <= log2(sqrt2 L/h)+1.
    from scipy.spatial import cKDTree
    m = gen.grid2d(33, 5, graded=True)
    o = oracle.Oracle(m, stage=0)
    bc = m.verts[m.elems].mean(1)
    dist, _ = cKDTree(bc).query(bc, k=2)
    h = dist[:, 1].min()
    L = o.root()[3]
    depth = len(o.tree_levels()) - 1
    assert depth <= math.floor(math.log2(math.sqrt(2) * L / h)) + 1


# --------------------------------------------------------------------------
# Sec. 3.2: closure
# --------------------------------------------------------------------------

def _unpack(p):
    return int(p) & 0xFFFFFFFF, int(p) >> 32


def _minimal_balanced_by_neighbour_rule(o):
    """Different characterisation of the edge-2:1 balanced refinement: a tree
    is balanced iff every split box has all four same-depth edge neighbours.
    Close the cluster tree's split set under that rule with a worklist."""
    split = set()
    for d, segs in enumerate(o.tree_levels()):
        for prefix, b, e, s in segs:
            if s:
                q = [0, 0]
                for j in range(d):
                    q[0] |= ((int(prefix) >> (2 * j)) & 1) << j
                    q[1] |= ((int(prefix) >> (2 * j + 1)) & 1) << j
                split.add((d, q[0], q[1]))
    work = list(split)
    while work:
        d, x, y = work.pop()
        # ancestors must be split
        if d > 0 and (d - 1, x // 2, y // 2) not in split:
            split.add((d - 1, x // 2, y // 2))
            work.append((d - 1, x // 2, y // 2))
        for dx, dy in ((1, 0), (-1, 0), (0, 1), (0, -1)):
            nx, ny = x + dx, y + dy
            if not (0 <= nx < 2 ** d and 0 <= ny < 2 ** d) or d == 0:
                continue
            par = (d - 1, nx // 2, ny // 2)
            if par not in split:
                split.add(par)
                work.append(par)
    return split


def test_closure_is_minimal_balanced_refinement(gen):
    for m in (gen.grid2d(33, 6, graded=True), gen.grid2d(17, 7, graded=True)):
        o = oracle.Oracle(m, stage=1)
        got = set()
        allboxes = set()
        for d, arr in enumerate(o.boxes()):
            for p, s in arr:
                x, y = _unpack(p)
                allboxes.add((d, x, y))
                if s:
                    got.add((d, x, y))
        assert got == _minimal_balanced_by_neighbour_rule(o)
        # every split box has its four children; every non-root box its parent
        for d, x, y in got:
            for c in range(4):
                assert (d + 1, 2 * x + (c & 1), 2 * y + (c >> 1)) in allboxes
        for d, x, y in allboxes:
            if d:
                assert (d - 1, x // 2, y // 2) in got


def test_closure_leaves_are_edge_balanced_by_brute_force(gen):
    m = gen.grid2d(17, 8, graded=True)
    o = oracle.Oracle(m, stage=1)
    leaves = []
    for d, arr in enumerate(o.boxes()):
        for p, s in arr:
            if not s:
                x, y = _unpack(p)
                w = 1 << (D2 - d)
                leaves.append((d, x * w, y * w, w))
    for i, (d1, x1, y1, w1) in enumerate(leaves):
        for d2, x2, y2, w2 in leaves[i + 1:]:
            # shared edge of positive length?
            ox = min(x1 + w1, x2 + w2) - max(x1, x2)
            oy = min(y1 + w1, y2 + w2) - max(y1, y2)
            if (ox == 0 and oy > 0) or (oy == 0 and ox > 0):
                assert abs(d1 - d2) <= 1


# --------------------------------------------------------------------------
# Sec. 3.3: auxiliary triangulations
# --------------------------------------------------------------------------

def _tri_xy(tri):
    x, y = lattice_xy(tri.reshape(-1))
    return x.reshape(-1, 3).astype(object), y.reshape(-1, 3).astype(object)


def test_aux_triangulations_conforming_right_isosceles_nested(gen):
    m = gen.grid2d(17, 9, graded=True)
    o = oracle.Oracle(m)
    prev = None
    for l in range(o.J + 1):
        tri = o.level_tri(l)
        X, Y = _tri_xy(tri)
        area2 = (X[:, 1] - X[:, 0]) * (Y[:, 2] - Y[:, 0]) - (X[:, 2] - X[:, 0]) * (Y[:, 1] - Y[:, 0])
        assert all(a > 0 for a in area2)                      # CCW
        assert sum(area2) == 2 * TOP * TOP                    # covers the root box
        for t in range(tri.shape[0]):                          # right isosceles => min angle 45
            sides = sorted((X[t, k] - X[t, (k + 1) % 3]) ** 2 + (Y[t, k] - Y[t, (k + 1) % 3]) ** 2 for k in range(3))
            assert sides[0] == sides[1] and sides[2] == 2 * sides[0]
        edges = {}
        for t in range(tri.shape[0]):
            for k in range(3):
                e = tuple(sorted((int(tri[t, k]), int(tri[t, (k + 1) % 3]))))
                edges[e] = edges.get(e, 0) + 1
        for (a, b), cnt in edges.items():
            (xa, xb), (ya, yb) = lattice_xy(np.array([a, b], np.uint64))
            on_bnd = (xa == xb and xa in (0, TOP)) or (ya == yb and ya in (0, TOP))
            assert cnt == (1 if on_bnd else 2)
        if prev is not None:
            # nested: each fine triangle lies in one coarse triangle
            PX, PY = prev
            for t in range(tri.shape[0]):
                ok = False
                for s in range(PX.shape[0]):
                    inside = True
                    for k in range(3):
                        px, py = X[t, k], Y[t, k]
                        for e in range(3):
                            ax, ay, bx, by = PX[s, e], PY[s, e], PX[s, (e + 1) % 3], PY[s, (e + 1) % 3]
                            if (bx - ax) * (py - ay) - (by - ay) * (px - ax) < 0:
                                inside = False
                    if inside:
                        ok = True
                        break
                assert ok
        prev = (X, Y)


def test_interpolation_reproduces_linears(gen):
    m = gen.grid2d(17, 10, graded=True)
    o = oracle.Oracle(m, coarse_max=1)
    for l in range(max(1, o.c + 1), o.J + 1):
        I = o.I(l)
        fx, fy = lattice_xy(o.level_keys(l))
        cx, cy = lattice_xy(o.level_keys(l - 1))
        fx, fy, cx, cy = (v.astype(np.float64) for v in (fx, fy, cx, cy))
        rs = np.asarray(I.sum(1)).ravel()
        full = np.abs(rs - 1.0) < 1e-15
        assert np.allclose((I @ cx)[full], fx[full], rtol=0, atol=1e-6)
        assert np.allclose((I @ cy)[full], fy[full], rtol=0, atol=1e-6)
        assert (I.getnnz(1) <= 2).all()   # new nodes are midpoints of coarse edges


def _rediscretise(o, l):
    tri = o.level_tri(l)
    keys = o.level_keys(l)
    a0, a1, _, L = o.root()
    X, Y = lattice_xy(tri.reshape(-1))
    X = (a0 + np.ldexp(X.astype(np.float64), -D2) * L).reshape(-1, 3)
    Y = (a1 + np.ldexp(Y.astype(np.float64), -D2) * L).reshape(-1, 3)
    n = keys.size
    rows, cols, vals = [], [], []
    for t in range(tri.shape[0]):
        det = (X[t, 1] - X[t, 0]) * (Y[t, 2] - Y[t, 0]) - (X[t, 2] - X[t, 0]) * (Y[t, 1] - Y[t, 0])
        b = np.array([Y[t, 1] - Y[t, 2], Y[t, 2] - Y[t, 0], Y[t, 0] - Y[t, 1]])
        c = np.array([X[t, 2] - X[t, 1], X[t, 0] - X[t, 2], X[t, 1] - X[t, 0]])
        K = (np.outer(b, b) + np.outer(c, c)) / (2.0 * det)
        idx = np.searchsorted(keys, tri[t])
        for i in range(3):
            for j in range(3):
                if idx[i] < n and keys[idx[i]] == tri[t, i] and idx[j] < n and keys[idx[j]] == tri[t, j]:
                    rows.append(idx[i]); cols.append(idx[j]); vals.append(K[i, j])
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, n))


def test_galerkin_equals_rediscretisation_for_constant_coefficient(gen):
    m = gen.grid2d(17, 11, graded=True)
    o = oracle.Oracle(m, coarse_max=1)
    for l in range(o.c, o.J + 1):
        G = o.A(l)
        R = _rediscretise(o, l)
        assert abs(G - R).max() <= 1e-12 * abs(R).max()


def test_uniform_aux_levels_are_five_point(gen):
    m, _ = gen.workload_small_poisson()
    o = oracle.Oracle(m, coarse_max=1)
    for l in range(1, o.J + 1):
        n1 = 2 ** l - 1
        assert o.info("nlevel", l) == n1 * n1
        A = o.A(l).toarray()
        # canonical (Morton) order -> row-major order
        x, y = lattice_xy(o.level_keys(l))
        step = TOP >> l
        rm = (y // step - 1) * n1 + (x // step - 1)
        Pm = np.zeros((n1 * n1, n1 * n1))
        Pm[rm.astype(np.int64), np.arange(n1 * n1)] = 1
        T = sp.diags([-1.0, 2.0, -1.0], [-1, 0, 1], shape=(n1, n1))
        L5 = (sp.kron(sp.eye(n1), T) + sp.kron(T, sp.eye(n1))).toarray()
        assert np.abs(Pm @ A @ Pm.T - L5).max() < 1e-12


# --------------------------------------------------------------------------
# Sec. 4.1: Scott-Zhang transfer
# --------------------------------------------------------------------------

def test_scott_zhang_reproduces_linears(gen):
    for m in (gen.grid2d(17, 12), gen.grid2d(17, 13, graded=True)):
        o = oracle.Oracle(m)
        Pf = o.P(full=True)
        a0, a1, _, L = o.root()
        x, y = lattice_xy(o.level_keys(o.J, all_nodes=True))
        X = a0 + np.ldexp(x.astype(np.float64), -D2) * L
        Y = a1 + np.ldexp(y.astype(np.float64), -D2) * L
        vf = o.vertex_of_free()
        for c0, gx, gy in ((1.0, 0.0, 0.0), (0.3, 1.5, -2.0)):
            got = Pf @ (c0 + gx * X + gy * Y)
            want = c0 + gx * m.verts[vf, 0] + gy * m.verts[vf, 1]
            assert np.abs(got - want).max() < 1e-11


def test_scott_zhang_is_identity_when_aux_grid_equals_fine_grid(gen):
    # Unjittered SW-NE grid with 2^k cells per side: leaves are the cells, so
    # T_J is the fine mesh and Pi is the identity (Sec. 4.1: Pi preserves
    # piecewise linears).
    m = gen.grid2d(17, 1, jitter=0.0, random_diag=False)
    o = oracle.Oracle(m)
    P = o.P().toarray()
    vf = o.vertex_of_free()
    x, y = lattice_xy(o.level_keys(o.J))
    X = np.ldexp(x.astype(np.float64), -D2)
    Y = np.ldexp(y.astype(np.float64), -D2)
    # match fine free vertices to aux nodes by position
    order = np.lexsort((X, Y))
    fine_order = np.lexsort((m.verts[vf, 0], m.verts[vf, 1]))
    Pm = P[np.ix_(fine_order, order)]
    assert np.abs(Pm - np.eye(P.shape[0])).max() < 1e-13


# --------------------------------------------------------------------------
# Algorithms 1 and 2: smoother, V-cycle, preconditioner
# --------------------------------------------------------------------------

def _couplings(A):
    """Off-diagonal entries with |a_ij| > 1e-12 sqrt(a_ii a_jj): the graph the colouring must respect.
    The rest vanish by symmetry (e.g. across the hypotenuse of a right isosceles triangle)."""
    A = A.tocoo()
    d = A.diagonal()
    off = A.row != A.col
    strong = np.abs(A.data) > 1e-12 * np.sqrt(d[A.row] * d[A.col])
    weak = off & ~strong
    if weak.any():   # ignored entries are rounding residue, far below every real coupling
        assert np.abs(A.data[weak]).max() <= 1e-14 * np.abs(A.data).max()
    return A.row[off & strong], A.col[off & strong]


def test_colourings_are_valid_and_smoothing_sets_contain_new_nodes(gen):
    m = gen.grid2d(33, 14, graded=True)
    o = oracle.Oracle(m)
    sm, cs, col = o.smoothing_set(-1)
    r, c = _couplings(o.A())
    assert (col[r] != col[c]).all()
    for l in range(o.c + 1, o.J + 1):
        sm, cs, col = o.smoothing_set(l)
        r, c = _couplings(o.A(l))
        both = (col[r] >= 0) & (col[c] >= 0)
        assert (col[r[both]] != col[c[both]]).all()
        new = ~np.isin(o.level_keys(l), o.level_keys(l - 1))
        assert np.isin(np.nonzero(new)[0], sm).all()


def test_sequential_colouring_gives_lexicographic_gauss_seidel(gen):
    # One colour per row in index order turns the sweep into (D - L)^{-1}.
    m = gen.grid2d(12, 15)
    o = oracle.Oracle(m, colouring=1)
    A = o.A().tocsr()
    r = np.random.default_rng(0).uniform(-1, 1, o.nfree)
    u = o.gs_sweep(r, np.zeros(o.nfree), forward=True)
    ref = spla.spsolve_triangular(sp.tril(A).tocsr(), r, lower=True)
    assert np.abs(u - ref).max() < 1e-12 * np.abs(ref).max()
    ub = o.gs_sweep(r, np.zeros(o.nfree), forward=False)
    refb = spla.spsolve_triangular(sp.triu(A).tocsr(), r, lower=False)
    assert np.abs(ub - refb).max() < 1e-12 * np.abs(refb).max()


def test_single_aux_level_vcycle_is_exact_solve(gen):
    m = gen.grid2d(17, 16, graded=True)
    o = oracle.Oracle(m, coarse_max=10 ** 6)
    assert o.c == o.J
    AJ = o.A(o.J)
    f = np.random.default_rng(1).uniform(-1, 1, AJ.shape[0])
    e = o.vcycle(f)
    assert np.abs(AJ @ e - f).max() < 1e-10 * np.abs(f).max()


def test_preconditioner_is_symmetric_positive_definite(gen):
    # Algorithm 1 applies S then S^T around a symmetric V-cycle (Alg. 2 with
    # forward pre- and backward post-smoothing), so B_co is SPD.
    for m in (gen.grid2d(12, 17), gen.grid2d(13, 18, graded=True)):
        o = oracle.Oracle(m, coarse_max=20)
        n = o.nfree
        B = np.stack([o.precond(np.eye(n)[k]) for k in range(n)], 1)
        assert np.abs(B - B.T).max() <= 1e-12 * np.abs(B).max()
        assert np.linalg.eigvalsh(0.5 * (B + B.T)).min() > 0


def test_vcycle_is_symmetric(gen):
    m = gen.grid2d(17, 19, graded=True)
    o = oracle.Oracle(m, coarse_max=10)
    n = o.info("nlevel", o.J)
    rng = np.random.default_rng(2)
    x, y = rng.standard_normal(n), rng.standard_normal(n)
    assert abs(o.vcycle(x) @ y - x @ o.vcycle(y)) <= 1e-12 * abs(x @ o.vcycle(x))


# --------------------------------------------------------------------------
# Coefficient sensitivity (not in the paper): dL/da_e = -lambda_e^T K_e^(1) u_e
# --------------------------------------------------------------------------

def test_element_gradient_matches_central_differences(gen):
    # L(a) = 1/2 ||u(a) - u_obs||^2 with A(a) u = b; the adjoint A lambda = u - u_obs
    # gives dL/da_e = -lambda^T (dA/da_e) u.  Checked against central differences
    # of L in log a_e on a few elements (FP64 solves at rtol 1e-14).
    m = gen.grid2d(13, 21)
    rng = np.random.default_rng(3)
    g = rng.normal(0, 0.5, m.ne)
    m.coeff = np.exp(g)
    f = gen.nodal_uniform(m, 22)
    o = oracle.Oracle(m)
    b = o.mass_apply(f)
    u_obs = rng.uniform(-0.1, 0.1, o.nfree)
    u, st, _, _ = o.solve(b, rtol=1e-14)
    lam, st2, _, _ = o.solve(u - u_obs, rtol=1e-14)
    dLda = o.elem_grad(u, lam)
    h = 1e-5
    for e in rng.choice(m.ne, 6, replace=False):
        ups = []
        for sgn in (1, -1):
            mm = gen.grid2d(13, 21)
            mm.coeff = np.exp(g + sgn * h * (np.arange(m.ne) == e))
            oo = oracle.Oracle(mm)
            ups.append(oo.solve(b, rtol=1e-14, u0=u)[0])
        dL = 0.5 * (ups[0] - ups[1]) @ (ups[0] + ups[1] - 2 * u_obs)
        fd = dL / (2 * h)
        assert abs(fd - m.coeff[e] * dLda[e]) <= 1e-6 * np.abs(m.coeff * dLda).max(), (e, fd, m.coeff[e] * dLda[e])


def test_octree_membership_and_counts(gen):
    # the 3D cluster tree: every node's barycenters lie in its box, leaves hold
    # at most n_min, split nodes more, each split node has all 8 children
    m = gen.grid3d(9, 2)
    o = oracle.Oracle(m, stage=-1)
    levels = o.tree_levels()
    perm = o.perm()
    a = o.root()
    bc = m.verts[m.elems].sum(1) / 4.0
    assert np.array_equal(np.sort(perm), np.arange(m.ne))
    for d, segs in enumerate(levels):
        w = a[3] / 2 ** d
        for prefix, b, e, split in segs:
            q = np.zeros(3, np.int64)
            for j in range(d):
                for k in range(3):
                    q[k] |= ((int(prefix) >> (3 * j + k)) & 1) << j
            lo = a[:3] + q * w
            pts = bc[perm[b:e]]
            assert (pts >= lo - 1e-12).all() and (pts <= lo + w + 1e-12).all()
            assert (e - b > 3) if split else (e - b <= 3)
        if d + 1 < len(levels):
            assert levels[d + 1].shape[0] == 8 * int(segs[:, 3].sum())


# --------------------------------------------------------------------------
# 3D: octree closure, tetrahedral auxiliary grids, clipping transfer
# --------------------------------------------------------------------------

def _xyz3(keys):
    k = keys.astype(np.uint64)
    out = [np.zeros_like(k) for _ in range(3)]
    for j in range(21):
        for d in range(3):
            out[d] |= ((k >> np.uint64(3 * j + d)) & np.uint64(1)) << np.uint64(j)
    return [o.astype(object) for o in out]


@pytest.fixture(scope="module")
def o3(gen):
    m = gen.grid3d(9, 5)
    return m, oracle.Oracle(m)


def test_3d_aux_grids_conforming_positive_nested(o3):
    m, o = o3
    LB = o.info("LB")
    top = 1 << LB
    prev = None
    for l in range(o.J + 1):
        tet = o.level_tet(l)
        X, Y, Z = (a.reshape(-1, 4) for a in _xyz3(tet.reshape(-1)))
        vol6 = []
        for t in range(tet.shape[0]):
            e = [(X[t, v] - X[t, 0], Y[t, v] - Y[t, 0], Z[t, v] - Z[t, 0]) for v in (1, 2, 3)]
            d = (e[0][0] * (e[1][1] * e[2][2] - e[1][2] * e[2][1]) - e[0][1] * (e[1][0] * e[2][2] - e[1][2] * e[2][0])
                 + e[0][2] * (e[1][0] * e[2][1] - e[1][1] * e[2][0]))
            vol6.append(d)
        assert all(v > 0 for v in vol6)
        assert sum(vol6) == 6 * top ** 3                    # tiles the root cube
        faces = {}
        for t in range(tet.shape[0]):
            for skip in range(4):
                f = tuple(sorted(int(tet[t, v]) for v in range(4) if v != skip))
                faces[f] = faces.get(f, 0) + 1
        for f, cnt in faces.items():
            fx, fy, fz = _xyz3(np.array(f, np.uint64))
            on_bnd = any(len(set(c)) == 1 and c[0] in (0, top) for c in (fx, fy, fz))
            assert cnt == (1 if on_bnd else 2)              # conforming, no hanging nodes
        if prev is not None and tet.shape[0] < 4000:
            # nested: every vertex of a level-l tetrahedron lies in one level-(l-1) tetrahedron with it
            PX, PY, PZ = prev
            cen = [(sum(X[t]) / 4, sum(Y[t]) / 4, sum(Z[t]) / 4) for t in range(tet.shape[0])]
            for t in range(tet.shape[0]):
                ok = False
                for s in range(PX.shape[0]):
                    inside = True
                    for pt in [(X[t, v], Y[t, v], Z[t, v]) for v in range(4)] + [cen[t]]:
                        # barycentric signs (exact in rationals)
                        A = [(PX[s, v] - PX[s, 0], PY[s, v] - PY[s, 0], PZ[s, v] - PZ[s, 0]) for v in (1, 2, 3)]
                        r = (pt[0] - PX[s, 0], pt[1] - PY[s, 0], pt[2] - PZ[s, 0])

                        def det(a, b, c):
                            return (a[0] * (b[1] * c[2] - b[2] * c[1]) - a[1] * (b[0] * c[2] - b[2] * c[0])
                                    + a[2] * (b[0] * c[1] - b[1] * c[0]))
                        d0 = det(*A)
                        ls = [det(r, A[1], A[2]), det(A[0], r, A[2]), det(A[0], A[1], r)]
                        if min(ls) < 0 or sum(ls) > d0:
                            inside = False
                            break
                    if inside:
                        ok = True
                        break
                assert ok
        prev = (X, Y, Z)


def test_3d_interpolation_and_transfer_reproduce_linears(o3):
    m, o = o3
    LB = o.info("LB")
    a0, a1, a2, L = o.root()
    for l in range(max(1, o.c + 1), o.J + 1):
        I = o.I(l)
        fx, fy, fz = (np.array(v, np.float64) for v in _xyz3(o.level_keys(l)))
        cx, cy, cz = (np.array(v, np.float64) for v in _xyz3(o.level_keys(l - 1)))
        full = np.abs(np.asarray(I.sum(1)).ravel() - 1.0) < 1e-15
        for f, c in ((fx, cx), (fy, cy), (fz, cz)):
            assert np.allclose((I @ c)[full], f[full], atol=1e-6)
    Pf = o.P(full=True)
    X, Y, Z = (a + np.ldexp(np.array(v, np.float64), -LB) * L for a, v in zip((a0, a1, a2), _xyz3(o.level_keys(o.J, True))))
    vf = o.vertex_of_free()
    for c0, gx, gy, gz in ((1.0, 0, 0, 0), (0.2, 1.0, -2.0, 0.5)):
        got = Pf @ (c0 + gx * X + gy * Y + gz * Z)
        want = c0 + gx * m.verts[vf, 0] + gy * m.verts[vf, 1] + gz * m.verts[vf, 2]
        assert np.abs(got - want).max() < 1e-12


@pytest.mark.parametrize("seed", [4, 11])
def test_3d_finest_coefficient_is_the_volume_average(gen, seed):
    # Sec. 4: the finest auxiliary coefficient on a tetrahedron t is
    # (1/|t|) sum_e a_e |e cap t|.  A constant a is reproduced exactly; for
    # any a the integral over the cube is conserved (both grids tile it) and
    # every average lies between the extreme fine values.
    m = gen.grid3d(9, seed)
    m.coeff = np.full(m.ne, 3.7)
    o = oracle.Oracle(m)
    assert np.abs(o.finest_coef() / 3.7 - 1).max() < 1e-13
    rng = np.random.default_rng(seed)
    m.coeff = np.exp(rng.normal(size=m.ne))
    o = oracle.Oracle(m)
    LB = o.info("LB")
    a0, a1, a2, L = o.root()
    tet = o.level_tet(o.J)
    P = np.stack([a + np.ldexp(np.array(v, np.float64), -LB) * L
                  for a, v in zip((a0, a1, a2), _xyz3(tet.reshape(-1)))], 1).reshape(-1, 4, 3)
    vol = np.abs(np.linalg.det(P[:, 1:] - P[:, :1])) / 6
    E = m.verts[m.elems]
    fvol = np.abs(np.linalg.det(E[:, 1:] - E[:, :1])) / 6
    c = o.finest_coef()
    assert abs(c @ vol - m.coeff @ fvol) <= 1e-13 * (m.coeff @ fvol)
    assert c.min() >= m.coeff.min() * (1 - 1e-13) and c.max() <= m.coeff.max() * (1 + 1e-13)


def test_3d_galerkin_equals_rediscretisation(o3):
    m, o = o3
    LB = o.info("LB")
    a0, a1, a2, L = o.root()
    for l in range(o.c, o.J + 1):
        tet = o.level_tet(l)
        keys = o.level_keys(l)
        P = [a + np.ldexp(np.array(v, np.float64), -LB) * L for a, v in zip((a0, a1, a2), _xyz3(tet.reshape(-1)))]
        P = np.stack(P, 1).reshape(-1, 4, 3)
        n = keys.size
        R = np.zeros((n, n))
        for t in range(tet.shape[0]):
            Jm = (P[t, 1:] - P[t, 0]).T
            G = np.vstack([-np.linalg.inv(Jm).sum(0), np.linalg.inv(Jm)])
            K = abs(np.linalg.det(Jm)) / 6.0 * G @ G.T
            idx = np.searchsorted(keys, tet[t])
            ok = (idx < n) & (keys[np.minimum(idx, n - 1)] == tet[t])
            for i in range(4):
                for j in range(4):
                    if ok[i] and ok[j]:
                        R[idx[i], idx[j]] += K[i, j]
        Al = o.A(l).toarray()
        assert np.abs(Al - R).max() <= 1e-12 * np.abs(R).max()


def test_3d_pcg_dense_and_symmetric_preconditioner(gen):
    m = gen.grid3d(5, 6)
    o = oracle.Oracle(m, coarse_max=4)
    b = o.mass_apply(gen.nodal_uniform(m, 8))
    u, st, it, _ = o.solve(b, rtol=1e-14)
    ref = np.linalg.solve(o.A().toarray(), b)
    assert np.linalg.norm(u - ref) <= 1e-12 * np.linalg.norm(ref)
    n = o.nfree
    B = np.stack([o.precond(np.eye(n)[k]) for k in range(n)], 1)
    assert np.abs(B - B.T).max() <= 1e-12 * np.abs(B).max()
    assert np.linalg.eigvalsh(0.5 * (B + B.T)).min() > 0


def test_3d_manufactured_solution_second_order(gen):
    errs = []
    for n in (5, 9, 17):
        m = gen.grid3d(n, 7)
        x, y, z = m.verts.T
        f = 3 * math.pi ** 2 * np.sin(math.pi * x) * np.sin(math.pi * y) * np.sin(math.pi * z)
        o = oracle.Oracle(m)
        u, st, it, _ = o.solve(o.mass_apply(f), rtol=1e-12)
        assert st == 0
        vf = o.vertex_of_free()
        ue = np.sin(math.pi * x[vf]) * np.sin(math.pi * y[vf]) * np.sin(math.pi * z[vf])
        errs.append(np.sqrt(np.mean((u - ue) ** 2)))
    r = [errs[i] / errs[i + 1] for i in range(2)]
    assert all(3.0 < q < 5.0 for q in r), (errs, r)


# --------------------------------------------------------------------------
# Variants of B (Sec. 4.1 smoothers, eq. fasp additive form) and the ASMG
# iteration (Sec. 5.1 rates)
# --------------------------------------------------------------------------

def _exact_aux(gen, **kw):
    # one auxiliary level solved exactly (coarse_max above its size): Btilde = A_J^{-1}
    m = gen.grid2d(9, 4)
    o = oracle.Oracle(m, coarse_max=100000, **kw)
    assert o.c == o.J
    return m, o


def _dense_parts(o):
    A = o.A().toarray()
    P = o.P().toarray()
    AJ = o.A(o.J).toarray()
    return A, np.diag(1.0 / np.diag(A)), P, np.linalg.inv(AJ)


@pytest.mark.parametrize("sweeps", [1, 2])
def test_additive_jacobi_preconditioner_closed_form(gen, sweeps):
    # eq. fasp with S = D^{-1} (Sec. 4.1): B r = S_m r + Pi A_J^{-1} Pi^t r, where m
    # Jacobi steps from zero give S_1 r = D^{-1} r, S_2 r = D^{-1} (2 r - A D^{-1} r)
    m, o = _exact_aux(gen, smoother=1, additive=1, fine_sweeps=sweeps)
    A, Dinv, P, AJinv = _dense_parts(o)
    r = np.random.default_rng(1).standard_normal(o.nfree)
    s = Dinv @ r if sweeps == 1 else Dinv @ (2 * r - A @ (Dinv @ r))
    want = s + P @ (AJinv @ (P.T @ r))
    assert np.abs(o.precond(r) - want).max() <= 1e-12 * np.abs(want).max()


def test_multiplicative_jacobi_preconditioner_closed_form(gen):
    # Algorithm 1 with S = S^t = D^{-1}: u1 = D^{-1} r, u2 = u1 + Pi A_J^{-1} Pi^t (r - A u1),
    # u3 = u2 + D^{-1} (r - A u2); B is then symmetric positive definite
    m, o = _exact_aux(gen, smoother=1)
    A, Dinv, P, AJinv = _dense_parts(o)
    r = np.random.default_rng(2).standard_normal(o.nfree)
    u1 = Dinv @ r
    u2 = u1 + P @ (AJinv @ (P.T @ (r - A @ u1)))
    u3 = u2 + Dinv @ (r - A @ u2)
    assert np.abs(o.precond(r) - u3).max() <= 1e-12 * np.abs(u3).max()
    n = o.nfree
    B = np.stack([o.precond(np.eye(n)[k]) for k in range(n)], 1)
    assert np.abs(B - B.T).max() <= 1e-12 * np.abs(B).max()
    assert np.linalg.eigvalsh(0.5 * (B + B.T)).min() > 0


def test_asmg_iteration_rates_bounded_and_mesh_independent(gen):
    # Sec. 5.1: the ASMG iteration u <- u + B (b - A u) contracts at a rate bounded away
    # from 1 (roughly 0.4 on the paper's mesh) uniformly in h
    rates = []
    for n in (17, 33, 65):
        m = gen.grid2d(n, 3)
        o = oracle.Oracle(m, iteration=1, max_iter=100)
        b = o.mass_apply(gen.nodal_uniform(m, 1))
        u, st, it, hist = o.solve(b, rtol=1e-8)
        assert st == 0 and hist.size == it + 1
        assert np.all(hist[1:] < hist[:-1])
        rates.append((hist[-1] / hist[0]) ** (1.0 / it))
        # the iterate is the solution of A u = b to the stopping tolerance
        assert np.linalg.norm(b - o.spmv(u)) <= 1e-8 * np.linalg.norm(b) * (1 + 1e-12)
    assert max(rates) <= 0.4, rates
    assert max(rates) <= 2.5 * min(rates), rates


# --------------------------------------------------------------------------
# Domains that do not fill the root box: Dirichlet auxiliary grids
# T^D_l = {tau in sigma^(l) | tau in Omega} (Sec. 3.4), checked against an
# independent computation of each triangle's coverage by the fine elements
# (polygon clipping written here) and of each node's interior angle sum.
# --------------------------------------------------------------------------

def _clip_poly(poly, tri):
    # Sutherland-Hodgman: poly (list of (x, y)) cut by the three half-planes of a CCW triangle
    out = poly
    for k in range(3):
        ax, ay = tri[k]
        bx, by = tri[(k + 1) % 3]
        inp, out = out, []
        if not inp:
            break
        side = lambda p: (bx - ax) * (p[1] - ay) - (by - ay) * (p[0] - ax)
        for i in range(len(inp)):
            p, q = inp[i], inp[(i + 1) % len(inp)]
            sp, sq = side(p), side(q)
            if sp >= 0:
                out.append(p)
            if (sp >= 0) != (sq >= 0):
                t = sp / (sp - sq)
                out.append((p[0] + t * (q[0] - p[0]), p[1] + t * (q[1] - p[1])))
    return out


def _area(poly):
    return 0.5 * sum(poly[i][0] * poly[(i + 1) % len(poly)][1] - poly[(i + 1) % len(poly)][0] * poly[i][1]
                     for i in range(len(poly))) if len(poly) >= 3 else 0.0


@pytest.fixture(scope="module")
def lshape(gen):
    m = gen.grid2d_domain(17, 3, "L")
    return m, oracle.Oracle(m)


def _lattice_pts(o, keys):
    x, y = oracle.lattice_xy(keys)
    a0, a1, _, L = o.root()
    return a0 + np.ldexp(x.astype(np.float64), -31) * L, a1 + np.ldexp(y.astype(np.float64), -31) * L


def test_dirichlet_aux_triangles_are_those_inside_omega(gen, lshape):
    m, o = lshape
    E = m.verts[m.elems]
    lo, hi = E.min(axis=1), E.max(axis=1)
    boxarea = 1.0
    for l in range(o.J + 1):
        # every triangle of sigma^(l): the inside ones are the oracle's level triangles; the
        # others are found from the full box triangulation of the oracle run on the square
        tri = o.level_tri(l)
        X, Y = _lattice_pts(o, tri.reshape(-1))
        X, Y = X.reshape(-1, 3), Y.reshape(-1, 3)
        tot = 0.0
        for t in range(tri.shape[0]):
            T = [(X[t, k], Y[t, k]) for k in range(3)]
            a = _area(T)
            tot += a
            tlo, thi = np.array([X[t].min(), Y[t].min()]), np.array([X[t].max(), Y[t].max()])
            sel = np.where(np.all(lo <= thi, axis=1) & np.all(hi >= tlo, axis=1))[0]
            cov = sum(_area(_clip_poly([tuple(p) for p in E[e]], T)) for e in sel)
            assert cov >= (1 - 1e-9) * a, (l, t, cov, a)       # inside Omega
        # Omega^D_l grows with l and stays inside Omega
        assert tot <= 0.75 * boxarea * (1 + 1e-9) + 0.05
        if l:
            assert tot >= prev - 1e-12
        prev = tot


def test_dirichlet_aux_grids_are_maximal(gen, lshape):
    # the triangles of sigma^(l) left out are not covered by the fine elements
    m, o = lshape
    E = m.verts[m.elems]
    lo, hi = E.min(axis=1), E.max(axis=1)
    for l in range(o.J + 1):
        inside = set(map(tuple, o.level_tri(l).tolist()))
        tri = o.level_alltri(l)
        X, Y = _lattice_pts(o, tri.reshape(-1))
        X, Y = X.reshape(-1, 3), Y.reshape(-1, 3)
        left_out = 0
        for t in range(tri.shape[0]):
            if tuple(tri[t].tolist()) in inside:
                continue
            left_out += 1
            T = [(X[t, k], Y[t, k]) for k in range(3)]
            tlo, thi = np.array([X[t].min(), Y[t].min()]), np.array([X[t].max(), Y[t].max()])
            sel = np.where(np.all(lo <= thi, axis=1) & np.all(hi >= tlo, axis=1))[0]
            cov = sum(_area(_clip_poly([tuple(p) for p in E[e]], T)) for e in sel)
            assert cov < (1 - 1e-9) * _area(T), (l, t)
        assert left_out > 0


def test_dirichlet_free_nodes_are_interior_by_angle_sum(lshape):
    # a node of T^D_J is free exactly when the inside triangles around it close
    # up (interior angles sum to 2 pi)
    m, o = lshape
    tri = o.level_tri(o.J)
    X, Y = _lattice_pts(o, tri.reshape(-1))
    X, Y = X.reshape(-1, 3), Y.reshape(-1, 3)
    ang = {}
    for t in range(tri.shape[0]):
        for k in range(3):
            p = np.array([X[t, k], Y[t, k]])
            u = np.array([X[t, (k + 1) % 3], Y[t, (k + 1) % 3]]) - p
            v = np.array([X[t, (k + 2) % 3], Y[t, (k + 2) % 3]]) - p
            a = np.arccos(np.clip(u @ v / np.linalg.norm(u) / np.linalg.norm(v), -1, 1))
            ang[int(tri[t, k])] = ang.get(int(tri[t, k]), 0.0) + a
    free = set(int(k) for k in o.level_keys(o.J))
    interior = set(k for k, a in ang.items() if abs(a - 2 * np.pi) < 1e-9)
    assert free == interior


@pytest.mark.parametrize("shape", ["L", "hole"])
def test_dirichlet_domain_pcg_dense_and_spd(gen, shape):
    m = gen.grid2d_domain(17, 5, shape)
    o = oracle.Oracle(m, coarse_max=8)
    assert o.c < o.J
    b = o.mass_apply(gen.nodal_uniform(m, 2))
    u, st, it, _ = o.solve(b, rtol=1e-13)
    ref = np.linalg.solve(o.A().toarray(), b)
    assert st == 0 and np.linalg.norm(u - ref) <= 1e-11 * np.linalg.norm(ref)
    n = o.nfree
    B = np.stack([o.precond(np.eye(n)[k]) for k in range(n)], 1)
    assert np.abs(B - B.T).max() <= 1e-12 * np.abs(B).max()
    assert np.linalg.eigvalsh(0.5 * (B + B.T)).min() > 0
    # nested Dirichlet hierarchies: every level's free nodes are free on the finer levels
    for l in range(o.c + 1, o.J + 1):
        assert set(o.level_keys(l - 1).tolist()) <= set(o.level_keys(l).tolist())


# ------------------------------------------------ Dirichlet grids in 3D (R17)
def test_dirichlet3d_aligned_l_prism_tets_and_free_nodes(gen):
    # Unjittered L-shaped prism: the cut planes x = 1/2 and y = 1/2 are box
    # faces from depth 1 on, so a tetrahedron of sigma^(l >= 1) lies in Omega
    # exactly when its centroid does; the root cube's six tetrahedra all
    # contain the diagonal point (3/4, 3/4, 3/4) of the removed quarter.  The
    # free nodes are the lattice nodes of sigma^(l) off the boundary of Omega.
    m = gen.grid3d_domain(9, 1, "L", jitter=0.0)
    o = oracle.Oracle(m)
    a = o.root()
    amin, L = np.array(a[:3]), a[3]
    top = 2 ** (o.J + 1)
    for l in range(o.J + 1):
        allt = o.level_alltet(l)
        x, y, z = (np.asarray(v, dtype=np.float64).reshape(-1, 4) for v in _xyz3(allt.reshape(-1)))
        cx, cy = amin[0] + x.mean(1) / top * L, amin[1] + y.mean(1) / top * L
        want = {tuple(t) for t, ok in zip(allt.tolist(), (cx < 0.5) | (cy < 0.5)) if ok and l >= 1}
        got = {tuple(t) for t in o.level_tet(l).tolist()}
        assert got == want, l
        keys = np.unique(allt.reshape(-1))
        qx, qy, qz = (np.asarray(v, dtype=np.float64) / top for v in _xyz3(keys))
        px, py = amin[0] + qx * L, amin[1] + qy * L
        interior = (qx > 0) & (qx < 1) & (qy > 0) & (qy < 1) & (qz > 0) & (qz < 1)
        interior &= ~((px >= 0.5 - 1e-12) & (py >= 0.5 - 1e-12))
        assert np.array_equal(np.sort(keys[interior]), o.level_keys(l)), l


@pytest.mark.parametrize("shape", ["L", "hole"])
def test_dirichlet3d_domain_pcg_dense_and_spd(gen, shape):
    m = gen.grid3d_domain(7, 5, shape)
    o = oracle.Oracle(m, coarse_max=8)
    assert o.c < o.J
    # the domain cuts the finest grid: fewer tetrahedra than sigma^(J)
    assert o.level_tet(o.J).shape[0] < o.info("nalltet", o.J)
    b = o.mass_apply(gen.nodal_uniform(m, 2))
    u, st, it, _ = o.solve(b, rtol=1e-13)
    ref = np.linalg.solve(o.A().toarray(), b)
    assert st == 0 and np.linalg.norm(u - ref) <= 1e-11 * np.linalg.norm(ref)
    n = o.nfree
    B = np.stack([o.precond(np.eye(n)[k]) for k in range(n)], 1)
    assert np.abs(B - B.T).max() <= 1e-12 * np.abs(B).max()
    assert np.linalg.eigvalsh(0.5 * (B + B.T)).min() > 0
    for l in range(o.c + 1, o.J + 1):
        assert set(o.level_keys(l - 1).tolist()) <= set(o.level_keys(l).tolist())


@pytest.mark.parametrize("dim", [2, 3])
def test_dirichlet_aligned_l_kept_simplices_fully_covered(gen, dim):
    # Unjittered L domains: the cut lies on box faces from depth 1 on, so every
    # kept simplex of sigma^(J) is covered exactly and its mean coefficient
    # (a = 1 inside, 0 outside) is 1; and in 2D, as in 3D, a triangle of
    # sigma^(l >= 1) is kept exactly when its centroid lies in Omega.
    m = gen.grid2d_domain(17, 1, "L", jitter=0.0) if dim == 2 else gen.grid3d_domain(9, 1, "L", jitter=0.0)
    o = oracle.Oracle(m)
    assert np.abs(o.finest_coef() - 1.0).max() <= 1e-12
    if dim == 2:
        a0, a1, _, L = o.root()
        for l in range(o.J + 1):
            allt = o.level_alltri(l)
            X, Y = _lattice_pts(o, allt.reshape(-1))
            cx, cy = X.reshape(-1, 3).mean(1), Y.reshape(-1, 3).mean(1)
            want = {tuple(t) for t, ok in zip(allt.tolist(), (cx < 0.5) | (cy < 0.5)) if ok and l >= 1}
            assert {tuple(t) for t in o.level_tri(l).tolist()} == want, l


# --------------------------------------------------------------------------
# Mixed Dirichlet / Neumann boundaries (Sec. 3.4, remark on mixed boundary
# conditions) and the near-boundary correction (Sec. 3.5, Algorithm 3).
# Reading: a triangle meets Omega or Gamma_D when its interior does; Gamma_D
# is the union of the fine boundary edges with two Dirichlet endpoints.
# Checked against exact rational geometry, graph distances, point location
# and the textbook natural-boundary stencil, all written here.
# --------------------------------------------------------------------------

NEUMANN = 2


def _with_neumann(m, sel):
    m.bflag = m.bflag.copy()
    m.bflag[sel & (m.bflag == 1)] = NEUMANN
    return m


def _mixed_domain(gen, n, shape, where, seed=2):
    m = gen.grid2d_domain(n, seed, shape)
    x, y = m.verts[:, 0], m.verts[:, 1]
    inner = (x > 0) & (x < 1) & (y > 0) & (y < 1)
    return _with_neumann(m, inner if where == "inner" else ((x == 0) & (y > 0) & (y < 1)))


def test_mixed_square_levels_are_the_natural_boundary_stencil(gen):
    # Unit square, Neumann on x = 1 (0 < y < 1): every triangle of sigma^(l) is
    # kept, the free nodes are the lattice nodes off x = 0, y = 0, y = 1, and
    # each level operator is the P1 Laplacian with the natural condition on
    # x = 1: K_y (x) M_x + I (x) K_x with K the 1D stiffness (last diagonal 1
    # on the Neumann end) and M_x = diag(1, ..., 1, 1/2) the lumped 1D mass.
    m, _ = gen.workload_small_poisson()
    x, y = m.verts[:, 0], m.verts[:, 1]
    m = _with_neumann(m, (x == 1.0) & (y > 0) & (y < 1))
    o = oracle.Oracle(m, coarse_max=1)
    for l in range(1, o.J + 1):
        assert {tuple(t) for t in o.level_tri(l).tolist()} == {tuple(t) for t in o.level_alltri(l).tolist()}
        ak = o.level_keys(l, all_nodes=True)
        ax, ay = lattice_xy(ak)
        want = np.sort(ak[(ax > 0) & (ay > 0) & (ay < TOP)])
        assert np.array_equal(o.level_keys(l), want), l
        nx, ny = 2 ** l, 2 ** l - 1
        kx, ky = lattice_xy(o.level_keys(l))
        step = TOP >> l
        rm = ((ky // step - 1) * nx + (kx // step - 1)).astype(np.int64)
        Pm = np.zeros((nx * ny, nx * ny))
        Pm[rm, np.arange(nx * ny)] = 1
        Ky = sp.diags([-1.0, 2.0, -1.0], [-1, 0, 1], shape=(ny, ny)).toarray()
        Kx = sp.diags([-1.0, 2.0, -1.0], [-1, 0, 1], shape=(nx, nx)).toarray()
        Kx[-1, -1] = 1
        Mx = np.eye(nx)
        Mx[-1, -1] = 0.5
        want_A = np.kron(Ky, Mx) + np.kron(np.eye(ny), Kx)
        assert np.abs(Pm @ o.A(l).toarray() @ Pm.T - want_A).max() < 1e-12, l


def _fr_pt(p):
    return (Fraction(float(p[0])), Fraction(float(p[1])))


def _fr_orient(p, q, r):
    return (q[0] - p[0]) * (r[1] - p[1]) - (q[1] - p[1]) * (r[0] - p[0])


def _seg_hits_open_triangle(a, b, T):
    # exact: clip a + t (b - a), 0 <= t <= 1, by the three closed half-planes of
    # T; the interior is met when a piece of positive length remains and its
    # midpoint lies strictly inside
    t0, t1 = Fraction(0), Fraction(1)
    for k in range(3):
        p, q = T[k], T[(k + 1) % 3]
        fa, fb = _fr_orient(p, q, a), _fr_orient(p, q, b)
        if fa == fb:
            if fa < 0:
                return False
            continue
        tc = fa / (fa - fb)
        if fb > fa:
            t0 = max(t0, tc)
        else:
            t1 = min(t1, tc)
    if t1 <= t0:
        return False
    tm = (t0 + t1) / 2
    mid = (a[0] + tm * (b[0] - a[0]), a[1] + tm * (b[1] - a[1]))
    return all(_fr_orient(T[k], T[(k + 1) % 3], mid) > 0 for k in range(3))


def _fr_on_segment(a, b, p):
    return (_fr_orient(a, b, p) == 0 and min(a[0], b[0]) <= p[0] <= max(a[0], b[0])
            and min(a[1], b[1]) <= p[1] <= max(a[1], b[1]))


def _gamma_d(m):
    ed = np.sort(np.concatenate([m.elems[:, [0, 1]], m.elems[:, [1, 2]], m.elems[:, [2, 0]]]), axis=1)
    uniq, cnt = np.unique(ed, axis=0, return_counts=True)
    bd = uniq[cnt == 1]
    bd = bd[(m.bflag[bd[:, 0]] == 1) & (m.bflag[bd[:, 1]] == 1)]
    return [(_fr_pt(m.verts[a]), _fr_pt(m.verts[b])) for a, b in bd]


@pytest.mark.parametrize("shape,where", [("L", "inner"), ("hole", "outer")])
def test_mixed_kept_triangles_and_dirichlet_nodes_exact(gen, shape, where):
    m = _mixed_domain(gen, 17, shape, where)
    o = oracle.Oracle(m)
    gd = _gamma_d(m)
    assert gd and (m.bflag == NEUMANN).any()
    E = m.verts[m.elems]
    lo, hi = E.min(axis=1), E.max(axis=1)
    for l in range(o.J + 1):
        allt = o.level_alltri(l)
        X, Y = _lattice_pts(o, allt.reshape(-1))
        X, Y = X.reshape(-1, 3), Y.reshape(-1, 3)
        kept, dirn = set(), set()
        for t in range(allt.shape[0]):
            T = [(X[t, k], Y[t, k]) for k in range(3)]
            Tf = [_fr_pt(p) for p in T]
            tlo, thi = (X[t].min(), Y[t].min()), (X[t].max(), Y[t].max())
            hit = any(_seg_hits_open_triangle(a, b, Tf) for a, b in gd
                      if min(a[0], b[0]) <= thi[0] and max(a[0], b[0]) >= tlo[0]
                      and min(a[1], b[1]) <= thi[1] and max(a[1], b[1]) >= tlo[1])
            if hit:
                dirn.update(allt[t].tolist())
                continue
            sel = np.where(np.all(lo <= thi, axis=1) & np.all(hi >= tlo, axis=1))[0]
            cov = sum(_area(_clip_poly([tuple(p) for p in E[e]], T)) for e in sel)
            if cov > 1e-12 * _area(T):
                kept.add(tuple(allt[t].tolist()))
        assert {tuple(t) for t in o.level_tri(l).tolist()} == kept, l
        nodes = sorted({k for t in kept for k in t})
        PX, PY = _lattice_pts(o, np.array(nodes, dtype=np.uint64))
        free = [k for k, px, py in zip(nodes, PX, PY) if k not in dirn
                and not any(_fr_on_segment(a, b, _fr_pt((px, py))) for a, b in gd)]
        assert o.level_keys(l).tolist() == free, l


def _angle_sums(o, tri):
    X, Y = _lattice_pts(o, tri.reshape(-1))
    X, Y = X.reshape(-1, 3), Y.reshape(-1, 3)
    ang = {}
    for t in range(tri.shape[0]):
        for k in range(3):
            p = np.array([X[t, k], Y[t, k]])
            u = np.array([X[t, (k + 1) % 3], Y[t, (k + 1) % 3]]) - p
            v = np.array([X[t, (k + 2) % 3], Y[t, (k + 2) % 3]]) - p
            a = np.arccos(np.clip(u @ v / np.linalg.norm(u) / np.linalg.norm(v), -1, 1))
            ang[int(tri[t, k])] = ang.get(int(tri[t, k]), 0.0) + a
    return ang


@pytest.mark.parametrize("layers", [0, 2])
def test_near_boundary_sets_are_graph_balls_around_the_boundary(gen, layers):
    # Layer 0 holds the triangles touching Gamma_l, layer i those touching layer
    # i-1; on a conforming grid the nodes of layer j are exactly the nodes within
    # j + 1 edges of a boundary node (boundary nodes found here by angle sums)
    from scipy.sparse.csgraph import shortest_path
    m = _mixed_domain(gen, 17, "L", "inner")
    o = oracle.Oracle(m, coarse_max=8, nb_layers=layers)
    assert o.c < o.J
    for l in range(o.c + 1, o.J + 1):
        tri = o.level_tri(l)
        nodes = np.unique(tri.reshape(-1))
        pos = {int(k): i for i, k in enumerate(nodes)}
        r, c = [], []
        for t in tri.tolist():
            for a in range(3):
                r.append(pos[t[a]])
                c.append(pos[t[(a + 1) % 3]])
        G = sp.coo_matrix((np.ones(len(r)), (r, c)), shape=(nodes.size, nodes.size)).tocsr()
        bnd = [pos[k] for k, a in _angle_sums(o, tri).items() if abs(a - 2 * np.pi) > 1e-9]
        dist = shortest_path(G, directed=False, unweighted=True, indices=bnd).min(axis=0)
        ball = set(int(k) for k in nodes[dist <= layers + 1])
        keys = o.level_keys(l)
        want = [i for i, k in enumerate(keys.tolist()) if k in ball]
        assert o.near_boundary_set(l).tolist() == want, l
        assert len(want) > 0 and (l < o.J or len(want) < keys.size)


@pytest.mark.parametrize("shape,where", [("hole", "outer"), ("L", "inner")])
def test_mixed_interpolation_is_the_coarse_function_at_fine_nodes(gen, shape, where):
    # I_l e = the coarse P1 function (zero at Dirichlet nodes and outside the
    # kept coarse triangles) evaluated at the fine free nodes, by point location
    # over every kept coarse triangle (on the L with a Neumann cut, fine nodes
    # on box edges lie between kept and removed coarse triangles)
    m = _mixed_domain(gen, 17, shape, where)
    o = oracle.Oracle(m, coarse_max=8)
    rng = np.random.default_rng(7)
    for l in range(o.c + 1, o.J + 1):
        ctri, ckeys = o.level_tri(l - 1), o.level_keys(l - 1)
        ec = rng.standard_normal(ckeys.size)
        val = dict(zip(ckeys.tolist(), ec))
        CX, CY = _lattice_pts(o, ctri.reshape(-1))
        CX, CY = CX.reshape(-1, 3), CY.reshape(-1, 3)
        FX, FY = _lattice_pts(o, o.level_keys(l))
        want = np.zeros(FX.size)
        for i in range(FX.size):
            for t in range(ctri.shape[0]):
                x0, y0 = CX[t, 0], CY[t, 0]
                det = (CX[t, 1] - x0) * (CY[t, 2] - y0) - (CX[t, 2] - x0) * (CY[t, 1] - y0)
                l1 = ((FX[i] - x0) * (CY[t, 2] - y0) - (CX[t, 2] - x0) * (FY[i] - y0)) / det
                l2 = ((CX[t, 1] - x0) * (FY[i] - y0) - (FX[i] - x0) * (CY[t, 1] - y0)) / det
                lam = (1 - l1 - l2, l1, l2)
                if min(lam) >= -1e-12:
                    want[i] = sum(lam[k] * val.get(int(ctri[t, k]), 0.0) for k in range(3))
                    break
        got = o.I(l) @ ec
        assert np.abs(got - want).max() <= 1e-12 * max(1.0, np.abs(want).max()), l


@pytest.mark.parametrize("layers", [-1, 2])
def test_two_level_cycle_is_coarse_then_near_boundary_solve(gen, layers):
    # Algorithm 3 with no smoothing steps on two levels: u1 = I A_c^{-1} I^t f,
    # then u2 = u1 + E (E^t A_J E)^{-1} E^t (f - A_J u1), E the injection of J_{J,j}
    m = _mixed_domain(gen, 17, "L", "inner")
    o0 = oracle.Oracle(m)
    J = o0.J
    o = oracle.Oracle(m, coarse_max=o0.info("nlevel", J - 1), nu_pre=0, nu_post=0, nb_layers=layers)
    assert o.c == J - 1
    AJ, Ac, I = o.A(J).toarray(), o.A(J - 1).toarray(), o.I(J).toarray()
    f = np.random.default_rng(3).standard_normal(AJ.shape[0])
    u = I @ np.linalg.solve(Ac, I.T @ f)
    nb = o.near_boundary_set(J)
    assert (nb.size > 0) == (layers >= 0)
    if nb.size:
        r = f - AJ @ u
        u[nb] += np.linalg.solve(AJ[np.ix_(nb, nb)], r[nb])
    assert np.abs(o.vcycle(f) - u).max() <= 1e-11 * np.abs(u).max()


def test_mixed_level_coefficient_is_the_mean_over_the_covered_part(gen):
    # each level is rediscretised: A_l = sum over kept triangles of
    # a_tau K_tau with a_tau the area-weighted mean of a over tau n Omega
    m = _mixed_domain(gen, 17, "L", "inner")
    m.coeff = gen.subcube_coefficient(m, 5, ncube=4)
    o = oracle.Oracle(m, coarse_max=8)
    E = m.verts[m.elems]
    lo, hi = E.min(axis=1), E.max(axis=1)
    for l in range(o.c, o.J + 1):
        tri, keys = o.level_tri(l), o.level_keys(l)
        pos = {int(k): i for i, k in enumerate(keys)}
        X, Y = _lattice_pts(o, tri.reshape(-1))
        X, Y = X.reshape(-1, 3), Y.reshape(-1, 3)
        A = np.zeros((keys.size, keys.size))
        coef = []
        for t in range(tri.shape[0]):
            T = [(X[t, k], Y[t, k]) for k in range(3)]
            tlo, thi = (X[t].min(), Y[t].min()), (X[t].max(), Y[t].max())
            sel = np.where(np.all(lo <= thi, axis=1) & np.all(hi >= tlo, axis=1))[0]
            ar = np.array([_area(_clip_poly([tuple(p) for p in E[e]], T)) for e in sel])
            a_t = (ar * m.coeff[sel]).sum() / ar.sum()
            coef.append(a_t)
            B = np.array([[X[t, 1] - X[t, 0], X[t, 2] - X[t, 0]], [Y[t, 1] - Y[t, 0], Y[t, 2] - Y[t, 0]]])
            G = np.linalg.inv(B).T @ np.array([[-1.0, 1.0, 0.0], [-1.0, 0.0, 1.0]])
            K = a_t * abs(np.linalg.det(B)) / 2 * (G.T @ G)
            for i in range(3):
                for j in range(3):
                    if int(tri[t, i]) in pos and int(tri[t, j]) in pos:
                        A[pos[int(tri[t, i])], pos[int(tri[t, j])]] += K[i, j]
        assert np.abs(o.A(l).toarray() - A).max() <= 1e-12 * np.abs(A).max(), l
        if l == o.J:
            assert np.abs(o.finest_coef() - np.array(coef)).max() <= 1e-12 * max(coef)


@pytest.mark.parametrize("kind", ["lognormal", "subcube", "graded_lognormal", "L_lognormal", "hole_subcube"])
def test_2d_finest_coefficient_is_the_area_average(gen, kind):
    # Sec. 4.1 (the auxiliary operator from the bilinear form, R6 / R17): on
    # box and Dirichlet grids the finest auxiliary coefficient of a kept
    # triangle K is (1/|K|) sum_e a_e |e n K|, with a = 0 outside Omega.  Both
    # the intersections (the polygon clipper of this file) and |K| (from the
    # lattice corners) are computed here, independently of the oracle.
    rng = np.random.default_rng(7)
    if kind == "lognormal":
        m = gen.grid2d(17, 5)
    elif kind == "subcube":
        m = gen.grid2d(17, 6)
    elif kind == "graded_lognormal":
        m = gen.grid2d(17, 2, graded=True)
    elif kind == "L_lognormal":
        m = gen.grid2d_domain(17, 3, "L")
    else:
        m = gen.grid2d_domain(17, 4, "hole")
    if kind.endswith("lognormal"):
        m.coeff = np.exp(rng.normal(size=m.ne))
    else:
        m.coeff = gen.subcube_coefficient(m, 5, ncube=4)
    o = oracle.Oracle(m)
    E = m.verts[m.elems]
    lo, hi = E.min(axis=1), E.max(axis=1)
    tri = o.level_tri(o.J)
    X, Y = _lattice_pts(o, tri.reshape(-1))
    X, Y = X.reshape(-1, 3), Y.reshape(-1, 3)
    want = np.empty(tri.shape[0])
    for t in range(tri.shape[0]):
        T = [(X[t, k], Y[t, k]) for k in range(3)]
        area = 0.5 * ((X[t, 1] - X[t, 0]) * (Y[t, 2] - Y[t, 0]) - (X[t, 2] - X[t, 0]) * (Y[t, 1] - Y[t, 0]))
        sel = np.where(np.all(lo <= (X[t].max(), Y[t].max()), axis=1) & np.all(hi >= (X[t].min(), Y[t].min()), axis=1))[0]
        ar = np.array([_area(_clip_poly([tuple(p) for p in E[e]], T)) for e in sel])
        want[t] = (ar * m.coeff[sel]).sum() / area
    got = o.finest_coef()
    assert got.shape == want.shape
    assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()
    # the averages lie within the fine values' range (a = 0 outside Omega only lowers them)
    assert got.max() <= m.coeff.max() * (1 + 1e-13)


def test_mixed_pcg_and_iteration_reach_the_dense_solution(gen):
    m = _mixed_domain(gen, 17, "hole", "outer")
    b = None
    for layers in (-1, 2):
        o = oracle.Oracle(m, coarse_max=8, nb_layers=layers)
        assert o.c < o.J
        if b is None:
            b = o.mass_apply(gen.nodal_uniform(m, 2))
            ref = np.linalg.solve(o.A().toarray(), b)
        u, st, it, _ = o.solve(b, rtol=1e-13)
        assert st == 0 and np.linalg.norm(u - ref) <= 1e-11 * np.linalg.norm(ref)
        if layers < 0:
            # without the correction the cycle is symmetric and B is SPD
            n = o.nfree
            B = np.stack([o.precond(np.eye(n)[k]) for k in range(n)], 1)
            assert np.abs(B - B.T).max() <= 1e-12 * np.abs(B).max()
            assert np.linalg.eigvalsh(0.5 * (B + B.T)).min() > 0
        oi = oracle.Oracle(m, coarse_max=8, nb_layers=layers, iteration=1, max_iter=200)
        u, st, it, hist = oi.solve(b, rtol=1e-10)
        assert st == 0 and np.linalg.norm(u - ref) <= 1e-8 * np.linalg.norm(ref)


def test_near_boundary_correction_speeds_up_the_mixed_iteration(gen):
    # Sec. 3.5: the non-matching boundaries of the auxiliary grids slow the
    # cycle near the boundary; the correction on j = 2 layers restores a
    # mesh-independent rate
    rates = {}
    for n in (17, 33, 65):
        m = _mixed_domain(gen, n, "L", "inner")
        for layers in (-1, 2):
            o = oracle.Oracle(m, coarse_max=8, nb_layers=layers, iteration=1, max_iter=300)
            b = o.mass_apply(gen.nodal_uniform(m, 1))
            u, st, it, hist = o.solve(b, rtol=1e-8)
            assert st == 0
            rates[n, layers] = (hist[-1] / hist[0]) ** (1.0 / it)
    for n in (17, 33, 65):
        assert rates[n, 2] < 0.8 * rates[n, -1], rates
        assert rates[n, 2] <= 0.25, rates


# --------------------------------------------------------------------------
# Values printed by the paper: Table t_gmg (Sec. 6), tests/golden/t_gmg_dofs.txt
# --------------------------------------------------------------------------

def _golden_gmg():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "t_gmg_dofs.txt")
    rows = []
    with open(path) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                lab, n = line.split()
                rows.append((int(lab), int(n)))
    return rows


def test_gmg_table_sizes_are_uniform_grid_vertices(gen):
    rows = _golden_gmg()
    assert [r[0] for r in rows] == [9, 10, 11]
    for lab, n in rows:
        assert n == (2 ** (lab + 1) + 1) ** 2
    # the two smaller grids built and counted: vertices as printed, free unknowns
    # (interior vertices) as the text's n_l = (2^l - 1)^2 with l = label + 1
    for lab, n in rows[:2]:
        side = 2 ** (lab + 1) + 1
        m = gen.grid2d(side, 1, jitter=0.0, random_diag=False)
        assert m.nv == n
        o = oracle.Oracle(m, stage=0)
        assert o.nfree == (2 ** (lab + 1) - 1) ** 2
    # and the auxiliary hierarchy of a uniform grid has n_l = (2^l - 1)^2 free nodes per level
    m = gen.grid2d(129, 1, jitter=0.0, random_diag=False)
    o = oracle.Oracle(m)
    assert [o.info("nlevel", l) for l in range(o.J + 1)] == [(2 ** l - 1) ** 2 for l in range(o.J + 1)]


@pytest.mark.parametrize("shape,where", [("L", "inner"), ("hole", "outer"), ("hole", "inner")])
def test_mixed_hierarchy_keeps_the_in_place_properties(gen, shape, where):
    # What lets one in-place auxiliary vector carry the non-nested mixed
    # hierarchy: a free node never turns Dirichlet on the next level, a node
    # that left the grid never comes back, and every interpolation row is an
    # identity, a midpoint (one or two halves) or empty
    left = 0  # node-levels where a free node leaves the grid
    for n, seed in ((17, 1), (33, 2), (33, 3)):
        m = _mixed_domain(gen, n, shape, where, seed=seed)
        o = oracle.Oracle(m, coarse_max=8)
        ever = set(o.level_keys(o.c).tolist())
        for l in range(o.c + 1, o.J + 1):
            Fc, Ff = set(o.level_keys(l - 1).tolist()), set(o.level_keys(l).tolist())
            allf = set(o.level_keys(l, all_nodes=True).tolist())
            assert not (Fc & (allf - Ff)), (n, l)
            assert not ((ever - Fc) & Ff), (n, l)
            left += len(Fc - allf)
            I = o.I(l).tocsr()
            for r in range(I.shape[0]):
                vs = sorted(v for v in I.data[I.indptr[r]:I.indptr[r + 1]] if v != 0)
                assert vs in ([], [1.0], [0.5], [0.5, 0.5]), (n, l, vs)
            ever |= Fc | Ff
    # a Neumann cut through the lattice thins the coverage level by level
    assert left > 0 if where == "inner" else left == 0


# ------------------------------------------------ mixed boundaries in 3D (R18)

def _xyz3_keys(keys):
    k = keys.astype(np.uint64)
    out = []
    for a in range(3):
        v = np.zeros_like(k)
        for j in range(21):
            v |= ((k >> np.uint64(3 * j + a)) & np.uint64(1)) << np.uint64(j)
        out.append(v)
    return out


def _pts3(o, keys):
    a = o.root()
    lb = o.info("LB")
    return np.stack([a[k] + np.ldexp(v.astype(np.float64), -lb) * a[3] for k, v in enumerate(_xyz3_keys(keys))], -1)


def _fr3(p):
    return tuple(Fraction(float(v)) for v in p)


def _gamma_d3(m):
    f = np.sort(np.concatenate([m.elems[:, [1, 2, 3]], m.elems[:, [0, 2, 3]], m.elems[:, [0, 1, 3]],
                                m.elems[:, [0, 1, 2]]]), axis=1)
    uniq, cnt = np.unique(f, axis=0, return_counts=True)
    bd = uniq[cnt == 1]
    bd = bd[(m.bflag[bd] == 1).all(axis=1)]
    return [[_fr3(m.verts[v]) for v in t] for t in bd]


def _sub(a, b):
    return tuple(x - y for x, y in zip(a, b))


def _cross(a, b):
    return (a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0])


def _dot(a, b):
    return sum(x * y for x, y in zip(a, b))


def _tri_cuts_open_tet(T, K):
    # exact: clip the triangle by the four closed half-spaces of K; the interior
    # of K is met when a piece of positive area remains and the triangle does
    # not lie in the plane of a face of K
    faces = [(1, 2, 3, 0), (0, 2, 3, 1), (0, 1, 3, 2), (0, 1, 2, 3)]
    poly = list(T)
    for a, b, c, opp in faces:
        n = _cross(_sub(K[b], K[a]), _sub(K[c], K[a]))
        if _dot(n, _sub(K[opp], K[a])) < 0:
            n = tuple(-x for x in n)
        if all(_dot(n, _sub(p, K[a])) == 0 for p in T):
            return False
        side = [_dot(n, _sub(p, K[a])) for p in poly]
        out = []
        for i in range(len(poly)):
            p, q, sp_, sq = poly[i], poly[(i + 1) % len(poly)], side[i], side[(i + 1) % len(poly)]
            if sp_ >= 0:
                out.append(p)
            if (sp_ > 0 and sq < 0) or (sp_ < 0 and sq > 0):
                t = sp_ / (sp_ - sq)
                out.append(tuple(p[k] + t * (q[k] - p[k]) for k in range(3)))
        poly = out
        if len(poly) < 3:
            return False
    area = (0, 0, 0)
    for i in range(1, len(poly) - 1):
        area = tuple(x + y for x, y in zip(area, _cross(_sub(poly[i], poly[0]), _sub(poly[i + 1], poly[0]))))
    return area != (0, 0, 0)


def _on_tri3(T, p):
    n = _cross(_sub(T[1], T[0]), _sub(T[2], T[0]))
    if _dot(n, _sub(p, T[0])) != 0:
        return False
    s = [_dot(n, _cross(_sub(T[(k + 1) % 3], T[k]), _sub(p, T[k]))) for k in range(3)]
    return all(v >= 0 for v in s) or all(v <= 0 for v in s)


def test_mixed3_cube_levels_are_the_natural_boundary_7_point(gen):
    # Unjittered cube, Neumann on x = 1: every tetrahedron is kept.  On levels no
    # finer than the mesh the free nodes are the lattice nodes off the five
    # Dirichlet faces and A_l = h (K (x) M (x) M + M (x) K (x) M + M (x) M (x) K)
    # with the natural condition on x = 1 (1D stiffness with last diagonal 1,
    # lumped 1D mass with last entry 1/2).  On finer levels, lattice nodes inside
    # the face triangles whose three vertices are on the face's rim (Gamma_D)
    # are Dirichlet as well.
    m = gen.grid3d(9, 1, jitter=0.0)
    x = m.verts
    m.bflag = m.bflag.copy()
    m.bflag[(x[:, 0] == 1.0) & (x[:, 1] > 0) & (x[:, 1] < 1) & (x[:, 2] > 0) & (x[:, 2] < 1)] = NEUMANN
    o = oracle.Oracle(m, coarse_max=1)
    top = 1 << o.info("LB")
    gd = _gamma_d3(m)
    for l in range(1, o.J + 1):
        assert {tuple(t) for t in o.level_tet(l).tolist()} == {tuple(t) for t in o.level_alltet(l).tolist()}, l
        ak = o.level_keys(l, all_nodes=True)
        X, Y, Z = _xyz3_keys(ak)
        off = (X > 0) & (Y > 0) & (Y < top) & (Z > 0) & (Z < top)
        P = _pts3(o, ak)
        # exact on-Gamma_D test, for the nodes off the Dirichlet faces (the others are out anyway)
        on_gd = np.zeros(ak.size, bool)
        for i in np.where(off)[0]:
            q = _fr3(P[i])
            on_gd[i] = any(_on_tri3(T, q) for T in gd
                           if all(min(v[k] for v in T) <= q[k] <= max(v[k] for v in T) for k in range(3)))
        assert np.array_equal(o.level_keys(l), np.sort(ak[off & ~on_gd])), l
        if 2 ** l > 8:
            assert on_gd[off].any()                 # finer than the mesh: rim triangles bite
            continue
        keys = o.level_keys(l)
        X, Y, Z = _xyz3_keys(keys)
        step = top >> l
        nx, ny = 2 ** l, 2 ** l - 1
        rm = ((Z // step - 1) * ny * nx + (Y // step - 1) * nx + (X // step - 1)).astype(np.int64)
        Pm = np.zeros((keys.size, keys.size))
        Pm[rm, np.arange(keys.size)] = 1
        Ky = sp.diags([-1.0, 2.0, -1.0], [-1, 0, 1], shape=(ny, ny)).toarray()
        Kx = sp.diags([-1.0, 2.0, -1.0], [-1, 0, 1], shape=(nx, nx)).toarray()
        Kx[-1, -1] = 1
        Mx = np.eye(nx)
        Mx[-1, -1] = 0.5
        My = np.eye(ny)
        W = (np.kron(np.kron(Ky, My), Mx) + np.kron(np.kron(My, Ky), Mx) + np.kron(np.kron(My, My), Kx)) / 2 ** l
        assert np.abs(Pm @ o.A(l).toarray() @ Pm.T - W).max() <= 1e-14 * np.abs(W).max(), l


def _mixed3_lprism(gen):
    # jittered L prism: Dirichlet on the jagged cut, Neumann on the face x = 0
    m = gen.grid3d_domain(5, 2, "L")
    x = m.verts
    m.bflag = m.bflag.copy()
    inner = (x[:, 1] > 0) & (x[:, 1] < 1) & (x[:, 2] > 0) & (x[:, 2] < 1)
    m.bflag[(m.bflag == 1) & (x[:, 0] == 0) & inner] = NEUMANN
    return m


def test_mixed3_kept_tets_and_free_nodes_exact(gen):
    m = _mixed3_lprism(gen)
    o = oracle.Oracle(m, coarse_max=8)
    gd = _gamma_d3(m)
    E = m.verts[m.elems]
    lo, hi = E.min(axis=1), E.max(axis=1)
    rng = np.random.default_rng(5)
    cut_any = False
    for l in range(o.J + 1):
        allt, kept = o.level_alltet(l), {tuple(t) for t in o.level_tet(l).tolist()}
        P = _pts3(o, allt.reshape(-1)).reshape(-1, 4, 3)
        dirn = set()
        for t in range(allt.shape[0]):
            K = [_fr3(p) for p in P[t]]
            tlo, thi = P[t].min(axis=0), P[t].max(axis=0)
            cut = any(_tri_cuts_open_tet(T, K) for T in gd
                      if all(min(v[k] for v in T) <= thi[k] and max(v[k] for v in T) >= tlo[k] for k in range(3)))
            key = tuple(allt[t].tolist())
            if cut:
                cut_any = True
                dirn.update(key)
                assert key not in kept, (l, t)
            elif key not in kept:
                # left out without a cut: no fine element covers any of 20 random interior points
                w = rng.dirichlet(np.ones(4), size=20)
                pts = w @ P[t]
                sel = np.where(np.all(lo <= thi, axis=1) & np.all(hi >= tlo, axis=1))[0]
                for e in sel:
                    Te = E[e]
                    B = np.linalg.solve((Te[1:] - Te[0]).T, (pts - Te[0]).T).T
                    lam = np.concatenate([1 - B.sum(1, keepdims=True), B], 1)
                    assert not np.any(lam.min(1) > 1e-12), (l, t)
        nodes = sorted({k for t in kept for k in t})
        Pn = _pts3(o, np.array(nodes, dtype=np.uint64))
        def on_gd(p):
            q = _fr3(p)
            return any(_on_tri3(T, q) for T in gd if all(min(v[k] for v in T) <= q[k] <= max(v[k] for v in T)
                                                       for k in range(3)))
        free = [k for k, p in zip(nodes, Pn) if k not in dirn and not on_gd(p)]
        assert o.level_keys(l).tolist() == free, l
    assert cut_any


def _solid_angles(o, tets):
    # solid angle at each vertex of each tetrahedron (Van Oosterom-Strackee)
    P = _pts3(o, tets.reshape(-1)).reshape(-1, 4, 3)
    ang = {}
    for t in range(tets.shape[0]):
        for v in range(4):
            a, b, c = (P[t][(v + k) % 4] - P[t][v] for k in (1, 2, 3))
            la, lb, lc = np.linalg.norm(a), np.linalg.norm(b), np.linalg.norm(c)
            num = abs(np.dot(a, np.cross(b, c)))
            den = la * lb * lc + np.dot(a, b) * lc + np.dot(a, c) * lb + np.dot(b, c) * la
            ang[int(tets[t, v])] = ang.get(int(tets[t, v]), 0.0) + 2 * np.arctan2(num, den)
    return ang


@pytest.mark.parametrize("layers", [0, 1])
def test_mixed3_near_boundary_sets_are_graph_balls(gen, layers):
    from scipy.sparse.csgraph import shortest_path
    m = _mixed3_lprism(gen)
    o = oracle.Oracle(m, coarse_max=8, nb_layers=layers)
    for l in range(o.c + 1, o.J + 1):
        tets = o.level_tet(l)
        nodes = np.unique(tets.reshape(-1))
        pos = {int(k): i for i, k in enumerate(nodes)}
        r, c = [], []
        for t in tets.tolist():
            for a in range(4):
                for b in range(4):
                    if a != b:
                        r.append(pos[t[a]])
                        c.append(pos[t[b]])
        G = sp.coo_matrix((np.ones(len(r)), (r, c)), shape=(nodes.size, nodes.size)).tocsr()
        bnd = [pos[k] for k, a in _solid_angles(o, tets).items() if abs(a - 4 * np.pi) > 1e-9]
        dist = shortest_path(G, directed=False, unweighted=True, indices=bnd).min(axis=0)
        ball = set(int(k) for k in nodes[dist <= layers + 1])
        keys = o.level_keys(l)
        assert o.near_boundary_set(l).tolist() == [i for i, k in enumerate(keys.tolist()) if k in ball], l


def test_mixed3_interpolation_cycle_and_solve(gen):
    m = _mixed3_lprism(gen)
    o0 = oracle.Oracle(m)
    J = o0.J
    rng = np.random.default_rng(9)
    # nodal interpolation by point location over all kept coarse tetrahedra
    o = oracle.Oracle(m, coarse_max=8)
    for l in range(o.c + 1, o.J + 1):
        ct, ck = o.level_tet(l - 1), o.level_keys(l - 1)
        ec = rng.standard_normal(ck.size)
        val = dict(zip(ck.tolist(), ec))
        CP = _pts3(o, ct.reshape(-1)).reshape(-1, 4, 3)
        FP = _pts3(o, o.level_keys(l))
        Minv = np.linalg.inv(np.transpose(CP[:, 1:] - CP[:, :1], (0, 2, 1)))   # per tet: point -> (l1, l2, l3)
        cval = np.array([[val.get(int(k), 0.0) for k in t] for t in ct])
        want = np.zeros(len(FP))
        for i, p in enumerate(FP):
            B = np.einsum("tij,tj->ti", Minv, p - CP[:, 0])
            lam = np.concatenate([1 - B.sum(1, keepdims=True), B], 1)
            hit = np.where(lam.min(1) >= -1e-12)[0]
            if hit.size:
                want[i] = lam[hit[0]] @ cval[hit[0]]
        assert np.abs(o.I(l) @ ec - want).max() <= 1e-12 * max(1.0, np.abs(want).max()), l
    # two levels without smoothing: coarse solve, then the J_{l,j} solve
    o2 = oracle.Oracle(m, coarse_max=o0.info("nlevel", J - 1), nu_pre=0, nu_post=0, nb_layers=1)
    assert o2.c == J - 1
    AJ, Ac, I = o2.A(J).toarray(), o2.A(J - 1).toarray(), o2.I(J).toarray()
    f = rng.standard_normal(AJ.shape[0])
    u = I @ np.linalg.solve(Ac, I.T @ f)
    nb = o2.near_boundary_set(J)
    assert nb.size > 0
    u[nb] += np.linalg.solve(AJ[np.ix_(nb, nb)], (f - AJ @ u)[nb])
    assert np.abs(o2.vcycle(f) - u).max() <= 1e-11 * np.abs(u).max()
    # PCG reaches the dense solution with and without the correction
    for layers in (-1, 1):
        o3 = oracle.Oracle(m, coarse_max=8, nb_layers=layers)
        b = o3.mass_apply(gen.nodal_uniform(m, 2))
        ref = np.linalg.solve(o3.A().toarray(), b)
        u3, st, it, _ = o3.solve(b, rtol=1e-13)
        assert st == 0 and np.linalg.norm(u3 - ref) <= 1e-11 * np.linalg.norm(ref)


# --------------------------------------------------------------------------
# Colouring option 2: lattice parity on bipartite auxiliary levels (R10)
# --------------------------------------------------------------------------

def _check_valid_classes(A, smooth, cstart):
    A = A.tocsr()
    d = A.diagonal()
    cls = np.full(A.shape[0], -1)
    for c in range(len(cstart) - 1):
        cls[smooth[cstart[c]:cstart[c + 1]]] = c
    C = A.tocoo()
    off = (C.row != C.col) & (np.abs(C.data) > 1e-12 * np.sqrt(np.abs(d[C.row] * d[C.col])))
    r, c = C.row[off], C.col[off]
    both = (cls[r] >= 0) & (cls[c] >= 0)
    assert not np.any(cls[r][both] == cls[c][both])


@pytest.mark.parametrize("case", ["graded2d", "kuhn3d"])
def test_parity_colouring_uses_two_classes_where_bipartite(gen, case):
    m = gen.grid2d(129, 1, graded=True) if case == "graded2d" else gen.grid3d(9, 1)
    o = oracle.Oracle(m, colouring=2)
    classes = []
    for l in range(o.c + 1, o.J + 1):
        sm, cs, _ = o.smoothing_set(l)
        _check_valid_classes(o.A(l), sm, cs)
        classes.append(cs.size - 1)
    # the uniform levels are bipartite (right-isosceles triangles / Kuhn
    # tetrahedra: no coupling across a hypotenuse), the first one at least
    assert classes[0] == 2
    if case == "graded2d":
        assert max(classes) > 2              # closure transitions: odd cycles, default colouring
    else:
        assert all(c == 2 for c in classes)


def test_parity_colouring_keeps_the_preconditioner_spd_and_exact(gen):
    m = gen.grid3d(7, 2)
    o = oracle.Oracle(m, colouring=2, coarse_max=8)
    assert o.c < o.J
    n = o.nfree
    B = np.stack([o.precond(np.eye(n)[k]) for k in range(n)], 1)
    assert np.abs(B - B.T).max() <= 1e-12 * np.abs(B).max()
    assert np.linalg.eigvalsh(0.5 * (B + B.T)).min() > 0
    b = o.mass_apply(gen.nodal_uniform(m, 3))
    u, st, it, _ = o.solve(b, rtol=1e-13)
    ref = np.linalg.solve(o.A().toarray(), b)
    assert st == 0 and np.linalg.norm(u - ref) <= 1e-11 * np.linalg.norm(ref)

"""The library's host part of the setup against the oracle, on CPU.

The closure, the auxiliary grids (box and Dirichlet), the free nodes of
every level, the smoothing sets, the level simplices with their averaged
coefficients, the new nodes with their parents and the Scott-Zhang transfer
rows come from the library's own sources (`aux_setup.cpp`, `aux_setup3.cpp`,
the row routine of `sz_row.h`), built here with g++ around
`tests/host_setup_shim.cpp` and run on the oracle's cluster tree (the tree
itself is checked bit for bit on the GPU).  Integer results must be equal;
the level operators rediscretised from the shim's simplices agree with the
oracle's Galerkin products to 1e-12 of the largest entry (1e-10 on 3D
domains cut by Omega, whose boundary tetrahedra are clipped by two different
exact methods), and P to 1e-11.
"""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest
import scipy.sparse as sp

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1410_2153_gb300", "csrc")


@pytest.fixture(scope="module")
def shim(tmp_path_factory):
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    cuda_inc, cuda_lib = os.path.join(cuda, "include"), os.path.join(cuda, "lib64")
    if not shutil.which("g++") or not os.path.exists(os.path.join(cuda_inc, "cuda_runtime.h")):
        pytest.skip("g++ or the CUDA headers are missing")
    out = str(tmp_path_factory.mktemp("shim") / "libshim.so")
    # (the CUDA runtime is linked for the device-buffer types in the shared
    # headers; nothing here calls it)
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-pthread", "-I", cuda_inc,
                           os.path.join(ROOT, "tests", "host_setup_shim.cpp"), os.path.join(CSRC, "aux_setup.cpp"),
                           os.path.join(CSRC, "aux_setup3.cpp"), "-o", out, "-L", cuda_lib, "-lcudart",
                           "-Wl,-rpath," + cuda_lib])
    lib = ctypes.CDLL(out)
    lib.shim_build.restype = ctypes.c_void_p
    lib.shim_build.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                               ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                               ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                               ctypes.c_int]
    lib.shim_error.restype = ctypes.c_char_p
    lib.shim_error.argtypes = [ctypes.c_void_p]
    lib.shim_free.argtypes = [ctypes.c_void_p]
    lib.shim_get.restype = ctypes.c_int64
    lib.shim_get.argtypes = [ctypes.c_void_p, ctypes.c_char_p, ctypes.c_int, ctypes.c_void_p]
    lib.shim_keyindex.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p, ctypes.c_int64,
                                  ctypes.c_void_p]
    lib.shim_nbsolve.restype = ctypes.c_int64
    lib.shim_nbsolve.argtypes = [ctypes.c_int64] + [ctypes.c_void_p] * 5
    lib.shim_level_nbsolve.restype = ctypes.c_int64
    lib.shim_level_nbsolve.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    lib.shim_bf16.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64]
    return lib


@pytest.mark.parametrize("kind", ["empty", "one", "uniform", "clustered", "top_bits"])
@pytest.mark.parametrize("bits", [1, 8, 20])
def test_key_index_matches_binary_search(shim, kind, bits):
    rng = np.random.default_rng(bits)
    if kind == "empty":
        keys = np.zeros(0, np.uint64)
    elif kind == "one":
        keys = np.array([12345], np.uint64)
    elif kind == "uniform":
        keys = np.unique(rng.integers(0, 2 ** 62, 5000, dtype=np.uint64))
    elif kind == "clustered":                    # graded meshes: keys crowd near one corner
        keys = np.unique(np.concatenate([rng.integers(0, 2 ** 20, 4000, dtype=np.uint64),
                                         rng.integers(0, 2 ** 62, 100, dtype=np.uint64)]))
    else:
        keys = np.unique(rng.integers(2 ** 63 - 2 ** 40, 2 ** 63, 3000, dtype=np.uint64))
    present = keys[rng.integers(0, max(1, keys.size), 200)] if keys.size else np.zeros(0, np.uint64)
    q = np.concatenate([present, rng.integers(0, 2 ** 63, 300, dtype=np.uint64), keys[:1] + np.uint64(1),
                        np.array([0, 2 ** 63 - 1], np.uint64)]).astype(np.uint64)
    out = np.empty(q.size, np.int32)
    shim.shim_keyindex(keys.ctypes.data, keys.size, bits, q.ctypes.data, q.size, out.ctypes.data)
    pos = np.searchsorted(keys, q)
    want = np.where((pos < keys.size) & (keys[np.minimum(pos, max(keys.size - 1, 0))] == q) if keys.size
                    else np.zeros(q.size, bool), pos, -1)
    assert np.array_equal(out, want)


def _get(lib, h, what, l, dt):
    n = lib.shim_get(h, what.encode(), l, None)
    assert n >= 0, what
    a = np.empty(n, dt)
    if n:
        lib.shim_get(h, what.encode(), l, a.ctypes.data_as(ctypes.c_void_p))
    return a


def _deinterleave(keys, dim, bits):
    k = keys.astype(np.uint64)
    out = []
    for a in range(dim):
        v = np.zeros_like(k)
        for j in range(bits):
            v |= ((k >> np.uint64(dim * j + a)) & np.uint64(1)) << np.uint64(j)
        out.append(v)
    return out


def _interleave(coords, dim):
    out = np.zeros_like(coords[0], dtype=np.uint64)
    for a, c in enumerate(coords):
        c = c.astype(np.uint64)
        for j in range(32 if dim == 2 else 21):
            out |= ((c >> np.uint64(j)) & np.uint64(1)) << np.uint64(dim * j + a)
    return out


def _stiffness(P, a):
    """P1 element stiffness (per simplex: (dim+1) x (dim+1)) times the coefficient a."""
    dim = P.shape[2]
    e = P[:, 1:, :] - P[:, :1, :]              # rows: edge vectors from vertex 0
    G = np.linalg.inv(e)                       # column k: gradient of lambda_(k+1)
    grads = np.concatenate([-G.sum(axis=2)[:, None, :], G.transpose(0, 2, 1)], axis=1)
    vol = np.abs(np.linalg.det(e)) / (2.0 if dim == 2 else 6.0)
    return a[:, None, None] * vol[:, None, None] * np.einsum("tir,tjr->tij", grads, grads)


def _compare(lib, m, o, params, dim, op_tol):
    segs = o.tree_levels()
    splits = [s_[s_[:, 3] == 1, 0].astype(np.uint64) for s_ in segs]
    while splits and len(splits[-1]) == 0:
        splits.pop()
    cnt = np.array([len(s_) for s_ in splits], np.int64)
    flat = np.concatenate(splits) if splits else np.zeros(0, np.uint64)
    r = o.root()
    amin = np.ascontiguousarray(r[:dim], dtype=np.float64)
    L = float(r[3])
    X = np.ascontiguousarray(m.verts, dtype=np.float64)
    E = np.ascontiguousarray(m.elems, dtype=np.int32)
    B = np.ascontiguousarray(m.bflag, dtype=np.uint8)
    C = None if m.coeff is None else np.ascontiguousarray(m.coeff, dtype=np.float64)
    h = lib.shim_build(dim, m.nv, X.ctypes.data, m.ne, E.ctypes.data, B.ctypes.data,
                       None if C is None else C.ctypes.data, len(cnt), cnt.ctypes.data, flat.ctypes.data,
                       amin.ctypes.data, L, params.get("n_min", 3), params.get("coarse_max", 512),
                       params.get("smoothing", 0), params.get("nb_layers", 2))
    try:
        assert lib.shim_error(h) == b"", lib.shim_error(h)
        # closure: the split boxes of every depth
        for d, arr in enumerate(o.boxes()):
            spl = arr[arr[:, 1] == 1, 0]
            bits = 32 if dim == 2 else 21
            coords = [(spl >> np.uint64(bits * a)) & np.uint64((1 << bits) - 1) for a in range(dim)]
            want = np.sort(_interleave(coords, dim))
            assert np.array_equal(_get(lib, h, "split", d, np.uint64), want), ("closure", d)
        J, c = lib.shim_get(h, b"J", 0, None), lib.shim_get(h, b"c", 0, None)
        assert J == o.J and c == o.c, (J, o.J, c, o.c)
        ak = _get(lib, h, "aux_key", 0, np.uint64)
        assert np.array_equal(ak, o.level_keys(o.J))
        nl = _get(lib, h, "nlevel", 0, np.int64)
        assert [int(v) for v in nl] == [o.info("nlevel", l) for l in range(J + 1)]
        assert np.array_equal(ak[_get(lib, h, "coarse_id", 0, np.int32)], o.level_keys(c))
        lb = 31 if dim == 2 else o.info("LB")
        for l in range(c + 1, J + 1):
            sm = _get(lib, h, "smooth", l, np.int32)
            lk = o.level_keys(l)
            assert np.array_equal(np.sort(ak[sm]), np.sort(lk[o.smoothing_set(l)[0]])), ("smooth", l)
            # the level operator on the rows and columns of N~_l, rediscretised from the
            # shim's simplices, against the oracle's Galerkin product
            tk = _get(lib, h, "tri_key", l, np.uint64)
            tid = _get(lib, h, "tri_id", l, np.int32).reshape(-1, dim + 1)
            tc = _get(lib, h, "tri_coef", l, np.float64)
            P = np.stack([amin[a] + np.ldexp(v.astype(np.float64), -lb) * L
                          for a, v in enumerate(_deinterleave(tk, dim, 32 if dim == 2 else 21))], -1)
            K = _stiffness(P.reshape(-1, dim + 1, dim), tc)
            inset = np.zeros(len(ak), bool)
            inset[sm] = True
            got = {}
            for t in range(len(tc)):
                for i in range(dim + 1):
                    for j in range(dim + 1):
                        a_, b_ = tid[t, i], tid[t, j]
                        if a_ >= 0 and b_ >= 0 and (inset[a_] or inset[b_]):
                            got[(a_, b_)] = got.get((a_, b_), 0.0) + K[t, i, j]
            idx = {int(k): i for i, k in enumerate(ak)}
            Ag = o.A(l).tocoo()
            want = {}
            for r_, c_, v_ in zip(Ag.row, Ag.col, Ag.data):
                ri, ci = idx[int(lk[r_])], idx[int(lk[c_])]
                if inset[ri] or inset[ci]:
                    want[(ri, ci)] = v_
            scale = max(abs(v) for v in want.values())
            err = max(abs(got.get(k, 0.0) - want.get(k, 0.0)) for k in set(got) | set(want))
            assert err <= op_tol * scale, ("A level", l, err)
            # new nodes: parents against the oracle's interpolation rows
            nid = _get(lib, h, "new_id", l, np.int32)
            p0 = _get(lib, h, "new_p0", l, np.int32)
            p1 = _get(lib, h, "new_p1", l, np.int32)
            I = o.I(l).tocsr()
            lkc = o.level_keys(l - 1)
            lpos = {int(k): i for i, k in enumerate(lk)}
            for a_, b_, c2 in zip(nid, p0, p1):
                row = I[lpos[int(ak[a_])]]
                w = {int(lkc[j]): v for j, v in zip(row.indices, row.data)}
                g = {}
                for q in (b_, c2):
                    if q >= 0:
                        g[int(ak[q])] = g.get(int(ak[q]), 0.0) + 0.5
                assert w.keys() == g.keys() and all(abs(w[k] - g[k]) < 1e-15 for k in w), ("I", l)
            assert set(int(k) for k in lk) - set(int(k) for k in lkc) == set(int(ak[a_]) for a_ in nid)
        Pr = _get(lib, h, "P_r", 0, np.int32)
        Pc = _get(lib, h, "P_c", 0, np.int32)
        Pv = _get(lib, h, "P_v", 0, np.float64)
        Ph = sp.csr_matrix((Pv, (Pr, Pc)), shape=(o.nfree, len(ak)))
        assert abs(Ph - o.P()).max() <= 1e-11
    finally:
        lib.shim_free(h)


def _cases(gen):
    jump = gen.grid2d(33, 7, graded=True)
    jump.coeff = np.exp(np.random.default_rng(0).normal(size=jump.ne))
    lc = gen.grid2d_domain(17, 3, "L")
    lc.coeff = np.exp(np.random.default_rng(1).normal(size=lc.ne))
    t3 = gen.grid3d(9, 3)
    t3.coeff = gen.subcube_coefficient(t3, 5, ncube=4)
    return {
        "2d_jitter17": (gen.grid2d(17, 3), {}, 2, 1e-12),
        "2d_graded33_lognormal": (jump, {}, 2, 1e-12),
        "2d_graded33_all_levels": (gen.grid2d(33, 4, graded=True), {"smoothing": 1}, 2, 1e-12),
        "2d_L17_lognormal": (lc, {}, 2, 1e-12),
        "2d_hole33_c10": (gen.grid2d_domain(33, 5, "hole"), {"coarse_max": 10}, 2, 1e-12),
        "3d_kuhn5": (gen.grid3d(5, 1), {}, 3, 1e-12),
        "3d_kuhn9_jump": (t3, {}, 3, 1e-12),
        "3d_kuhn9_nmin6": (gen.grid3d(9, 8), {"n_min": 6}, 3, 1e-12),
        "3d_L7": (gen.grid3d_domain(7, 1, "L"), {}, 3, 1e-10),
        "3d_cavity7": (gen.grid3d_domain(7, 2, "hole"), {"coarse_max": 10}, 3, 1e-10),
        # small and degenerate hierarchies: one free vertex, a coarse level of one
        # node, one-element leaves, every level smoothed with a tiny coarse cap
        "2d_grid3": (gen.grid2d(3, 1), {}, 2, 1e-12),
        "2d_L5_c1": (gen.grid2d_domain(5, 1, "L"), {"coarse_max": 1}, 2, 1e-12),
        "2d_L9_nmin1": (gen.grid2d_domain(9, 3, "L"), {"n_min": 1}, 2, 1e-12),
        "2d_L9_all_c2": (gen.grid2d_domain(9, 3, "L"), {"smoothing": 1, "coarse_max": 2}, 2, 1e-12),
        "3d_grid3": (gen.grid3d(3, 1), {}, 3, 1e-12),
        "3d_L5_nmin1": (gen.grid3d_domain(5, 3, "L"), {"n_min": 1}, 3, 1e-10),
    }


@pytest.mark.parametrize("name", ["2d_jitter17", "2d_graded33_lognormal", "2d_graded33_all_levels",
                                  "2d_L17_lognormal", "2d_hole33_c10", "3d_kuhn5", "3d_kuhn9_jump",
                                  "3d_kuhn9_nmin6", "3d_L7", "3d_cavity7", "2d_grid3", "2d_L5_c1",
                                  "2d_L9_nmin1", "2d_L9_all_c2", "3d_grid3", "3d_L5_nmin1"])
def test_host_setup_matches_oracle(shim, gen, name):
    m, params, dim, op_tol = _cases(gen)[name]
    o = oracle.Oracle(m, **params)
    _compare(shim, m, o, params, dim, op_tol)


# --------------------------------------------------------------------------
# Mixed Dirichlet / Neumann boundaries (2D): the library's host setup of the
# mixed grids against the oracle's construction of the same grids.  The
# library keeps one aux ID per node that is free on some level, free on the
# levels phi <= l < psi; the oracle keeps each level's free nodes.
# --------------------------------------------------------------------------

def _mixed_mesh(gen, kind, n, seed):
    if kind == "square":
        m = gen.grid2d(n, seed)
    elif kind == "graded":
        m = gen.grid2d(n, seed, graded=True)
    else:
        m = gen.grid2d_domain(n, seed, kind)
    x, y = m.verts[:, 0], m.verts[:, 1]
    return m, x, y


def _mixed_cases(gen):
    out = {}
    m, x, y = _mixed_mesh(gen, "square", 17, 1)
    m.bflag = m.bflag.copy()
    m.bflag[(x == 1.0) & (y > 0) & (y < 1)] = 2
    out["square17_right"] = (m, {})
    m, x, y = _mixed_mesh(gen, "L", 17, 2)
    m.bflag = m.bflag.copy()
    m.bflag[(m.bflag == 1) & (x > 0) & (x < 1) & (y > 0) & (y < 1)] = 2
    out["L17_cut_c8"] = (m, {"coarse_max": 8})
    m, x, y = _mixed_mesh(gen, "hole", 17, 2)
    m.bflag = m.bflag.copy()
    m.bflag[(m.bflag == 1) & (x == 0) & (y > 0) & (y < 1)] = 2
    m.coeff = np.exp(np.random.default_rng(4).normal(size=m.ne))
    out["hole17_left_lognormal"] = (m, {"coarse_max": 8})
    m, x, y = _mixed_mesh(gen, "L", 33, 3)
    m.bflag = m.bflag.copy()
    m.bflag[(m.bflag == 1) & (x > 0) & (x < 1) & (y > 0) & (y < 1)] = 2
    out["L33_cut_nb0"] = (m, {"coarse_max": 8, "nb_layers": 0})
    m, x, y = _mixed_mesh(gen, "graded", 33, 5)
    m.bflag = m.bflag.copy()
    m.bflag[((x == 1.0) | (y == 1.0)) & (x > 0) & (y > 0)] = 2
    out["graded33_two_sides_nb3"] = (m, {"coarse_max": 16, "nb_layers": 3})
    m = gen.grid3d(9, 1)
    x = m.verts
    m.bflag = m.bflag.copy()
    m.bflag[(x[:, 0] == 1.0) & (x[:, 1] > 0) & (x[:, 1] < 1) & (x[:, 2] > 0) & (x[:, 2] < 1)] = 2
    out["cube9_face"] = (m, {"coarse_max": 8})
    m = gen.grid3d_domain(5, 2, "L")
    x = m.verts
    m.bflag = m.bflag.copy()
    m.bflag[(m.bflag == 1) & (x[:, 0] == 0) & (x[:, 1] > 0) & (x[:, 1] < 1) & (x[:, 2] > 0) & (x[:, 2] < 1)] = 2
    m.coeff = np.exp(np.random.default_rng(6).normal(size=m.ne))
    out["Lprism5_cut_lognormal"] = (m, {"coarse_max": 8, "nb_layers": 1})
    m = gen.grid3d_domain(7, 3, "L")
    x = m.verts
    m.bflag = m.bflag.copy()
    m.bflag[(m.bflag == 1) & (x[:, 0] > 0) & (x[:, 0] < 1) & (x[:, 1] > 0) & (x[:, 1] < 1)] = 2
    out["Lprism7_neumann_cut"] = (m, {"coarse_max": 8})
    return out


def _compare_mixed(lib, m, o, params):
    segs = o.tree_levels()
    splits = [s_[s_[:, 3] == 1, 0].astype(np.uint64) for s_ in segs]
    while splits and len(splits[-1]) == 0:
        splits.pop()
    cnt = np.array([len(s_) for s_ in splits], np.int64)
    flat = np.concatenate(splits) if splits else np.zeros(0, np.uint64)
    dim = m.dim
    r = o.root()
    amin = np.ascontiguousarray(r[:dim], dtype=np.float64)
    L = float(r[3])
    X = np.ascontiguousarray(m.verts, dtype=np.float64)
    E = np.ascontiguousarray(m.elems, dtype=np.int32)
    B = np.ascontiguousarray(m.bflag, dtype=np.uint8)
    C = None if m.coeff is None else np.ascontiguousarray(m.coeff, dtype=np.float64)
    h = lib.shim_build(dim, m.nv, X.ctypes.data, m.ne, E.ctypes.data, B.ctypes.data,
                       None if C is None else C.ctypes.data, len(cnt), cnt.ctypes.data, flat.ctypes.data,
                       amin.ctypes.data, L, params.get("n_min", 3), params.get("coarse_max", 512), 1,
                       params.get("nb_layers", 2))
    nv_s = dim + 1
    lb = 31 if dim == 2 else o.info("LB")
    try:
        assert lib.shim_error(h) == b"", lib.shim_error(h)
        J, c = lib.shim_get(h, b"J", 0, None), lib.shim_get(h, b"c", 0, None)
        assert J == o.J and c == o.c, (J, o.J, c, o.c)
        ak = _get(lib, h, "aux_key", 0, np.uint64)
        phi = _get(lib, h, "phi", 0, np.int32)
        psi = _get(lib, h, "psi", 0, np.int32)
        assert phi.size == ak.size == psi.size and np.all(phi < psi)
        # the free nodes of every level
        for l in range(J + 1):
            assert np.array_equal(ak[(phi <= l) & (l < psi)], o.level_keys(l)), ("free", l)
        assert np.array_equal(ak[_get(lib, h, "coarse_id", 0, np.int32)], o.level_keys(c))
        for l in range(c + 1, J + 1):
            lk, lkc = o.level_keys(l), o.level_keys(l - 1)
            pos = {int(k): i for i, k in enumerate(lk)}
            sm = _get(lib, h, "smooth", l, np.int32)
            assert np.array_equal(np.sort(ak[sm]), lk), ("smooth", l)
            # the level operator rediscretised from the shim's kept triangles
            tk = _get(lib, h, "tri_key", l, np.uint64)
            tid = _get(lib, h, "tri_id", l, np.int32).reshape(-1, nv_s)
            tc = _get(lib, h, "tri_coef", l, np.float64)
            P = np.stack([amin[a] + np.ldexp(v.astype(np.float64), -lb) * L
                          for a, v in enumerate(_deinterleave(tk, dim, 32 if dim == 2 else 21))], -1)
            K = _stiffness(P.reshape(-1, nv_s, dim), tc)
            n = lk.size
            Ah = np.zeros((n, n))
            for t in range(len(tc)):
                for i in range(nv_s):
                    for j in range(nv_s):
                        if tid[t, i] >= 0 and tid[t, j] >= 0:
                            Ah[pos[int(ak[tid[t, i]])], pos[int(ak[tid[t, j]])]] += K[t, i, j]
            Ao = o.A(l).toarray()
            assert np.abs(Ah - Ao).max() <= 1e-12 * np.abs(Ao).max(), ("A level", l)
            # interpolation: nodes free on both levels carry over, new ones take
            # the midpoint of their free parents
            I = o.I(l).tocsr()
            nid = _get(lib, h, "new_id", l, np.int32)
            p0 = _get(lib, h, "new_p0", l, np.int32)
            p1 = _get(lib, h, "new_p1", l, np.int32)
            assert set(int(ak[q]) for q in nid) == set(int(k) for k in lk) - set(int(k) for k in lkc)
            for a_, b_, c2 in zip(nid, p0, p1):
                row = I[pos[int(ak[a_])]]
                w = {int(lkc[j]): v for j, v in zip(row.indices, row.data) if v != 0}
                g = {}
                for q in (b_, c2):
                    if q >= 0:
                        g[int(ak[q])] = g.get(int(ak[q]), 0.0) + 0.5
                assert w.keys() == g.keys() and all(abs(w[k] - g[k]) < 1e-15 for k in w), ("I", l)
            cpos = {int(k): i for i, k in enumerate(lkc)}
            for k in set(int(k) for k in lk) & set(cpos):
                row = I[pos[k]]
                assert {int(lkc[j]): v for j, v in zip(row.indices, row.data) if v != 0} == {k: 1.0}
            # the near-boundary set J_{l,j}, the block A_l[J,J] the setup assembles from its
            # kept simplices, and the solve with the factor it stores
            nb = _get(lib, h, "nb_id", l, np.int32)
            want = o.near_boundary_set(l)
            assert sorted(pos[int(ak[q])] for q in nb) == want.tolist(), ("J_lj", l)
            if nb.size:
                Bh = sp.csr_matrix((_get(lib, h, "nb_val", l, np.float64), _get(lib, h, "nb_col", l, np.int32),
                                    _get(lib, h, "nb_ptr", l, np.int64)), shape=(nb.size, nb.size)).toarray()
                perm = np.array([pos[int(ak[q])] for q in nb])
                Bo = Ao[np.ix_(perm, perm)]
                assert np.abs(Bh - Bo).max() <= 1e-12 * np.abs(Bo).max(), ("A_JJ", l)
                rhs = np.random.default_rng(l).standard_normal(nb.size)
                xs = np.zeros(nb.size)
                assert lib.shim_level_nbsolve(h, l, rhs.ctypes.data, xs.ctypes.data) == nb.size
                ref = np.linalg.solve(Bo, rhs)
                assert np.abs(xs - ref).max() <= 1e-10 * np.abs(ref).max(), ("J solve", l)
        # Scott-Zhang rows, columns mapped to the oracle's free nodes of level J
        lkJ = {int(k): i for i, k in enumerate(o.level_keys(J))}
        Pr = _get(lib, h, "P_r", 0, np.int32)
        Pc = np.array([lkJ[int(ak[q])] for q in _get(lib, h, "P_c", 0, np.int32)], dtype=np.int64)
        Pv = _get(lib, h, "P_v", 0, np.float64)
        Ph = sp.csr_matrix((Pv, (Pr, Pc)), shape=(o.nfree, len(lkJ)))
        assert abs(Ph - o.P()).max() <= 1e-11
    finally:
        lib.shim_free(h)


@pytest.mark.parametrize("name", ["square17_right", "L17_cut_c8", "hole17_left_lognormal", "L33_cut_nb0",
                                  "graded33_two_sides_nb3", "cube9_face", "Lprism5_cut_lognormal",
                                  "Lprism7_neumann_cut"])
def test_host_setup_mixed_grids_match_oracle(shim, gen, name):
    m, params = _mixed_cases(gen)[name]
    o = oracle.Oracle(m, **params)
    _compare_mixed(shim, m, o, params)


# --------------------------------------------------------------------------
# Near-boundary solve (Algorithm 3): the library's block cyclic reduction over
# breadth-first level sets, against dense solves
# --------------------------------------------------------------------------

def _nbsolve(lib, A, b):
    A = sp.csr_matrix(A)
    ptr = np.ascontiguousarray(A.indptr, dtype=np.int64)
    col = np.ascontiguousarray(A.indices, dtype=np.int32)
    val = np.ascontiguousarray(A.data, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros_like(b)
    nbk = lib.shim_nbsolve(A.shape[0], ptr.ctypes.data, col.ctypes.data, val.ctypes.data, b.ctypes.data,
                           x.ctypes.data)
    return nbk, x


@pytest.mark.parametrize("kind", ["empty", "one", "path", "grid", "two_components", "random_graph"])
def test_nbsolve_random_spd(shim, kind):
    rng = np.random.default_rng(11)
    if kind == "empty":
        A = sp.csr_matrix((0, 0))
    elif kind == "one":
        A = sp.csr_matrix(np.array([[3.0]]))
    elif kind == "path":
        A = sp.diags([-1.0, 2.5, -1.0], [-1, 0, 1], shape=(37, 37))
    elif kind == "grid":               # a 5 x 40 strip: level sets are its cross-sections
        T = sp.diags([-1.0, 2.0, -1.0], [-1, 0, 1], shape=(40, 40))
        S = sp.diags([-1.0, 2.0, -1.0], [-1, 0, 1], shape=(5, 5))
        A = sp.kron(sp.eye(5), T) + sp.kron(S, sp.eye(40)) + 0.01 * sp.eye(200)
    elif kind == "two_components":
        B1 = sp.diags([-1.0, 2.2, -1.0], [-1, 0, 1], shape=(15, 15))
        A = sp.block_diag([B1, B1 + sp.eye(15)])
    else:                              # SPD by diagonal dominance on a random sparse graph
        R = sp.random(120, 120, density=0.03, random_state=3)
        R = R + R.T
        A = -R + sp.diags(np.asarray(abs(R).sum(axis=1)).ravel() + 0.5)
    n = A.shape[0]
    b = rng.standard_normal(n)
    nbk, x = _nbsolve(shim, A, b)
    assert nbk >= 0
    if n:
        ref = np.linalg.solve(A.toarray(), b)
        assert np.abs(x - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("dim", [2, 3])
def test_nbsolve_near_boundary_blocks_of_the_oracle(shim, gen, dim):
    if dim == 2:
        m = gen.grid2d_domain(65, 2, "hole")
        x, y = m.verts[:, 0], m.verts[:, 1]
        m.bflag = m.bflag.copy()
        m.bflag[(m.bflag == 1) & (x > 0) & (x < 1) & (y > 0) & (y < 1)] = 2
    else:
        m = gen.grid3d_domain(7, 3, "L")
        x = m.verts
        m.bflag = m.bflag.copy()
        m.bflag[(m.bflag == 1) & (x[:, 0] > 0) & (x[:, 0] < 1) & (x[:, 1] > 0) & (x[:, 1] < 1)] = 2
    o = oracle.Oracle(m, coarse_max=8, nb_layers=2)
    rng = np.random.default_rng(dim)
    tried = 0
    for l in range(o.c + 1, o.J + 1):
        nb = o.near_boundary_set(l)
        if nb.size == 0:
            continue
        A = o.A(l).tocsr()[nb][:, nb]
        b = rng.standard_normal(nb.size)
        nbk, xs = _nbsolve(shim, A, b)
        ref = np.linalg.solve(A.toarray(), b)
        assert nbk > 0 and np.abs(xs - ref).max() <= 1e-10 * np.abs(ref).max(), (l, nbk)
        tried += 1
    assert tried >= 2


# --------------------------------------------------------------------------
# Mixed grids end to end: one V-cycle (Algorithm 3) run in numpy on the
# library's host structures only -- level intervals phi <= l < psi, carried and
# new nodes with their parents, the rediscretised levels from the emitted
# simplices, the near-boundary factor -- with the oracle's colour classes,
# against the oracle's V-cycle.  This is the composition the device V-cycle
# will follow: a node that leaves the grid receives only its midpoint weights
# in the restriction and is read only as a parent.
# --------------------------------------------------------------------------

def _level_matrix(lib, h, o, l, ak, dim):
    lb = 31 if dim == 2 else o.info("LB")
    r = o.root()
    amin, L = np.asarray(r[:dim]), float(r[3])
    tk = _get(lib, h, "tri_key", l, np.uint64)
    tid = _get(lib, h, "tri_id", l, np.int32).reshape(-1, dim + 1)
    tc = _get(lib, h, "tri_coef", l, np.float64)
    P = np.stack([amin[a] + np.ldexp(v.astype(np.float64), -lb) * L
                  for a, v in enumerate(_deinterleave(tk, dim, 32 if dim == 2 else 21))], -1)
    K = _stiffness(P.reshape(-1, dim + 1, dim), tc)
    rows, cols, vals = [], [], []
    for t in range(len(tc)):
        for i in range(dim + 1):
            for j in range(dim + 1):
                if tid[t, i] >= 0 and tid[t, j] >= 0:
                    rows.append(tid[t, i])
                    cols.append(tid[t, j])
                    vals.append(K[t, i, j])
    return sp.csr_matrix((vals, (rows, cols)), shape=(ak.size, ak.size))


@pytest.mark.parametrize("name", ["L17_cut_c8", "Lprism7_neumann_cut"])
def test_mixed_vcycle_from_library_structures_matches_oracle(shim, gen, name):
    m, params = _mixed_cases(gen)[name]
    o = oracle.Oracle(m, **params)
    dim = m.dim
    segs = o.tree_levels()
    splits = [s_[s_[:, 3] == 1, 0].astype(np.uint64) for s_ in segs]
    while splits and len(splits[-1]) == 0:
        splits.pop()
    cnt = np.array([len(s_) for s_ in splits], np.int64)
    flat = np.concatenate(splits)
    r = o.root()
    amin = np.ascontiguousarray(r[:dim], dtype=np.float64)
    X = np.ascontiguousarray(m.verts, dtype=np.float64)
    E = np.ascontiguousarray(m.elems, dtype=np.int32)
    B = np.ascontiguousarray(m.bflag, dtype=np.uint8)
    C = None if m.coeff is None else np.ascontiguousarray(m.coeff, dtype=np.float64)
    h = shim.shim_build(dim, m.nv, X.ctypes.data, m.ne, E.ctypes.data, B.ctypes.data,
                        None if C is None else C.ctypes.data, len(cnt), cnt.ctypes.data, flat.ctypes.data,
                        amin.ctypes.data, float(r[3]), params.get("n_min", 3), params.get("coarse_max", 512), 1,
                        params.get("nb_layers", 2))
    try:
        assert shim.shim_error(h) == b""
        J, c = o.J, o.c
        ak = _get(shim, h, "aux_key", 0, np.uint64)
        phi, psi = _get(shim, h, "phi", 0, np.int32), _get(shim, h, "psi", 0, np.int32)
        idx = {int(k): i for i, k in enumerate(ak)}
        free = {l: np.where((phi <= l) & (l < psi))[0] for l in range(J + 1)}
        A = {l: _level_matrix(shim, h, o, l, ak, dim) for l in range(c + 1, J + 1)}
        # coarsest level: the oracle's operator on the library's IDs (checked equal elsewhere)
        cid = _get(shim, h, "coarse_id", 0, np.int32)
        assert np.array_equal(ak[cid], o.level_keys(c))
        Ac = o.A(c).toarray()
        classes = {}
        for l in range(c + 1, J + 1):
            sm, cs, _ = o.smoothing_set(l)
            ids = np.array([idx[int(k)] for k in o.level_keys(l)])
            classes[l] = [ids[sm[cs[q]:cs[q + 1]]] for q in range(cs.size - 1)]
        newn = {l: (_get(shim, h, "new_id", l, np.int32), _get(shim, h, "new_p0", l, np.int32),
                    _get(shim, h, "new_p1", l, np.int32)) for l in range(c + 1, J + 1)}
        nbid = {l: _get(shim, h, "nb_id", l, np.int32) for l in range(c + 1, J + 1)}

        def gs(Al, d, cls, f, u, forward):
            for q in (cls if forward else cls[::-1]):
                u[q] += (f[q] - Al[q] @ u) / d[q]

        def vcycle(l, f):
            u = np.zeros(ak.size)
            if l == c:
                u[cid] = np.linalg.solve(Ac, f[cid])
                return u
            Al, d = A[l], A[l].diagonal()
            for _ in range(2):
                gs(Al, d, classes[l], f, u, True)
            res = f - Al @ u
            Fl, Fc = free[l], free[l - 1]
            fc = np.zeros(ak.size)
            carried = np.intersect1d(Fl, Fc)
            fc[carried] = res[carried]
            w, p0, p1 = newn[l]
            for a_, b_, c_ in zip(w, p0, p1):
                if b_ >= 0:
                    fc[b_] += 0.5 * res[a_]
                if c_ >= 0:
                    fc[c_] += 0.5 * res[a_]
            e = vcycle(l - 1, fc)
            u[carried] += e[carried]
            for a_, b_, c_ in zip(w, p0, p1):
                u[a_] += 0.5 * ((e[b_] if b_ >= 0 else 0.0) + (e[c_] if c_ >= 0 else 0.0))
            J_ = nbid[l]
            if J_.size:
                rj = np.ascontiguousarray((f - Al @ u)[J_])
                dj = np.zeros(J_.size)
                assert shim.shim_level_nbsolve(h, l, rj.ctypes.data, dj.ctypes.data) == J_.size
                u[J_] += dj
            for _ in range(2):
                gs(Al, d, classes[l], f, u, False)
            u[np.setdiff1d(np.arange(ak.size), Fl)] = 0.0
            return u

        assert np.any(psi <= J)          # some node leaves the grid before the finest level
        fJ = np.random.default_rng(4).standard_normal(o.info("nlevel", J))
        f = np.zeros(ak.size)
        f[[idx[int(k)] for k in o.level_keys(J)]] = fJ
        got = vcycle(J, f)[[idx[int(k)] for k in o.level_keys(J)]]
        want = o.vcycle(fJ)
        assert np.abs(got - want).max() <= 1e-10 * np.abs(want).max()
    finally:
        shim.shim_free(h)


def test_bf16_rounding_is_round_to_nearest_even(shim):
    # the library's FP32 -> BF16 rounding of level values against torch's
    # conversion (round to nearest, ties to even) and against the definition
    # on hand-made ties: x = (kept half) + exactly half an ulp of BF16
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(4)
    x = np.concatenate([rng.standard_normal(20000) * 10.0 ** rng.integers(-30, 30, 20000),
                        [0.0, -0.0, 1.0, -2.5, 4.0, -0.5, 1e-38, 3.0e38]]).astype(np.float32)
    # finite kept halves (exponent below all ones), either sign
    kept = rng.integers(0, 0x7F00, 64, dtype=np.uint32) | (rng.integers(0, 2, 64, dtype=np.uint32) << 15)
    ties = ((kept << 16) | np.uint32(0x8000)).astype(np.uint32)
    x = np.concatenate([x, ties.view(np.float32)])
    y = np.zeros(x.size, dtype=np.uint16)
    shim.shim_bf16(x.ctypes.data, y.ctypes.data, x.size)
    ref = torch.from_numpy(x.copy()).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    assert np.array_equal(y, ref)
    # the ties: the kept half rounds up exactly when it is odd
    kept = (ties >> 16).astype(np.uint32)
    want = np.where(kept & 1, kept + 1, kept).astype(np.uint16)
    assert np.array_equal(y[-64:], want)

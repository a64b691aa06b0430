"""The C ABI library: it builds, loads, exports every declared symbol, and
rejects bad input before touching a GPU.  No compute call is made."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1410_2153_gb300 import build as B
    B.build()
    from paper_1410_2153_gb300 import asmg
    return asmg


def _declared_functions():
    hdr = open(os.path.join(ROOT, "include", "asmg.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    return sorted(set(re.findall(r"\b((?:amg|asmg)_[a-z_]+)\s*\(", hdr)))


def test_library_exports_every_declared_symbol(lib):
    names = _declared_functions()
    assert "amg_setup" in names and "amg_solve" in names
    L = lib.lib()
    for n in names:
        assert hasattr(L, n), n
    # the exported symbols are C (unmangled)
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", lib.LIB_PATH], capture_output=True, text=True).stdout
    for n in names:
        assert re.search(rf"\bT {n}$", out, flags=re.M), n


def test_default_params(lib):
    p = lib.asmg_default_params()
    assert (p.n_min, p.nu_pre, p.nu_post, p.coarse_max_dofs, p.precision, p.max_iter, p.smoothing, p.use_graph,
            p.use_pdl) == (3, 2, 2, 512, 0, 500, 0, 1, 1)


def _mesh(gen):
    return gen.grid2d(5, 1)


def _setup_code(lib, m, **kw):
    p = lib.asmg_default_params()
    dim = kw.pop("dim", 2)
    for k, v in kw.items():
        setattr(p, k, v)
    try:
        lib.amg_setup(dim, m.nv, m.verts, m.ne, m.elems, m.bflag, m.coeff, p)
    except lib.AsmgError as e:
        return e.code
    return 0


def test_rejections_before_any_gpu_work(lib, gen):
    m = _mesh(gen)
    assert _setup_code(lib, m, dim=4) == lib.ASMG_ERR_UNSUPPORTED
    assert _setup_code(lib, m, dim=1) == lib.ASMG_ERR_UNSUPPORTED
    t = gen.grid3d(3, 1)                                         # tetrahedra take the same checks
    t.bflag = t.bflag.copy()
    t.bflag[0] = 3
    assert _setup_code(lib, t, dim=3) == lib.ASMG_ERR_BAD_MESH
    t = gen.grid3d(3, 1)
    t.coeff = np.ones(t.ne)
    t.coeff[5] = 0.0
    assert _setup_code(lib, t, dim=3) == lib.ASMG_ERR_BAD_MESH
    # Neumann vertices (flag 2) are accepted: only the parameters of the
    # near-boundary correction and of the schedule are checked here
    assert _setup_code(lib, _mesh(gen), nb_layers=-2) == lib.ASMG_ERR_INVALID_ARG
    assert _setup_code(lib, _mesh(gen), nb_layers=17) == lib.ASMG_ERR_INVALID_ARG
    assert _setup_code(lib, _mesh(gen), tile_rows=5) == lib.ASMG_ERR_INVALID_ARG
    assert _setup_code(lib, _mesh(gen), inject_timeout=2) == lib.ASMG_ERR_INVALID_ARG
    m3 = _mesh(gen)
    m3.bflag = m3.bflag.copy()
    m3.bflag[0] = 7
    assert _setup_code(lib, m3) == lib.ASMG_ERR_BAD_MESH
    m4 = _mesh(gen)
    m4.coeff = np.ones(m4.ne)
    m4.coeff[3] = -1.0
    assert _setup_code(lib, m4) == lib.ASMG_ERR_BAD_MESH
    m5 = _mesh(gen)
    m5.coeff = np.ones(m5.ne)
    m5.coeff[2] = np.nan
    assert _setup_code(lib, m5) == lib.ASMG_ERR_BAD_MESH
    assert _setup_code(lib, _mesh(gen), nu_pre=0) == lib.ASMG_ERR_INVALID_ARG
    assert _setup_code(lib, _mesh(gen), precision=5) == lib.ASMG_ERR_INVALID_ARG
    assert _setup_code(lib, _mesh(gen), max_iter=0) == lib.ASMG_ERR_INVALID_ARG
    assert "parameter" in lib.amg_last_error()


def test_null_arguments(lib):
    L = lib.lib()
    h = ctypes.c_void_p()
    assert L.amg_setup(2, 4, None, 2, None, None, None, None, None, ctypes.byref(h)) == lib.ASMG_ERR_INVALID_ARG
    assert L.amg_solve(None, None, None, 1e-8, None, None, None) == lib.ASMG_ERR_INVALID_ARG
    assert L.asmg_default_params(None) == lib.ASMG_ERR_INVALID_ARG
    L.amg_destroy(None)


def test_variant_parameters_validated(lib, gen):
    m = _mesh(gen)
    assert _setup_code(lib, m, smoother=2) == lib.ASMG_ERR_INVALID_ARG
    assert _setup_code(lib, m, additive=-1) == lib.ASMG_ERR_INVALID_ARG
    assert _setup_code(lib, m, fine_sweeps=0) == lib.ASMG_ERR_INVALID_ARG
    assert _setup_code(lib, m, fine_sweeps=9) == lib.ASMG_ERR_INVALID_ARG
    assert _setup_code(lib, m, iteration=2) == lib.ASMG_ERR_INVALID_ARG
    # BF16 level matrices: a switch of the mixed form only
    assert lib.asmg_default_params().level_bf16 == 0
    assert _setup_code(lib, m, level_bf16=2, precision=1) == lib.ASMG_ERR_INVALID_ARG
    assert _setup_code(lib, m, level_bf16=1, precision=0) == lib.ASMG_ERR_INVALID_ARG
    p = lib.asmg_default_params()
    assert (p.smoother, p.additive, p.fine_sweeps, p.iteration) == (0, 0, 1, 0)

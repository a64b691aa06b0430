"""Python binding of libasmg (include/asmg.h): argument marshalling only.

Every function of the C ABI is exposed under the same name.  Arrays may be
numpy arrays (host) or CUDA torch tensors (device); the library accepts both.
The CUDA library must have been built (``__graft_entry__.build()`` or
``python -m paper_1410_2153_gb300.build``); importing this module on a machine
where it is missing raises, and there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libasmg.so")

ASMG_OK = 0
ASMG_NOT_CONVERGED = 1
ASMG_ERR_INVALID_ARG = -1
ASMG_ERR_BAD_MESH = -2
ASMG_ERR_UNSUPPORTED = -3
ASMG_ERR_BREAKDOWN = -4
ASMG_ERR_CUDA = -5
ASMG_ERR_OOM = -6
ASMG_ERR_TIMEOUT = -7
ASMG_FP64 = 0
ASMG_MIXED = 1

INFO = dict(nfree=0, J=1, coarse=2, naux=3, nsmooth=4, ncolours=5, ntree_levels=6, nseg=7, nsplit=8, nnz_A=9,
            nnz_P=10, nrows_E=11, bytes_iter=12, nnz_level=13, ntiles=14, halo_rows=15, ntiles_up=16, launches_per_iter=100, t_setup_us=101,
            t_tree_us=102, t_aux_us=103, t_fine_us=104, t_levels_us=105,
            t_lv_assemble_us=108, t_lv_colour_us=109, t_lv_pack_us=110, t_lv_export_us=111, t_coarse_us=112,
            t_transfer_us=113, t_slots_us=114, t_sz_us=115)
EXPORT = dict(keys=0, perm=1, seg=2, split=3, aux_keys=4, fine_colour=5, smooth=6, level_rows=7, P=8, fine_A=9)


class asmg_params(ctypes.Structure):
    _fields_ = [("n_min", ctypes.c_int32), ("nu_pre", ctypes.c_int32), ("nu_post", ctypes.c_int32),
                ("coarse_max_dofs", ctypes.c_int32), ("precision", ctypes.c_int32), ("max_iter", ctypes.c_int32),
                ("smoothing", ctypes.c_int32), ("use_graph", ctypes.c_int32), ("use_pdl", ctypes.c_int32),
                ("smoother", ctypes.c_int32), ("additive", ctypes.c_int32), ("fine_sweeps", ctypes.c_int32),
                ("iteration", ctypes.c_int32), ("tile_rows", ctypes.c_int32),
                ("inject_timeout", ctypes.c_int32), ("nb_layers", ctypes.c_int32),
                ("colouring", ctypes.c_int32), ("level_bf16", ctypes.c_int32)]


class AsmgError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"asmg error {code}: {msg}")
        self.code = code


_lib = None


def lib():
    """Load libasmg.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build the CUDA library first")
        L = ctypes.CDLL(LIB_PATH)
        vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
        L.asmg_default_params.argtypes = [ctypes.POINTER(asmg_params)]
        L.amg_setup.argtypes = [i32, i64, vp, i64, vp, vp, vp, ctypes.POINTER(asmg_params), vp, ctypes.POINTER(vp)]
        L.amg_solve.argtypes = [vp, vp, vp, ctypes.c_double, ctypes.POINTER(ctypes.c_int), vp, vp]
        L.amg_mass_apply.argtypes = [vp, vp, vp, vp]
        L.amg_precond_apply.argtypes = [vp, vp, vp, vp]
        L.amg_spmv.argtypes = [vp, vp, vp, vp]
        L.amg_element_grad.argtypes = [vp, vp, vp, vp, vp]
        L.amg_update_coefficients.argtypes = [vp, vp, vp]
        L.amg_element_grad_log.argtypes = [vp, vp, vp, vp, vp]
        L.amg_set_log_coefficients.argtypes = [vp, vp, vp]
        L.amg_info.argtypes = [vp, i32, i32, ctypes.POINTER(i64)]
        L.amg_export.argtypes = [vp, i32, i32, vp, ctypes.POINTER(i64)]
        L.amg_profile.argtypes = [vp, vp, ctypes.c_double, vp, ctypes.POINTER(ctypes.c_int), vp]
        L.amg_residual_norm_noalloc.argtypes = [vp, vp, vp, vp, vp]
        L.amg_solve_multi.argtypes = [vp, i32, vp, vp, ctypes.c_double, vp, vp, vp, vp]
        L.amg_profile_levels.argtypes = [vp, vp, ctypes.c_double, vp, vp, i32, ctypes.POINTER(ctypes.c_int), vp]
        L.amg_batch_create.argtypes = [i32, vp, i32, ctypes.c_double, vp, ctypes.POINTER(vp)]
        L.amg_batch_solve.argtypes = [vp, vp, vp, vp, vp, vp]
        L.amg_batch_destroy.argtypes = [vp]
        L.amg_batch_destroy.restype = None
        L.amg_cluster_tree.argtypes = [i32, i64, vp, i64, vp, vp, vp, vp]
        L.amg_destroy.argtypes = [vp]
        L.amg_destroy.restype = None
        L.amg_last_error.restype = ctypes.c_char_p
        for name in ("asmg_default_params", "amg_setup", "amg_solve", "amg_mass_apply", "amg_precond_apply",
                     "amg_spmv", "amg_element_grad", "amg_update_coefficients", "amg_element_grad_log",
                     "amg_set_log_coefficients", "amg_info", "amg_export",
                     "amg_profile", "amg_profile_levels", "amg_residual_norm_noalloc", "amg_solve_multi", "amg_batch_create", "amg_batch_solve", "amg_cluster_tree"):
            getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


def amg_last_error() -> str:
    return lib().amg_last_error().decode()


def _check(rc: int, allow=(ASMG_OK,)) -> int:
    if rc not in allow:
        raise AsmgError(rc, amg_last_error())
    return rc


def _ptr(a):
    """Raw pointer of a numpy array or torch tensor (None passes NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags.c_contiguous
        return ctypes.c_void_p(a.ctypes.data)
    assert a.is_contiguous()
    return ctypes.c_void_p(a.data_ptr())


def _stream(stream, *arrays):
    """The stream to enqueue on: the caller's, else torch's current stream of
    the first CUDA tensor among `arrays` (so that work queued there on the
    inputs comes first), else NULL (the legacy default stream)."""
    if stream is not None:
        return stream
    for a in arrays:
        if a is not None and not isinstance(a, np.ndarray) and getattr(a, "is_cuda", False):
            import torch
            return ctypes.c_void_p(torch.cuda.current_stream(a.device).cuda_stream)
    return None


def asmg_default_params() -> asmg_params:
    p = asmg_params()
    _check(lib().asmg_default_params(ctypes.byref(p)))
    return p


def amg_setup(dim, nv, vertices, ne, elements, boundary, coeff, params: Optional[asmg_params] = None,
              stream=None) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    prm = params if params is not None else asmg_default_params()
    _check(lib().amg_setup(dim, nv, _ptr(vertices), ne, _ptr(elements), _ptr(boundary), _ptr(coeff),
                           ctypes.byref(prm), stream, ctypes.byref(h)))
    return h


def amg_solve(h, b, u, rtol: float, res_history: Optional[np.ndarray] = None, stream=None):
    it = ctypes.c_int(0)
    rc = _check(lib().amg_solve(h, _ptr(b), _ptr(u), float(rtol), ctypes.byref(it), _ptr(res_history),
                            _stream(stream, b, u)),
                allow=(ASMG_OK, ASMG_NOT_CONVERGED))
    return rc, it.value


def amg_solve_multi(h, k: int, b, u, rtol: float, res_history: Optional[np.ndarray] = None, stream=None):
    """k right-hand sides at once: b, u float64 [k * nv] (column c at c * nv);
    returns (worst status, iterations [k], statuses [k])."""
    its = np.zeros(k, dtype=np.int32)
    st = np.zeros(k, dtype=np.int32)
    rc = _check(lib().amg_solve_multi(h, k, _ptr(b), _ptr(u), float(rtol), _ptr(its), _ptr(st), _ptr(res_history),
                                      _stream(stream, b, u)), allow=(ASMG_OK, ASMG_NOT_CONVERGED))
    return rc, its, st


def amg_mass_apply(h, f, b, stream=None):
    _check(lib().amg_mass_apply(h, _ptr(f), _ptr(b), _stream(stream, f, b)))


def amg_precond_apply(h, r, z, stream=None):
    _check(lib().amg_precond_apply(h, _ptr(r), _ptr(z), _stream(stream, r, z)))


def amg_spmv(h, x, y, stream=None):
    _check(lib().amg_spmv(h, _ptr(x), _ptr(y), _stream(stream, x, y)))


def amg_element_grad(h, u, lam, g, stream=None):
    _check(lib().amg_element_grad(h, _ptr(u), _ptr(lam), _ptr(g), _stream(stream, u, lam, g)))


def amg_element_grad_log(h, u, lam, g, stream=None):
    _check(lib().amg_element_grad_log(h, _ptr(u), _ptr(lam), _ptr(g), _stream(stream, u, lam, g)))


def amg_set_log_coefficients(h, g, stream=None):
    _check(lib().amg_set_log_coefficients(h, _ptr(g), _stream(stream, g)))


def amg_update_coefficients(h, coeff, stream=None):
    _check(lib().amg_update_coefficients(h, _ptr(coeff), _stream(stream, coeff)))


def amg_info(h, what, level: int = 0) -> int:
    v = ctypes.c_int64(0)
    _check(lib().amg_info(h, INFO[what] if isinstance(what, str) else what, level, ctypes.byref(v)))
    return int(v.value)


def amg_export(h, what, level: int = 0) -> np.ndarray:
    code = EXPORT[what] if isinstance(what, str) else what
    cnt = ctypes.c_int64(0)
    _check(lib().amg_export(h, code, level, None, ctypes.byref(cnt)))
    n = cnt.value
    if code in (EXPORT["level_rows"], EXPORT["P"], EXPORT["fine_A"]):
        dt = np.dtype([("row", np.uint64), ("col", np.uint64), ("val", np.float64)])
    elif code in (EXPORT["perm"], EXPORT["fine_colour"]):
        dt = np.dtype(np.int32)
    elif code == EXPORT["seg"]:
        dt = np.dtype(np.int64)
    else:
        dt = np.dtype(np.uint64)
    out = np.empty(n, dtype=dt)
    if n:
        _check(lib().amg_export(h, code, level, out.ctypes.data_as(ctypes.c_void_p), ctypes.byref(cnt)))
    return out


PROF_CLASSES = ["fine_gs", "fine_resid", "restrict", "prolong", "aux_gs", "aux_resid", "aux_transfer", "coarse",
                "cg_spmv", "cg_vector", "aux_small", "aux_nb"]


def amg_profile(h, b, rtol: float, stream=None):
    """Per kernel class: dict(launches, ms, bytes) of one event-timed solve, and the iterations."""
    out = np.zeros(3 * len(PROF_CLASSES))
    it = ctypes.c_int(0)
    _check(lib().amg_profile(h, _ptr(b), float(rtol), _ptr(out), ctypes.byref(it), _stream(stream, b)))
    res = {c: dict(launches=int(out[3 * k]), ms=float(out[3 * k + 1]), bytes=float(out[3 * k + 2]))
           for k, c in enumerate(PROF_CLASSES)}
    return res, it.value


def amg_profile_levels(h, b, rtol: float, stream=None):
    """amg_profile plus, per auxiliary level (index l - coarsest - 1), direction and part
    (sweeps, residual, transfer): dict(launches, ms, bytes)."""
    nlev = amg_info(h, "J") - amg_info(h, "coarse")
    out = np.zeros(3 * len(PROF_CLASSES))
    lv = np.zeros(nlev * 2 * 3 * 3)
    it = ctypes.c_int(0)
    _check(lib().amg_profile_levels(h, _ptr(b), float(rtol), _ptr(out), _ptr(lv), nlev, ctypes.byref(it),
                                    _stream(stream, b)))
    res = {c: dict(launches=int(out[3 * k]), ms=float(out[3 * k + 1]), bytes=float(out[3 * k + 2]))
           for k, c in enumerate(PROF_CLASSES)}
    lv = lv.reshape(nlev, 2, 3, 3)
    levels = [{d: {part: dict(launches=int(lv[k, di, pi, 0]), ms=float(lv[k, di, pi, 1]), bytes=float(lv[k, di, pi, 2]))
                   for pi, part in enumerate(("sweeps", "residual", "transfer"))}
               for di, d in enumerate(("down", "up"))} for k in range(nlev)]
    return res, levels, it.value


def amg_residual_norm_noalloc(h, b, u, stream=None):
    """(||b - A u||, ||b||) over free dofs; b and u must be CUDA tensors.  Allocates nothing.

    Runs on `stream`, by default torch's current stream of b, after the work
    already queued there."""
    out = np.zeros(2)
    _check(lib().amg_residual_norm_noalloc(h, _ptr(b), _ptr(u), _ptr(out), _stream(stream, b, u)))
    return float(out[0]), float(out[1])


def amg_cluster_tree(mesh, stream=None):
    """(keys, perm) of the cluster tree of a 2D or 3D mesh (host arrays out)."""
    X = np.ascontiguousarray(mesh.verts, dtype=np.float64)
    E = np.ascontiguousarray(mesh.elems, dtype=np.int32)
    keys = np.empty(mesh.ne, dtype=np.uint64)
    perm = np.empty(mesh.ne, dtype=np.int32)
    _check(lib().amg_cluster_tree(mesh.dim, mesh.nv, _ptr(X), mesh.ne, _ptr(E), _ptr(keys), _ptr(perm), stream))
    return keys, perm


def amg_destroy(h):
    if h:
        lib().amg_destroy(h)


def amg_batch_create(handles, nrhs: int, rtol: float, stream=None):
    arr = (ctypes.c_void_p * len(handles))(*[h.value if isinstance(h, ctypes.c_void_p) else h for h in handles])
    out = ctypes.c_void_p()
    _check(lib().amg_batch_create(len(handles), arr, nrhs, float(rtol), stream, ctypes.byref(out)))
    return out


def amg_batch_solve(batch, bs, us, stream=None):
    """bs, us: flat lists (problem-major) of arrays; returns (worst status, iterations, statuses)."""
    n = len(bs)
    pb = (ctypes.c_void_p * n)(*[_ptr(x).value for x in bs])
    pu = (ctypes.c_void_p * n)(*[_ptr(x).value for x in us])
    its = np.zeros(n, dtype=np.int32)
    st = np.zeros(n, dtype=np.int32)
    rc = _check(lib().amg_batch_solve(batch, pb, pu, _ptr(its), _ptr(st), stream),
                allow=(ASMG_OK, ASMG_NOT_CONVERGED))
    return rc, its, st


def amg_batch_destroy(batch):
    if batch:
        lib().amg_batch_destroy(batch)


class Solver:
    """Owns one handle.  Inputs: a Mesh from ``meshgen`` (or the same fields)."""

    def __init__(self, mesh, precision: int = ASMG_FP64, stream=None, **overrides):
        p = asmg_default_params()
        p.precision = precision
        for k, v in overrides.items():
            setattr(p, k, v)
        self.params = p
        self.nv, self.ne = mesh.nv, mesh.ne
        X = np.ascontiguousarray(mesh.verts, dtype=np.float64)
        E = np.ascontiguousarray(mesh.elems, dtype=np.int32)
        B = np.ascontiguousarray(mesh.bflag, dtype=np.uint8)
        C = None if mesh.coeff is None else np.ascontiguousarray(mesh.coeff, dtype=np.float64)
        self.h = amg_setup(mesh.dim, mesh.nv, X, mesh.ne, E, B, C, p, stream)

    def close(self):
        if getattr(self, "h", None):
            amg_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def info(self, what, level: int = 0) -> int:
        return amg_info(self.h, what, level)

    def export(self, what, level: int = 0) -> np.ndarray:
        return amg_export(self.h, what, level)

    def mass_apply(self, f):
        out = np.empty(self.nv) if isinstance(f, np.ndarray) else f.new_empty(self.nv)
        amg_mass_apply(self.h, f, out)
        return out

    def solve(self, b, u0=None, rtol: float = 1e-8):
        """Returns (u, status, iterations, residual history)."""
        if isinstance(b, np.ndarray):
            u = np.zeros(self.nv) if u0 is None else np.array(u0, dtype=np.float64, copy=True)
        else:
            u = b.new_zeros(self.nv) if u0 is None else u0.clone()
        hist = np.zeros(self.params.max_iter + 1)
        rc, it = amg_solve(self.h, b, u, rtol, hist)
        return u, rc, it, hist[: it + 1]

    def precond(self, r):
        z = np.empty(self.nv) if isinstance(r, np.ndarray) else r.new_empty(self.nv)
        amg_precond_apply(self.h, r, z)
        return z

    def spmv(self, x):
        y = np.empty(self.nv) if isinstance(x, np.ndarray) else x.new_empty(self.nv)
        amg_spmv(self.h, x, y)
        return y

    def element_grad(self, u, lam):
        g = np.empty(self.ne) if isinstance(u, np.ndarray) else u.new_empty(self.ne)
        amg_element_grad(self.h, u, lam, g)
        return g

    def element_grad_log(self, u, lam):
        g = np.empty(self.ne) if isinstance(u, np.ndarray) else u.new_empty(self.ne)
        amg_element_grad_log(self.h, u, lam, g)
        return g

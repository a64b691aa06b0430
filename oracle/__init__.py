"""CPU oracle of the ASMG-preconditioned CG solve -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never loads it and
shares no code with it.  The oracle is a plain single-threaded FP64 C++
program (``asmg_oracle.cpp``) driven through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "asmg_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

# colouring = 2 (lattice parity on the auxiliary levels it 2-colours, Jones-
# Plassmann elsewhere) is the library's default too
PARAM_DEFAULTS = dict(n_min=3, nu_pre=2, nu_post=2, coarse_max=512, smoothing=0, max_iter=500,
                      colouring=2, stage=2, smoother=0, additive=0, fine_sweeps=1, iteration=0, nb_layers=2)
PARAM_ORDER = ("n_min", "nu_pre", "nu_post", "coarse_max", "smoothing", "max_iter", "colouring", "stage",
               "smoother", "additive", "fine_sweeps", "iteration", "nb_layers")


def build(force: bool = False) -> str:
    """Compile the oracle (g++ -O2 -ffp-contract=off) next to its source."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-ffp-contract=off", "-std=c++17", "-shared", "-fPIC",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        lib.orc_create.restype = ctypes.c_void_p
        lib.orc_create.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_char_p, ctypes.c_int]
        lib.orc_destroy.argtypes = [ctypes.c_void_p]
        lib.orc_info.restype = ctypes.c_int64
        lib.orc_info.argtypes = [ctypes.c_void_p, ctypes.c_char_p, ctypes.c_int]
        lib.orc_get.restype = ctypes.c_int
        lib.orc_get.argtypes = [ctypes.c_void_p, ctypes.c_char_p, ctypes.c_int, ctypes.c_void_p]
        for name in ("orc_mass_apply", "orc_precond", "orc_vcycle", "orc_elem_grad"):
            getattr(lib, name).argtypes = [ctypes.c_void_p] + [ctypes.c_void_p] * (3 if name == "orc_elem_grad" else 2)
        lib.orc_spmv.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
        lib.orc_gs_sweep.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
        lib.orc_solve.restype = ctypes.c_int
        lib.orc_solve.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double,
                                  ctypes.c_void_p, ctypes.c_void_p]
        _lib = lib
    return _lib


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


class Oracle:
    """Handle on one oracle setup (tree, closure, auxiliary hierarchy, transfer)."""

    def __init__(self, mesh, **params):
        lib = _load()
        p = dict(PARAM_DEFAULTS)
        p.update(params)
        self.params = p
        self.dim = mesh.dim
        self.nv = mesh.nv
        self.ne = mesh.ne
        self._X = np.ascontiguousarray(mesh.verts, dtype=np.float64)
        self._E = np.ascontiguousarray(mesh.elems, dtype=np.int32)
        self._B = np.ascontiguousarray(mesh.bflag, dtype=np.uint8)
        self._C = None if mesh.coeff is None else np.ascontiguousarray(mesh.coeff, dtype=np.float64)
        prm = np.array([p[k] for k in PARAM_ORDER], dtype=np.int32)
        err = ctypes.create_string_buffer(512)
        h = lib.orc_create(mesh.dim, mesh.nv, _ptr(self._X), mesh.ne, _ptr(self._E), _ptr(self._B), _ptr(self._C),
                           _ptr(prm), err, 512)
        if not h:
            raise RuntimeError(err.value.decode())
        self._h = h
        self._lib = lib

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.orc_destroy(h)
            self._h = None

    # -- information -----------------------------------------------------
    def info(self, what: str, level: int = 0) -> int:
        return int(self._lib.orc_info(self._h, what.encode(), level))

    def _get(self, what: str, level: int, shape, dtype) -> np.ndarray:
        out = np.empty(shape, dtype=dtype)
        if out.size:
            rc = self._lib.orc_get(self._h, what.encode(), level, _ptr(out))
            if rc != 0:
                raise KeyError(what)
        return out

    @property
    def nfree(self) -> int:
        return self.info("nfree")

    @property
    def J(self) -> int:
        return self.info("J")

    @property
    def c(self) -> int:
        return self.info("c")

    def keys(self):
        return self._get("keys", 0, (self.ne,), np.uint64)

    def perm(self):
        return self._get("perm", 0, (self.ne,), np.int32)

    def root(self):
        return self._get("root", 0, (4,), np.float64)

    def tree_levels(self):
        out = []
        for l in range(self.info("ntree_levels")):
            out.append(self._get("seg", l, (self.info("nseg", l), 4), np.int64))
        return out

    def boxes(self):
        """Per depth: uint64 [nbox, 2] of (packed coordinates, split)."""
        return [self._get("box", l, (self.info("nbox", l), 2), np.uint64) for l in range(self.info("nbox_levels"))]

    def level_keys(self, l: int, all_nodes: bool = False):
        if all_nodes:
            return self._get("level_allkey", l, (self.info("nall", l),), np.uint64)
        return self._get("level_key", l, (self.info("nlevel", l),), np.uint64)

    def level_tri(self, l: int):
        return self._get("level_tri", l, (self.info("ntri", l), 3), np.uint64)

    def level_alltri(self, l: int):
        """Every triangle of sigma^(l), also those outside a non-box domain."""
        return self._get("level_alltri", l, (self.info("nalltri", l), 3), np.uint64)

    def level_alltet(self, l: int):
        """Every tetrahedron of sigma^(l), also those outside a non-box domain."""
        return self._get("level_alltet", l, (self.info("nalltet", l), 4), np.uint64)

    def level_tet(self, l: int):
        return self._get("level_tet", l, (self.info("ntet", l), 4), np.uint64)

    def finest_coef(self):
        n = self.info("ntri", self.J) if self.dim == 2 else self.info("ntet", self.J)
        return self._get("finest_coef", 0, (n,), np.float64)

    def _csr(self, prefix: str, level: int, nr: int, nc: int, nnz: int):
        import scipy.sparse as sp
        ptr = self._get(prefix + "ptr", level, (nr + 1,), np.int64)
        col = self._get(prefix + "col", level, (nnz,), np.int32)
        val = self._get(prefix + "val", level, (nnz,), np.float64)
        return sp.csr_matrix((val, col, ptr), shape=(nr, nc))

    def A(self, level: int = -1):
        n = self.nfree if level < 0 else self.info("nlevel", level)
        return self._csr("A_", level, n, n, self.info("nnzA", level))

    def I(self, level: int):
        return self._csr("I_", level, self.info("nlevel", level), self.info("nlevel", level - 1), self.info("nI", level))

    def P(self, full: bool = False):
        J = self.J
        if full:
            return self._csr("Pfull_", 0, self.nfree, self.info("nall", J), self.info("nPfull"))
        return self._csr("P_", 0, self.nfree, self.info("nlevel", J), self.info("nP"))

    def smoothing_set(self, level: int = -1):
        """(nodes sorted by colour, colour class starts, colour per node)."""
        n = self.nfree if level < 0 else self.info("nlevel", level)
        ns = self.info("nsmooth", level)
        nc = self.info("ncolours", level)
        return (self._get("smooth", level, (ns,), np.int32), self._get("cstart", level, (nc + 1,), np.int32),
                self._get("colour", level, (n,), np.int32))

    def near_boundary_set(self, level: int):
        """Level-l free-node indices J_{l,j} of the near-boundary correction (Algorithm 3)."""
        return self._get("nbset", level, (self.info("nnb", level),), np.int32)

    def vertex_of_free(self):
        return self._get("vertex_of_free", 0, (self.nfree,), np.int32)

    # -- operations --------------------------------------------------------
    def mass_apply(self, f_nodal: np.ndarray) -> np.ndarray:
        f = np.ascontiguousarray(f_nodal, dtype=np.float64)
        b = np.empty(self.nfree)
        self._lib.orc_mass_apply(self._h, _ptr(f), _ptr(b))
        return b

    def spmv(self, x: np.ndarray, level: int = -1) -> np.ndarray:
        x = np.ascontiguousarray(x, dtype=np.float64)
        n = self.nfree if level < 0 else self.info("nlevel", level)
        y = np.empty(n)
        self._lib.orc_spmv(self._h, level, _ptr(x), _ptr(y))
        return y

    def precond(self, r: np.ndarray) -> np.ndarray:
        r = np.ascontiguousarray(r, dtype=np.float64)
        z = np.empty(self.nfree)
        self._lib.orc_precond(self._h, _ptr(r), _ptr(z))
        return z

    def vcycle(self, f: np.ndarray) -> np.ndarray:
        f = np.ascontiguousarray(f, dtype=np.float64)
        e = np.empty(self.info("nlevel", self.J))
        self._lib.orc_vcycle(self._h, _ptr(f), _ptr(e))
        return e

    def gs_sweep(self, f: np.ndarray, u: np.ndarray, forward: bool = True) -> np.ndarray:
        f = np.ascontiguousarray(f, dtype=np.float64)
        u = np.array(u, dtype=np.float64, copy=True)
        self._lib.orc_gs_sweep(self._h, _ptr(f), _ptr(u), 1 if forward else 0)
        return u

    def solve(self, b: np.ndarray, rtol: float = 1e-8, u0: Optional[np.ndarray] = None):
        """PCG; returns (u, status, iterations, residual history)."""
        b = np.ascontiguousarray(b, dtype=np.float64)
        u = np.zeros(self.nfree) if u0 is None else np.array(u0, dtype=np.float64, copy=True)
        it = ctypes.c_int(0)
        hist = np.zeros(self.params["max_iter"] + 1)
        st = self._lib.orc_solve(self._h, _ptr(b), _ptr(u), rtol, ctypes.byref(it), _ptr(hist))
        return u, int(st), int(it.value), hist[: it.value + 1].copy()

    def elem_grad(self, u: np.ndarray, lam: np.ndarray) -> np.ndarray:
        u = np.ascontiguousarray(u, dtype=np.float64)
        lam = np.ascontiguousarray(lam, dtype=np.float64)
        g = np.empty(self.ne)
        self._lib.orc_elem_grad(self._h, _ptr(u), _ptr(lam), _ptr(g))
        return g


def lattice_xy(keys: np.ndarray):
    """Split 64-bit 2D lattice Morton keys into (x, y) integer coordinates."""
    k = keys.astype(np.uint64)
    x = np.zeros_like(k)
    y = np.zeros_like(k)
    for j in range(32):
        x |= ((k >> np.uint64(2 * j)) & np.uint64(1)) << np.uint64(j)
        y |= ((k >> np.uint64(2 * j + 1)) & np.uint64(1)) << np.uint64(j)
    return x, y

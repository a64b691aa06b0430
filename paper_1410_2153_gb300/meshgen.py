"""Seeded synthetic meshes and right-hand sides.

This module only *generates inputs*: vertex coordinates, element connectivity,
boundary flags, per-element coefficients and nodal source values.  It holds no
step of the solver (no assembly, no tree, no multigrid), so both the CUDA path
and the CPU oracle can consume its arrays without sharing any arithmetic of the
method.

The paper's test geometry (a locally refined triangulation of the Baltic sea,
Sec. 5, Table t_asmg_D) is not available; these meshes stand in for it with the
properties the method assumes (Sec. 2.1): conforming simplicial meshes with
Dirichlet boundary vertices, optionally graded strongly towards one corner.

All randomness comes from ``numpy.random.Generator(PCG64(seed))`` in a fixed
draw order, documented per function.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

DIRICHLET = 1
FREE = 0


@dataclass
class Mesh:
    dim: int
    verts: np.ndarray          # float64 [nv, dim]
    elems: np.ndarray          # int32 [ne, dim+1], positively oriented
    bflag: np.ndarray          # uint8 [nv]: 0 free, 1 Dirichlet
    coeff: Optional[np.ndarray] = None   # float64 [ne] or None (= 1)
    meta: dict = field(default_factory=dict)

    @property
    def nv(self) -> int:
        return int(self.verts.shape[0])

    @property
    def ne(self) -> int:
        return int(self.elems.shape[0])

    @property
    def nfree(self) -> int:
        return int((self.bflag == FREE).sum())


def _orientation_2d(v: np.ndarray, e: np.ndarray) -> np.ndarray:
    p0, p1, p2 = v[e[:, 0]], v[e[:, 1]], v[e[:, 2]]
    return (p1[:, 0] - p0[:, 0]) * (p2[:, 1] - p0[:, 1]) - (p2[:, 0] - p0[:, 0]) * (p1[:, 1] - p0[:, 1])


def _orientation_3d(v: np.ndarray, e: np.ndarray) -> np.ndarray:
    p0 = v[e[:, 0]]
    a, b, c = v[e[:, 1]] - p0, v[e[:, 2]] - p0, v[e[:, 3]] - p0
    return np.einsum("ij,ij->i", a, np.cross(b, c))


def grid2d(nside: int, seed: int, jitter: float = 0.2, random_diag: bool = True,
           graded: bool = False) -> Mesh:
    """Jittered ``nside x nside`` vertex grid on [0,1]^2, two triangles per cell.

    Draw order: (1) jitter U[-jitter*h, jitter*h] for every vertex and both
    coordinates (shape [nv, 2], applied to interior vertices only), then
    (2) one Bernoulli(1/2) per cell choosing the SW-NE (0) or NW-SE (1)
    diagonal.  With ``graded`` the jittered coordinates are mapped by
    x -> x^2, y -> y^2, which refines the mesh towards x=0 and y=0 (element
    size varies about 2/h between the corner and the far side).
    Vertex (i, j) has index j*nside + i; cell (i, j) owns elements 2c, 2c+1
    with c = j*(nside-1) + i.  Boundary vertices are Dirichlet.
    """
    if nside < 2:
        raise ValueError("nside must be >= 2")
    rng = np.random.Generator(np.random.PCG64(seed))
    h = 1.0 / (nside - 1)
    t = np.arange(nside, dtype=np.float64) * h
    t[-1] = 1.0
    X, Y = np.meshgrid(t, t, indexing="xy")
    verts = np.stack([X.ravel(), Y.ravel()], axis=1)
    jit = rng.uniform(-jitter * h, jitter * h, size=(nside * nside, 2)) if jitter > 0 else np.zeros((nside * nside, 2))
    ii = np.tile(np.arange(nside), nside)
    jj = np.repeat(np.arange(nside), nside)
    interior = (ii > 0) & (ii < nside - 1) & (jj > 0) & (jj < nside - 1)
    verts[interior] += jit[interior]
    if graded:
        verts = verts * verts
    nc = nside - 1
    ci = np.tile(np.arange(nc), nc)
    cj = np.repeat(np.arange(nc), nc)
    v00 = cj * nside + ci
    v10 = v00 + 1
    v01 = v00 + nside
    v11 = v01 + 1
    if random_diag:
        diag = rng.integers(0, 2, size=nc * nc)
    else:
        diag = np.zeros(nc * nc, dtype=np.int64)
    e = np.empty((2 * nc * nc, 3), dtype=np.int64)
    sw = diag == 0
    # SW-NE diagonal: (v00, v10, v11), (v00, v11, v01)
    e[0::2][sw] = np.stack([v00, v10, v11], 1)[sw]
    e[1::2][sw] = np.stack([v00, v11, v01], 1)[sw]
    # NW-SE diagonal: (v00, v10, v01), (v10, v11, v01)
    nw = ~sw
    e[0::2][nw] = np.stack([v00, v10, v01], 1)[nw]
    e[1::2][nw] = np.stack([v10, v11, v01], 1)[nw]
    elems = e.astype(np.int32)
    bflag = np.where(interior, FREE, DIRICHLET).astype(np.uint8)
    o = _orientation_2d(verts, elems)
    assert (o > 0).all(), "generator produced a non-positively oriented triangle"
    return Mesh(2, verts, elems, bflag, None,
                dict(kind="grid2d", nside=nside, seed=seed, jitter=jitter, graded=graded))


_KUHN_PERMS = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]


def grid3d(nside: int, seed: int, jitter: float = 0.15) -> Mesh:
    """Jittered ``nside^3`` vertex grid on [0,1]^3, 6 Kuhn tetrahedra per cell.

    Each cube is split along its (0,0,0)-(1,1,1) diagonal into the tetrahedra
    (v000, v000+e_a, v000+e_a+e_b, v111) for the 6 axis permutations (a,b,c);
    the last two vertices are swapped where needed for positive orientation.
    Draw order: jitter U[-jitter*h, jitter*h], shape [nv, 3], interior only.
    Vertex (i,j,k) has index (k*nside + j)*nside + i.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    h = 1.0 / (nside - 1)
    t = np.arange(nside, dtype=np.float64) * h
    t[-1] = 1.0
    Z, Y, X = np.meshgrid(t, t, t, indexing="ij")
    verts = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    jit = rng.uniform(-jitter * h, jitter * h, size=(nside ** 3, 3)) if jitter > 0 else np.zeros((nside ** 3, 3))
    idx = np.arange(nside ** 3)
    ii, jj, kk = idx % nside, (idx // nside) % nside, idx // (nside * nside)
    interior = ((ii > 0) & (ii < nside - 1) & (jj > 0) & (jj < nside - 1)
                & (kk > 0) & (kk < nside - 1))
    verts[interior] += jit[interior]
    nc = nside - 1
    c = np.arange(nc ** 3)
    ci, cj, ck = c % nc, (c // nc) % nc, c // (nc * nc)
    base = (ck * nside + cj) * nside + ci
    step = np.array([1, nside, nside * nside])
    tets = []
    for (a, b, _c) in _KUHN_PERMS:
        v0 = base
        v1 = base + step[a]
        v2 = base + step[a] + step[b]
        v3 = base + step.sum()
        tets.append(np.stack([v0, v1, v2, v3], 1))
    e = np.stack(tets, 1).reshape(-1, 4)
    o = _orientation_3d(verts, e)
    neg = o < 0
    e[neg, 2], e[neg, 3] = e[neg, 3].copy(), e[neg, 2].copy()
    elems = e.astype(np.int32)
    assert (_orientation_3d(verts, elems) > 0).all()
    bflag = np.where(interior, FREE, DIRICHLET).astype(np.uint8)
    return Mesh(3, verts, elems, bflag, None, dict(kind="grid3d", nside=nside, seed=seed, jitter=jitter))


def subcube_coefficient(mesh: Mesh, seed: int, ncube: int = 8, values=(1.0, 1e3)) -> np.ndarray:
    """Piecewise-constant coefficient on an ``ncube^3`` partition of [0,1]^3.

    One Bernoulli(1/2) draw per subcube (shape [ncube^3], C order over
    (k, j, i)); an element takes the value of the subcube holding its
    generating cell, found from the cell index of its first vertex.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    pick = rng.integers(0, 2, size=ncube ** 3)
    nside = mesh.meta["nside"]
    nc = nside - 1
    cell = np.arange(mesh.ne) // 6
    ci, cj, ck = cell % nc, (cell // nc) % nc, cell // (nc * nc)
    per = max(1, nc // ncube)
    si, sj, sk = np.minimum(ci // per, ncube - 1), np.minimum(cj // per, ncube - 1), np.minimum(ck // per, ncube - 1)
    sc = (sk * ncube + sj) * ncube + si
    return np.where(pick[sc] == 1, values[1], values[0]).astype(np.float64)


def grf_coefficient_field(points: np.ndarray, seed: int, length: float = 0.1,
                          nfeat: int = 4096) -> np.ndarray:
    """Random-Fourier-feature sample of a squared-exponential Gaussian field.

    g(x) = sqrt(2/nfeat) * sum_m cos(w_m . x + b_m), w_m ~ N(0, I/length^2),
    b_m ~ U[0, 2 pi): unit variance, correlation exp(-|x-y|^2 / (2 length^2)).
    Draw order: w [nfeat, dim] then b [nfeat].
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    dim = points.shape[1]
    w = rng.normal(0.0, 1.0 / length, size=(nfeat, dim))
    b = rng.uniform(0.0, 2.0 * math.pi, size=nfeat)
    out = np.empty(points.shape[0])
    chunk = 1 << 15
    for s in range(0, points.shape[0], chunk):
        out[s:s + chunk] = np.cos(points[s:s + chunk] @ w.T + b).sum(1)
    return out * math.sqrt(2.0 / nfeat)


def centroids(mesh: Mesh) -> np.ndarray:
    return mesh.verts[mesh.elems].mean(axis=1)


def grid2d_domain(nside: int, seed: int, shape: str = "L", jitter: float = 0.2) -> Mesh:
    """A non-box domain cut from ``grid2d(nside, seed, jitter)``.

    shape "L": the elements whose centroid lies in (1/2, 1]^2 are removed (an
    L-shaped domain); "hole": those with centroid within 1/4 (max norm) of
    (1/2, 1/2) are removed (a square with a square hole).  Jittered vertices
    make the cut boundaries jagged.  Unused vertices are dropped; every vertex
    on a boundary edge (an edge of one element only) is Dirichlet.  The bounding
    box stays [0,1]^2.
    """
    m = grid2d(nside, seed, jitter=jitter)
    c = centroids(m)
    if shape == "L":
        drop = (c[:, 0] > 0.5) & (c[:, 1] > 0.5)
    elif shape == "hole":
        drop = (np.abs(c[:, 0] - 0.5) < 0.25) & (np.abs(c[:, 1] - 0.5) < 0.25)
    else:
        raise ValueError(shape)
    E = m.elems[~drop]
    used = np.unique(E)
    remap = -np.ones(m.nv, dtype=np.int64)
    remap[used] = np.arange(used.size)
    E = remap[E].astype(np.int32)
    V = m.verts[used]
    ed = np.sort(np.concatenate([E[:, [0, 1]], E[:, [1, 2]], E[:, [2, 0]]]), axis=1)
    uniq, cnt = np.unique(ed, axis=0, return_counts=True)
    bflag = np.zeros(V.shape[0], dtype=np.uint8)
    bflag[np.unique(uniq[cnt == 1])] = DIRICHLET
    return Mesh(2, V, E, bflag, None, dict(kind="grid2d_domain", nside=nside, seed=seed, shape=shape, jitter=jitter))


def grid3d_domain(nside: int, seed: int, shape: str = "L", jitter: float = 0.15) -> Mesh:
    """A non-box domain cut from ``grid3d(nside, seed, jitter)``.

    shape "L": the elements whose centroid lies in (1/2, 1]^2 x [0, 1] are
    removed (an L-shaped prism); "hole": those with centroid within 1/4 (max
    norm) of (1/2, 1/2, 1/2) are removed (a cube with a cubic cavity).
    Unused vertices are dropped; every vertex on a boundary face (a face of one
    element only) is Dirichlet.  The bounding box stays [0,1]^3.
    """
    m = grid3d(nside, seed, jitter=jitter)
    c = m.verts[m.elems].mean(axis=1)
    if shape == "L":
        drop = (c[:, 0] > 0.5) & (c[:, 1] > 0.5)
    elif shape == "hole":
        drop = np.all(np.abs(c - 0.5) < 0.25, axis=1)
    else:
        raise ValueError(shape)
    E = m.elems[~drop]
    used = np.unique(E)
    remap = -np.ones(m.nv, dtype=np.int64)
    remap[used] = np.arange(used.size)
    E = remap[E].astype(np.int32)
    V = m.verts[used]
    fc = np.sort(np.concatenate([E[:, [1, 2, 3]], E[:, [0, 2, 3]], E[:, [0, 1, 3]], E[:, [0, 1, 2]]]), axis=1)
    uniq, cnt = np.unique(fc, axis=0, return_counts=True)
    bflag = np.zeros(V.shape[0], dtype=np.uint8)
    bflag[np.unique(uniq[cnt == 1])] = DIRICHLET
    return Mesh(3, V, E, bflag, None, dict(kind="grid3d_domain", nside=nside, seed=seed, shape=shape, jitter=jitter))


def nodal_uniform(mesh: Mesh, seed: int, k: int = 1) -> np.ndarray:
    """Nodal source values U[-1, 1], shape [nv] (k=1) or [k, nv]; 0 on Dirichlet vertices."""
    rng = np.random.Generator(np.random.PCG64(seed))
    f = rng.uniform(-1.0, 1.0, size=(k, mesh.nv))
    f[:, mesh.bflag == DIRICHLET] = 0.0
    return f[0] if k == 1 else f


def nodal_manufactured(mesh: Mesh) -> np.ndarray:
    """Nodal values of f = 2 pi^2 sin(pi x) sin(pi y), the source of u = sin(pi x) sin(pi y)."""
    x, y = mesh.verts[:, 0], mesh.verts[:, 1]
    return 2.0 * math.pi ** 2 * np.sin(math.pi * x) * np.sin(math.pi * y)


# ----------------------------------------------------------------------------
# The five workloads (seeded).  Each returns (mesh, nodal_f) or a list of them.
# ----------------------------------------------------------------------------

def workload_small_poisson(seed: int = 1, nside: int = 65) -> tuple[Mesh, np.ndarray]:
    """65x65 jittered random-diagonal grid, f from u = sin(pi x) sin(pi y)."""
    m = grid2d(nside, seed, jitter=0.2, random_diag=True)
    return m, nodal_manufactured(m)


def workload_graded(seed: int = 1, nside: int = 2049) -> tuple[Mesh, np.ndarray]:
    """2049x2049 jittered random-diagonal grid mapped by x->x^2, y->y^2; f ~ U[-1,1]."""
    m = grid2d(nside, seed, jitter=0.2, random_diag=True, graded=True)
    return m, nodal_uniform(m, seed + 1000)


def workload_3d(seed: int = 1, nside: int = 129) -> tuple[Mesh, np.ndarray]:
    """129^3 Kuhn tetrahedra, jitter 0.15h, coefficient 1 or 1e3 on 8^3 subcubes, f = 1."""
    m = grid3d(nside, seed, jitter=0.15)
    m.coeff = subcube_coefficient(m, seed + 2000)
    f = np.ones(m.nv)
    f[m.bflag == DIRICHLET] = 0.0
    return m, f


def workload_batch_sizes(seed: int = 1, nprob: int = 256, lo: float = 1e4, hi: float = 5e5) -> np.ndarray:
    """Vertex-grid sides of the batched workload: nv ~ exp(U[ln lo, ln hi]), side = round(sqrt(nv))."""
    rng = np.random.Generator(np.random.PCG64(seed))
    nv = np.exp(rng.uniform(math.log(lo), math.log(hi), size=nprob))
    return np.maximum(np.rint(np.sqrt(nv)).astype(np.int64), 3)


def workload_inverse(seed: int = 1, nside: int = 1025) -> tuple[Mesh, np.ndarray, np.ndarray]:
    """1025^2 jittered grid, a_e = exp(g_e) with g a GRF (length 0.1) at centroids.

    Returns (mesh with coeff, g, g_obs): g_obs is the field of a second seed,
    whose solve gives the observations u_obs.
    """
    m = grid2d(nside, seed, jitter=0.2, random_diag=True)
    c = centroids(m)
    g = grf_coefficient_field(c, seed + 3000)
    g_obs = grf_coefficient_field(c, seed + 4000)
    m.coeff = np.exp(g)
    return m, g, g_obs

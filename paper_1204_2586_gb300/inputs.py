"""Seeded synthetic inputs: jittered Kuhn meshes of the unit cube, element-wise
coefficient fields and random right-hand sides.

This module generates *inputs* only. It holds none of the solver's arithmetic
(no basis functions, no assembly, no preconditioner), so the CUDA library and the
CPU oracle can both consume exactly the same arrays without sharing any code of
the method itself.

Random numbers come from one counter-based generator, SplitMix64 (Steele, Lea &
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014): output i of
stream s is mix(s + (i + 1) * 0x9E3779B97F4A7C15) with the published finaliser.

The paper's experiments (Sec. 6) run on unstructured tetrahedral meshes of the unit
cube whose generator is not stated; the jittered Kuhn meshes below stand in for them.
"""
from __future__ import annotations

import itertools

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(stream: int, idx) -> np.ndarray:
    """Output ``idx`` (array of non-negative ints) of SplitMix64 stream ``stream``."""
    i = np.asarray(idx, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(stream) + (i + np.uint64(1)) * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(stream: int, idx) -> np.ndarray:
    """53-bit uniforms in [0, 1) from SplitMix64 outputs."""
    return (splitmix64(stream, idx) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(stream: int, count: int) -> np.ndarray:
    """``count`` standard normals by Box-Muller on uniforms 2j and 2j+1 of the stream."""
    j = np.arange(count, dtype=np.uint64)
    u1 = uniform01(stream, 2 * j)
    u2 = uniform01(stream, 2 * j + np.uint64(1))
    return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * np.pi * u2)


# The six Kuhn tetrahedra of a cube: for each permutation s of the axes (in
# lexicographic order) the path c, c+e_s0, c+e_s0+e_s1, c+(1,1,1). Odd permutations
# get their last two vertices swapped so every tetrahedron is positively oriented.
_PERMS = list(itertools.permutations(range(3)))


def _perm_parity(p) -> int:
    inv = sum(1 for a in range(3) for b in range(a + 1, 3) if p[a] > p[b])
    return inv & 1


def kuhn_mesh(n: int, jitter: float = 0.2, seed: int = 0):
    """Unit cube split into n^3 cubes x 6 Kuhn tetrahedra.

    Vertex (i, j, l) has id (i*(n+1) + j)*(n+1) + l and sits at h*(i, j, l), h = 1/n.
    Every interior vertex is moved by jitter*h*(2U-1) per coordinate with U drawn from
    stream ``seed`` (uniforms 3v, 3v+1, 3v+2 for vertex v); boundary vertices stay put,
    so the domain is exactly the unit cube. Tetrahedron ids run over cubes (i, j, l)
    lexicographically (l fastest), six per cube in the permutation order above.

    Returns (xyz float64 [nv,3], tets int32 [nt,4]). Raises if a tetrahedron is not
    positively oriented after jitter.
    """
    if n < 1:
        raise ValueError("n must be >= 1")
    h = 1.0 / n
    m = n + 1
    g = np.arange(m)
    I, J, L = np.meshgrid(g, g, g, indexing="ij")
    ijk = np.stack([I.ravel(), J.ravel(), L.ravel()], axis=1)
    xyz = ijk.astype(np.float64) * h
    nv = m ** 3
    if jitter != 0.0:
        interior = np.all((ijk > 0) & (ijk < n), axis=1)
        v = np.nonzero(interior)[0].astype(np.uint64)
        d = np.stack([uniform01(seed, 3 * v + np.uint64(c)) for c in range(3)], axis=1)
        xyz[interior] += jitter * h * (2.0 * d - 1.0)

    def vid(i, j, l):
        return (i * m + j) * m + l

    ci, cj, cl = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    ci, cj, cl = ci.ravel(), cj.ravel(), cl.ravel()
    tets = np.empty((n ** 3, 6, 4), dtype=np.int64)
    for s, p in enumerate(_PERMS):
        pts = [np.zeros(3, dtype=np.int64)]
        cur = np.zeros(3, dtype=np.int64)
        for ax in p:
            cur = cur.copy()
            cur[ax] = 1
            pts.append(cur)
        ids = [vid(ci + q[0], cj + q[1], cl + q[2]) for q in pts]
        if _perm_parity(p):
            ids[2], ids[3] = ids[3], ids[2]
        for a in range(4):
            tets[:, s, a] = ids[a]
    tets = tets.reshape(-1, 4).astype(np.int32)
    assert nv == xyz.shape[0]
    vol6 = signed_volume6(xyz, tets)
    if not np.all(vol6 > 0):
        raise RuntimeError("jittered Kuhn mesh has a non-positive tetrahedron")
    return xyz, tets


def signed_volume6(xyz: np.ndarray, tets: np.ndarray) -> np.ndarray:
    """Six times the signed volume of each tetrahedron (mesh validity check only)."""
    p = xyz[tets]
    a = p[:, 1] - p[:, 0]
    b = p[:, 2] - p[:, 0]
    c = p[:, 3] - p[:, 0]
    return np.einsum("ij,ij->i", a, np.cross(b, c))


def kappa_lognormal(nt: int, seed: int) -> np.ndarray:
    """Element-wise coefficient kappa_e = exp(N(0,1)) from stream ``seed``."""
    return np.exp(normal(seed, nt))


def rhs_normal(n: int, ncols: int, seed: int) -> np.ndarray:
    """Right-hand sides with i.i.d. N(0,1) entries, row-major [n, ncols]."""
    return normal(seed, n * ncols).reshape(n, ncols)


# Named workloads. Each entry lists what the generators above need.
WORKLOADS = {
    "p2_n8": dict(k=2, n=8, jitter=0.2, mesh_seed=0, kappa_seed=None),
    "p3_n32": dict(k=3, n=32, jitter=0.2, mesh_seed=0, kappa_seed=None),
    "p4_n48_lognormal": dict(k=4, n=48, jitter=0.2, mesh_seed=0, kappa_seed=1),
    "p2_n64_batched48": dict(k=2, n=64, jitter=0.2, mesh_seed=0, kappa_seed=None,
                             rhs_seed=2, ncols=48),
    "p3_n24_adjoint": dict(k=3, n=24, jitter=0.2, mesh_seed=0, kappa_seed=1,
                           kappa_obs_seed=3, fd_pick_seed=4),
}


def workload_inputs(name: str):
    """(xyz, tets, kappa, spec) for a named workload."""
    spec = dict(WORKLOADS[name])
    xyz, tets = kuhn_mesh(spec["n"], spec["jitter"], spec["mesh_seed"])
    if spec.get("kappa_seed") is None:
        kappa = np.ones(tets.shape[0])
    else:
        kappa = kappa_lognormal(tets.shape[0], spec["kappa_seed"])
    return xyz, tets, kappa, spec

"""Seeded structured-then-scrambled simplex meshes.

Every mesh is returned as a :class:`Mesh` with

* ``x``     float64 ``[n_nodes][dim]`` node coordinates,
* ``elems`` int32   ``[n_elems][4]`` node ids per element; triangles use the
  first three columns and carry ``-1`` in the fourth.

All randomness comes from ``numpy.random.Generator(PCG64(seed))`` so a mesh
is a pure function of its arguments.  Nothing here computes a grid metric.
"""

from __future__ import annotations

import dataclasses
import itertools

import numpy as np

SEED_BASE = 2502000778

# Kuhn split of the unit cube: for each permutation (a, b, c) of the axes the
# tetrahedron  v, v+e_a, v+e_a+e_b, v+(1,1,1).  All six share the diagonal.
_KUHN_PERMS = list(itertools.permutations(range(3)))


@dataclasses.dataclass
class Mesh:
    name: str
    dim: int
    x: np.ndarray       # float64 [n_nodes, dim]
    elems: np.ndarray   # int32 [n_elems, 4]
    h: float            # nominal cell size (1 / cells per side)
    meta: dict

    @property
    def n_nodes(self) -> int:
        return int(self.x.shape[0])

    @property
    def n_elems(self) -> int:
        return int(self.elems.shape[0])


# ----------------------------------------------------------------------------
# helpers
# ----------------------------------------------------------------------------

def _orient(x: np.ndarray, el: np.ndarray, dim: int) -> np.ndarray:
    """Orientation predicate (twice / six times the signed measure).

    Used only to reject inverted elements after jittering.
    """
    if dim == 2:
        a = x[el[:, 1]] - x[el[:, 0]]
        b = x[el[:, 2]] - x[el[:, 0]]
        return a[:, 0] * b[:, 1] - a[:, 1] * b[:, 0]
    a = x[el[:, 1]] - x[el[:, 0]]
    b = x[el[:, 2]] - x[el[:, 0]]
    c = x[el[:, 3]] - x[el[:, 0]]
    return (a[:, 0] * (b[:, 1] * c[:, 2] - b[:, 2] * c[:, 1])
            - a[:, 1] * (b[:, 0] * c[:, 2] - b[:, 2] * c[:, 0])
            + a[:, 2] * (b[:, 0] * c[:, 1] - b[:, 1] * c[:, 0]))


def _jitter(rng, x0, el, dim, interior, amp, h, min_frac):
    """Uniform per-coordinate jitter of interior nodes, with validity repair.

    Every interior node of an element whose orientation relative to the
    unjittered grid falls below ``min_frac * h**dim`` is re-drawn with half
    its previous amplitude, until no such element is left.
    """
    nv = x0.shape[0]
    s0 = np.sign(_orient(x0, el, dim))
    amp_n = np.where(interior, amp * h, 0.0)
    x = x0 + rng.uniform(-1.0, 1.0, size=(nv, dim)) * amp_n[:, None]
    redraws = 0
    thr = min_frac * h ** dim
    for _ in range(60):
        bad = (s0 * _orient(x, el, dim)) < thr
        if not bad.any():
            break
        nodes = np.unique(el[bad, :dim + 1].ravel())
        nodes = nodes[interior[nodes]]
        if nodes.size == 0:
            break
        redraws += int(nodes.size)
        amp_n[nodes] *= 0.5
        x[nodes] = x0[nodes] + rng.uniform(-1.0, 1.0, size=(nodes.size, dim)) * amp_n[nodes, None]
    else:  # pragma: no cover - never reached for the amplitudes used here
        raise RuntimeError("jitter repair did not converge")
    return x, redraws


def _scramble(rng, x, el, dim, permute_nodes=True, permute_elems=True, permute_local=True):
    nv, ne = x.shape[0], el.shape[0]
    k = dim + 1
    if permute_nodes:
        p = rng.permutation(nv).astype(np.int64)
        xn = np.empty_like(x)
        xn[p] = x
        x = xn
        el = np.where(el >= 0, p[np.maximum(el, 0)], -1)
    if permute_elems:
        el = el[rng.permutation(ne)]
    if permute_local:
        perms = np.array(list(itertools.permutations(range(k))), dtype=np.int64)
        order = perms[rng.integers(0, perms.shape[0], size=ne)]
        el = el.copy()
        el[:, :k] = np.take_along_axis(el[:, :k], order, axis=1)
    return x, el


def _part1by2(v: np.ndarray) -> np.ndarray:
    v = v.astype(np.uint64) & np.uint64(0x1FFFFF)
    v = (v | (v << np.uint64(32))) & np.uint64(0x1F00000000FFFF)
    v = (v | (v << np.uint64(16))) & np.uint64(0x1F0000FF0000FF)
    v = (v | (v << np.uint64(8))) & np.uint64(0x100F00F00F00F00F)
    v = (v | (v << np.uint64(4))) & np.uint64(0x10C30C30C30C30C3)
    v = (v | (v << np.uint64(2))) & np.uint64(0x1249249249249249)
    return v


def _part1by1(v: np.ndarray) -> np.ndarray:
    v = v.astype(np.uint64) & np.uint64(0xFFFFFFFF)
    v = (v | (v << np.uint64(16))) & np.uint64(0x0000FFFF0000FFFF)
    v = (v | (v << np.uint64(8))) & np.uint64(0x00FF00FF00FF00FF)
    v = (v | (v << np.uint64(4))) & np.uint64(0x0F0F0F0F0F0F0F0F)
    v = (v | (v << np.uint64(2))) & np.uint64(0x3333333333333333)
    v = (v | (v << np.uint64(1))) & np.uint64(0x5555555555555555)
    return v


def _morton_keys(p: np.ndarray, lo: np.ndarray, hi: np.ndarray) -> np.ndarray:
    dim = p.shape[1]
    bits = 21 if dim == 3 else 31
    scale = (2 ** bits - 1) / np.maximum(hi - lo, 1e-300)
    q = np.clip(np.floor((p - lo) * scale), 0, 2 ** bits - 1).astype(np.uint64)
    if dim == 3:
        return _part1by2(q[:, 0]) | (_part1by2(q[:, 1]) << np.uint64(1)) | (_part1by2(q[:, 2]) << np.uint64(2))
    return _part1by1(q[:, 0]) | (_part1by1(q[:, 1]) << np.uint64(1))


def _morton_reorder(x, el, dim):
    """Renumber nodes by the Morton key of their coordinates and sort
    elements by the Morton key of their centroid (stable, so ties keep the
    prior random order)."""
    lo, hi = x.min(axis=0), x.max(axis=0)
    order = np.argsort(_morton_keys(x, lo, hi), kind="stable")
    rank = np.empty(order.size, dtype=np.int64)
    rank[order] = np.arange(order.size)
    x = x[order]
    k = dim + 1
    el = el.copy()
    el[:, :k] = rank[el[:, :k]]
    cen = x[el[:, 0]]
    for i in range(1, k):
        cen = cen + x[el[:, i]]
    cen *= 1.0 / k
    el = el[np.argsort(_morton_keys(cen, lo, hi), kind="stable")]
    return np.ascontiguousarray(x), el


def _finish(name, dim, x, el, h, meta):
    el = np.ascontiguousarray(el.astype(np.int32))
    if el.shape[1] == 3:
        el = np.concatenate([el, -np.ones((el.shape[0], 1), np.int32)], axis=1)
    return Mesh(name=name, dim=dim, x=np.ascontiguousarray(x, dtype=np.float64), elems=el, h=h, meta=meta)


# ----------------------------------------------------------------------------
# public generators
# ----------------------------------------------------------------------------

def tri_square(n: int, jitter: float = 0.2, seed: int = SEED_BASE + 1, permute: bool = True,
               morton: bool = False, offset: float = 0.0, min_frac: float = 0.02) -> Mesh:
    """Unit square, n x n cells, each split along its (i,j)->(i+1,j+1) diagonal."""
    rng = np.random.Generator(np.random.PCG64(seed))
    h = 1.0 / n
    i, j = np.meshgrid(np.arange(n + 1), np.arange(n + 1), indexing="ij")
    i, j = i.T.ravel(), j.T.ravel()          # node id = i + (n+1) * j
    x0 = np.stack([i * h, j * h], axis=1).astype(np.float64)
    interior = (i > 0) & (i < n) & (j > 0) & (j < n)
    ci, cj = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    ci, cj = ci.T.ravel(), cj.T.ravel()
    v00 = ci + (n + 1) * cj
    v10, v01, v11 = v00 + 1, v00 + (n + 1), v00 + (n + 2)
    el = np.concatenate([np.stack([v00, v10, v11], 1), np.stack([v00, v11, v01], 1)], 0).astype(np.int64)
    x, redraws = _jitter(rng, x0, el, 2, interior, jitter, h, min_frac) if jitter > 0 else (x0, 0)
    if permute:
        x, el = _scramble(rng, x, el, 2)
    if morton:
        x, el = _morton_reorder(x, el, 2)
    if offset:
        x = x + offset
    meta = dict(kind="tri_square", n=n, jitter=jitter, seed=seed, permute=permute, morton=morton,
                offset=offset, redraws=redraws, domain_volume=1.0)
    return _finish(f"tri{n}", 2, x, el, h, meta)


def kuhn_cube(n: int, jitter: float = 0.2, seed: int = SEED_BASE + 2, permute: bool = True,
              morton: bool = True, offset: float = 0.0, min_frac: float = 0.02) -> Mesh:
    """Unit cube, n^3 cells, each split into the 6 Kuhn tetrahedra."""
    rng = np.random.Generator(np.random.PCG64(seed))
    h = 1.0 / n
    m = n + 1
    idx = np.arange(m ** 3, dtype=np.int64)
    i, j, k = idx % m, (idx // m) % m, idx // (m * m)   # node id = i + m*(j + m*k)
    x0 = np.stack([i * h, j * h, k * h], axis=1).astype(np.float64)
    interior = (i > 0) & (i < n) & (j > 0) & (j < n) & (k > 0) & (k < n)
    c = np.arange(n ** 3, dtype=np.int64)
    ci, cj, ck = c % n, (c // n) % n, c // (n * n)
    base = ci + m * (cj + m * ck)
    step = np.array([1, m, m * m], dtype=np.int64)
    tets = []
    for a, b, _ in _KUHN_PERMS:
        tets.append(np.stack([base, base + step[a], base + step[a] + step[b], base + step.sum()], 1))
    el = np.stack(tets, 1).reshape(-1, 4)          # cell-major: the 6 tets of a cell are adjacent
    x, redraws = _jitter(rng, x0, el, 3, interior, jitter, h, min_frac) if jitter > 0 else (x0, 0)
    if permute:
        x, el = _scramble(rng, x, el, 3)
    if morton:
        x, el = _morton_reorder(x, el, 3)
    if offset:
        x = x + offset
    meta = dict(kind="kuhn_cube", n=n, jitter=jitter, seed=seed, permute=permute, morton=morton,
                offset=offset, redraws=redraws, domain_volume=1.0)
    return _finish(f"kuhn{n}", 3, x, el, h, meta)


def single_simplex(dim: int, seed: int = SEED_BASE + 11, scale: float = 1.0) -> Mesh:
    """One random non-degenerate triangle or tetrahedron (every edge is a boundary edge)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    while True:
        x = rng.uniform(-1.0, 1.0, size=(dim + 1, dim)) * scale
        el = np.arange(dim + 1, dtype=np.int64)[None, :]
        vol = abs(_orient(x, el, dim)[0])
        if vol > 0.05 * scale ** dim:
            break
    meta = dict(kind="single", seed=seed, scale=scale)
    return _finish(f"single{dim}d", dim, x, el, scale, meta)


def batched_set(n_meshes: int = 64, seed: int = SEED_BASE + 7, nmin: int = 8, nmax: int = 64,
                amp_lo: float = 0.1, amp_hi: float = 0.3) -> list:
    """Uneven Kuhn cubes: n ~ U{nmin..nmax}, jitter amplitude ~ U[amp_lo, amp_hi] h."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ns = rng.integers(nmin, nmax + 1, size=n_meshes)
    amps = rng.uniform(amp_lo, amp_hi, size=n_meshes)
    seeds = rng.integers(0, 2 ** 62, size=n_meshes)
    return [kuhn_cube(int(n), float(a), int(s), permute=True, morton=True) for n, a, s in zip(ns, amps, seeds)]


def loss_weights(n_edges: int, n_nodes: int, dim: int, seed: int = SEED_BASE + 5):
    """w ~ N(0,1)^dim per edge and c ~ N(0,1) per node for L = sum w.n + sum c V."""
    rng = np.random.Generator(np.random.PCG64(seed))
    w = rng.standard_normal((n_edges, dim))
    c = rng.standard_normal(n_nodes)
    return w, c


def fd_nodes(n_nodes: int, count: int = 1000, seed: int = SEED_BASE + 6) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.sort(rng.choice(n_nodes, size=min(count, n_nodes), replace=False)).astype(np.int64)


WORKLOADS = {
    # name: (builder, kwargs)
    "tri16": (tri_square, dict(n=16, jitter=0.2, seed=SEED_BASE + 1, permute=True, morton=False)),
    "kuhn48": (kuhn_cube, dict(n=48, jitter=0.2, seed=SEED_BASE + 2, permute=True, morton=True)),
    "kuhn160_off1e3": (kuhn_cube, dict(n=160, jitter=0.2, seed=SEED_BASE + 3, permute=True, morton=True,
                                       offset=1000.0)),
    "kuhn96": (kuhn_cube, dict(n=96, jitter=0.2, seed=SEED_BASE + 4, permute=True, morton=True)),
    # the paper's largest 3D grid size (Sec. 5: 16,974,593 nodes, 100,663,296 tets)
    "kuhn256": (kuhn_cube, dict(n=256, jitter=0.2, seed=SEED_BASE + 8, permute=True, morton=True)),
    # the paper's 2D grid size (65,536 nodes, 130,050 triangles)
    "tri255": (tri_square, dict(n=255, jitter=0.2, seed=SEED_BASE + 9, permute=True, morton=True)),
}


def workload(name: str, **override) -> Mesh:
    fn, kw = WORKLOADS[name]
    kw = dict(kw)
    kw.update(override)
    m = fn(**kw)
    m.name = name
    return m


# ----------------------------------------------------------------------------
# optional on-disk cache (a directory named by EM_MESH_CACHE, or none)
# ----------------------------------------------------------------------------
def cached_workload(name: str, cache_dir: str = None, **override) -> Mesh:
    """workload(name) with an .npz cache, so separate processes of one run
    (tests, benchmark) generate the large grids only once."""
    import hashlib
    import json
    import os
    cache_dir = cache_dir or os.environ.get("EM_MESH_CACHE")
    if not cache_dir:
        return workload(name, **override)
    fn, kw = WORKLOADS[name]
    kw = dict(kw)
    kw.update(override)
    tag = hashlib.sha1(json.dumps([name, fn.__name__, sorted(kw.items())], default=str).encode()).hexdigest()[:16]
    path = os.path.join(cache_dir, f"{name}-{tag}.npz")
    if os.path.exists(path):
        z = np.load(path, allow_pickle=False)
        meta = json.loads(str(z["meta"]))
        return Mesh(name=name, dim=int(z["dim"]), x=z["x"], elems=z["elems"], h=float(z["h"]), meta=meta)
    m = workload(name, **override)
    os.makedirs(cache_dir, exist_ok=True)
    tmp = path + f".{os.getpid()}.tmp.npz"
    np.savez(tmp, x=m.x, elems=m.elems, dim=m.dim, h=m.h, meta=json.dumps(m.meta))
    os.replace(tmp, path)
    return m


def cached_batched_set(n_meshes: int = 64, cache_dir: str = None, **kw) -> list:
    """batched_set(...) with an .npz cache (one file for the whole batch)."""
    import hashlib
    import json
    import os
    cache_dir = cache_dir or os.environ.get("EM_MESH_CACHE")
    if not cache_dir:
        return batched_set(n_meshes, **kw)
    tag = hashlib.sha1(json.dumps(["batched", n_meshes, sorted(kw.items())], default=str).encode()).hexdigest()[:16]
    path = os.path.join(cache_dir, f"batched{n_meshes}-{tag}.npz")
    if os.path.exists(path):
        z = np.load(path, allow_pickle=False)
        return [Mesh(name=f"batched{k}", dim=3, x=z[f"x{k}"], elems=z[f"e{k}"], h=float(z[f"h{k}"]), meta={})
                for k in range(n_meshes)]
    ms = batched_set(n_meshes, **kw)
    os.makedirs(cache_dir, exist_ok=True)
    arrs = {}
    for k, m in enumerate(ms):
        arrs[f"x{k}"], arrs[f"e{k}"], arrs[f"h{k}"] = m.x, m.elems, m.h
    tmp = path + f".{os.getpid()}.tmp.npz"
    np.savez(tmp, **arrs)
    os.replace(tmp, path)
    return ms


# ----------------------------------------------------------------------------
# counter-based loss weights: w(j,k) and c(v) as functions of node ids
# (SplitMix64, Steele, Lea & Flood, OOPSLA 2014), so that a checker can
# evaluate them without the edge numbering
# ----------------------------------------------------------------------------
_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def _splitmix64(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (z + np.uint64(0x9E3779B97F4A7C15)) & _M64
        z = ((z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)) & _M64
        z = ((z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)) & _M64
        return z ^ (z >> np.uint64(31))


def _u11(z: np.ndarray) -> np.ndarray:
    return (_splitmix64(z) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0) * 2.0 - 1.0


def hash_weights(edges: np.ndarray, n_nodes: int, dim: int, seed: int):
    """w[e] = U[-1,1)^dim from the key (j << 32 | k); c[v] = U[-1,1) from v."""
    s = np.uint64(seed)
    key = (edges[:, 0].astype(np.uint64) << np.uint64(32)) | edges[:, 1].astype(np.uint64)
    with np.errstate(over="ignore"):
        w = np.stack([_u11(s ^ (key * np.uint64(4) + np.uint64(c))) for c in range(dim)], axis=1)
        v = np.arange(n_nodes, dtype=np.uint64)
        c = _u11(s ^ ((v << np.uint64(2)) | np.uint64(3)) ^ np.uint64(0x5BD1E995))
    return w, c

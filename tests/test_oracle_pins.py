"""Pins for the CPU oracle: every check compares the oracle with something
other than itself -- hand-derived closed forms, identities proved from the
paper, library routines (matrix inverse, Cayley-Menger determinants), brute
force on tiny inputs, and the grid sizes the paper prints.

A plausible mistake anywhere in the oracle (a dropped boundary term, a wrong
factor or sign, a transposed operand, a wrong edge index) fails at least one
of these tests.
"""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import meshgen
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _frac(v):
    if isinstance(v, list):
        return np.array([float(Fraction(s)) for s in v])
    return float(Fraction(v))


def _edge_index(edges):
    keys = edges[:, 0].astype(np.int64) << 32 | edges[:, 1].astype(np.int64)
    return keys


def _find(edges, a, b):
    keys = _edge_index(edges)
    j, k = min(a, b), max(a, b)
    i = np.searchsorted(keys, (j << 32) | k)
    assert i < keys.size and keys[i] == ((j << 32) | k), (a, b)
    return int(i)


def _metrics(mesh):
    t = oracle.topology(mesh.dim, mesh.elems, mesh.x)
    n, v, b = oracle.direct(mesh.dim, mesh.x, mesh.elems, t)
    return t, n, v, b


# ----------------------------------------------------------------------------
# closed forms on unjittered structured grids (tests/golden/uniform_closed_forms.json)
# ----------------------------------------------------------------------------

def test_closed_forms_triangles():
    g = json.load(open(os.path.join(GOLDEN, "uniform_closed_forms.json")))["tri"]
    n_c = 6
    m = meshgen.tri_square(n_c, jitter=0.0, permute=False)
    h = m.h
    t, n, v, b = _metrics(m)
    nid = lambda i, j: i + (n_c + 1) * j  # noqa: E731
    tol = 1e-14
    for i in range(n_c):
        for j in range(1, n_c):
            np.testing.assert_allclose(n[_find(t.edges, nid(i, j), nid(i + 1, j))] / h, _frac(g["edge_interior_plus_x"]), atol=tol)
            np.testing.assert_allclose(n[_find(t.edges, nid(j, i), nid(j, i + 1))] / h, _frac(g["edge_interior_plus_y"]), atol=tol)
        np.testing.assert_allclose(n[_find(t.edges, nid(i, 0), nid(i + 1, 0))] / h, _frac(g["edge_boundary_plus_x_on_y0"]), atol=tol)
        np.testing.assert_allclose(n[_find(t.edges, nid(0, i), nid(0, i + 1))] / h, _frac(g["edge_boundary_plus_y_on_x0"]), atol=tol)
        for j in range(n_c):
            np.testing.assert_allclose(n[_find(t.edges, nid(i, j), nid(i + 1, j + 1))] / h, _frac(g["edge_interior_diagonal"]), atol=tol)
    V = v.reshape(n_c + 1, n_c + 1)  # [j][i]
    np.testing.assert_allclose(V[1:-1, 1:-1] / h ** 2, _frac(g["vol_interior"]), atol=tol)
    np.testing.assert_allclose(V[0, 1:-1] / h ** 2, _frac(g["vol_boundary_side"]), atol=tol)
    np.testing.assert_allclose([V[0, 0] / h ** 2, V[-1, -1] / h ** 2], _frac(g["vol_corner_on_diagonal"]), atol=tol)
    np.testing.assert_allclose([V[0, -1] / h ** 2, V[-1, 0] / h ** 2], _frac(g["vol_corner_off_diagonal"]), atol=tol)
    bpos = {int(nd): r for r, nd in enumerate(t.bnode)}
    np.testing.assert_allclose(b[bpos[nid(3, 0)]] / h, _frac(g["bnormal_side_y0"]), atol=tol)
    np.testing.assert_allclose(b[bpos[nid(0, 0)]] / h, _frac(g["bnormal_corner_origin"]), atol=tol)


def test_closed_forms_tetrahedra():
    g = json.load(open(os.path.join(GOLDEN, "uniform_closed_forms.json")))["tet"]
    c = 4
    q = c + 1
    m = meshgen.kuhn_cube(c, jitter=0.0, permute=False, morton=False)
    h = m.h
    t, n, v, b = _metrics(m)
    nid = lambda i, j, k: i + q * (j + q * k)  # noqa: E731
    tol = 1e-14
    s2 = h * h
    for a in range(c):
        for p in range(1, c):
            for r in range(1, c):
                np.testing.assert_allclose(n[_find(t.edges, nid(a, p, r), nid(a + 1, p, r))] / s2, _frac(g["edge_interior_plus_x"]), atol=tol)
                np.testing.assert_allclose(n[_find(t.edges, nid(p, a, r), nid(p, a + 1, r))] / s2, _frac(g["edge_interior_plus_y"]), atol=tol)
                np.testing.assert_allclose(n[_find(t.edges, nid(p, r, a), nid(p, r, a + 1))] / s2, _frac(g["edge_interior_plus_z"]), atol=tol)
    for a in range(c):
        for bb in range(c):
            for p in range(1, c):
                np.testing.assert_allclose(n[_find(t.edges, nid(a, bb, p), nid(a + 1, bb + 1, p))] / s2, _frac(g["edge_interior_diag_xy"]), atol=tol)
                np.testing.assert_allclose(n[_find(t.edges, nid(a, p, bb), nid(a + 1, p, bb + 1))] / s2, _frac(g["edge_interior_diag_xz"]), atol=tol)
                np.testing.assert_allclose(n[_find(t.edges, nid(p, a, bb), nid(p, a + 1, bb + 1))] / s2, _frac(g["edge_interior_diag_yz"]), atol=tol)
            for p in range(c):
                np.testing.assert_allclose(n[_find(t.edges, nid(a, bb, p), nid(a + 1, bb + 1, p + 1))] / s2, _frac(g["edge_interior_body_diag"]), atol=tol)
    V = v.reshape(q, q, q)  # [k][j][i]
    h3 = h ** 3
    np.testing.assert_allclose(V[1:-1, 1:-1, 1:-1] / h3, _frac(g["vol_interior"]), atol=tol)
    np.testing.assert_allclose([V[0, 0, 0] / h3, V[-1, -1, -1] / h3], _frac(g["vol_corner_on_diagonal"]), atol=tol)
    off = [V[0, 0, -1], V[0, -1, 0], V[-1, 0, 0], V[0, -1, -1], V[-1, 0, -1], V[-1, -1, 0]]
    np.testing.assert_allclose(np.array(off) / h3, _frac(g["vol_corner_off_diagonal"]), atol=tol)
    bpos = {int(nd): r for r, nd in enumerate(t.bnode)}
    for i in range(1, c):
        for j in range(1, c):
            np.testing.assert_allclose(b[bpos[nid(i, j, 0)]] / s2, _frac(g["bnormal_face_interior_z0"]), atol=tol)


# ----------------------------------------------------------------------------
# the per-element dual-face identity, computed through barycentric gradients
# (numpy.linalg.inv), at every edge of jittered, scrambled meshes
# ----------------------------------------------------------------------------

def _symmetric_form(mesh):
    """n_jk = sum_E V_E/(D+1) (grad phi_k - grad phi_j): the total dual-face
    area vector of edge jk inside E (Eqs. njk_E1_2d and njk_local_formula_3d
    with n_i^E = -D V_E grad phi_i).  Holds at interior AND boundary edges,
    so it also pins the boundary correction of the proposed algorithm."""
    d = mesh.dim
    el = mesh.elems[:, :d + 1].astype(np.int64)
    X = mesh.x[el]                               # [ne, d+1, d]
    J = X[:, 1:, :] - X[:, :1, :]                # rows x_i - x_0
    G = np.linalg.inv(J)                         # columns: grad phi_1..d
    grads = np.concatenate([-G.sum(axis=2, keepdims=True), G], axis=2).transpose(0, 2, 1)  # [ne, d+1, d]
    VE = np.abs(np.linalg.det(J)) / (2.0 if d == 2 else 6.0)   # |det J| / D!
    pairs = [(0, 1), (0, 2), (1, 2)] if d == 2 else [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]
    keys, vals = [], []
    for p, q in pairs:
        gp, gq = el[:, p], el[:, q]
        lo_is_p = gp < gq
        jj = np.where(lo_is_p, gp, gq)
        kk = np.where(lo_is_p, gq, gp)
        grad_j = np.where(lo_is_p[:, None], grads[:, p], grads[:, q])
        grad_k = np.where(lo_is_p[:, None], grads[:, q], grads[:, p])
        keys.append(jj << 32 | kk)
        vals.append(VE[:, None] / (d + 1) * (grad_k - grad_j))
    keys = np.concatenate(keys)
    vals = np.concatenate(vals)
    uk, inv = np.unique(keys, return_inverse=True)
    out = np.zeros((uk.size, d))
    np.add.at(out, inv, vals)
    return uk, out, VE


@pytest.mark.parametrize("builder", [
    lambda: meshgen.tri_square(9, jitter=0.3, seed=11),
    lambda: meshgen.kuhn_cube(5, jitter=0.3, seed=12),
    lambda: meshgen.kuhn_cube(4, jitter=0.25, seed=13, offset=1000.0),
    lambda: meshgen.single_simplex(2),
    lambda: meshgen.single_simplex(3),
])
def test_direct_matches_barycentric_form_everywhere(builder):
    m = builder()
    t, n, v, _ = _metrics(m)
    uk, ref, _ = _symmetric_form(m)
    np.testing.assert_array_equal(uk, _edge_index(t.edges))
    scale = m.h ** (m.dim - 1) if m.elems.shape[0] > 1 else 1.0
    np.testing.assert_allclose(n, ref, rtol=0, atol=1e-12 * scale)
    nt = oracle.traditional(m.dim, m.x, m.elems, t)
    np.testing.assert_allclose(nt, ref, rtol=0, atol=1e-12 * scale)


# ----------------------------------------------------------------------------
# closure, volume sum, edge-based volume, linear exactness (jittered meshes)
# ----------------------------------------------------------------------------

def _outward_sums(mesh, t, n):
    """a_j = sum_k (+/-) n_jk (Sec. 3.2.3 edge loop), done here in numpy."""
    a = np.zeros_like(mesh.x)
    np.add.at(a, t.edges[:, 0], n)
    np.add.at(a, t.edges[:, 1], -n)
    return a


@pytest.mark.parametrize("builder", [
    lambda: meshgen.tri_square(12, jitter=0.3, seed=21),
    lambda: meshgen.kuhn_cube(6, jitter=0.3, seed=22),
    lambda: meshgen.kuhn_cube(5, jitter=0.2, seed=23, offset=1000.0),
])
def test_closure_volume_and_exactness(builder):
    m = builder()
    d = m.dim
    t, n, v, b = _metrics(m)
    hs = m.h ** (d - 1)
    # closure with the returned boundary normals: zero at every node
    a = _outward_sums(m, t, n)
    a[t.bnode] += b
    assert np.abs(a).max() <= 1e-13 * hs * (1e3 if m.meta.get("offset") else 1)
    # sum of dual volumes = domain volume (1), Sec. 4.3
    assert abs(v.sum() - 1.0) <= 1e-12
    # element volumes by Cayley-Menger / Heron: V_i = sum V_E / (D+1)
    VE = _cayley_menger(m)
    ref = np.zeros(m.n_nodes)
    for i in range(d + 1):
        np.add.at(ref, m.elems[:, i], VE / (d + 1))
    np.testing.assert_allclose(v, ref, rtol=0, atol=1e-11 * m.h ** d)
    # edge-based dual volume (Sec. 4.1) equals the element-based one
    np.testing.assert_allclose(oracle.edge_volume(d, m.x, t, n), v, rtol=0, atol=1e-12 * m.h ** d)
    # linear exactness (Sec. 2): sum_k 1/2 (x_k - x_j) (x) n_jk^out = V_j I at interior nodes
    dx = m.x[t.edges[:, 1]] - m.x[t.edges[:, 0]]
    M = np.zeros((m.n_nodes, d, d))
    outer = 0.5 * dx[:, :, None] * n[:, None, :]
    np.add.at(M, t.edges[:, 0], outer)
    np.add.at(M, t.edges[:, 1], outer)        # (x_j - x_k)(x)(-n) = same term
    interior = np.ones(m.n_nodes, bool)
    interior[t.bnode] = False
    resid = M[interior] - v[interior, None, None] * np.eye(d)[None]
    assert np.abs(resid).max() <= 1e-12 * m.h ** d * (1e3 if m.meta.get("offset") else 1)


@pytest.mark.parametrize("builder", [
    lambda: meshgen.tri_square(8, jitter=0.3, seed=24),
    lambda: meshgen.kuhn_cube(4, jitter=0.3, seed=25),
    lambda: meshgen.kuhn_cube(3, jitter=0.2, seed=26, offset=1000.0),
    lambda: meshgen.single_simplex(3),
])
def test_closure_function(builder):
    """or_closure (Sec. 3.2.3: sum over a node's edges of the outward directed
    areas plus (1/D) times the area vectors of its boundary faces) against
    the same sum done here in numpy, with face vectors from numpy cross
    products, for arbitrary edge values; zero at every node for the oracle's
    own n; and a planted change of one edge value moves the sums of exactly
    that edge's two nodes, by + and - the change."""
    m = builder()
    d = m.dim
    t, n, v, b = _metrics(m)
    rng = np.random.Generator(np.random.PCG64(7))
    # arbitrary edge values: the edge loop and the boundary term, independently
    r = rng.standard_normal(n.shape)
    ref = _outward_sums(m, t, r)
    for f in t.bface:
        P = m.x[f]
        if d == 3:
            nB = 0.5 * np.cross(P[1] - P[0], P[2] - P[0])
        else:
            nB = np.array([P[0, 1] - P[1, 1], P[1, 0] - P[0, 0]])
        ref[f] += nB / d
    got = oracle.closure(d, m.x, t, r)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-13 * max(1.0, np.abs(ref).max()))
    # the oracle's own directed areas close at every node
    a = oracle.closure(d, m.x, t, n)
    hs = m.h ** (d - 1) if m.n_elems > 1 else 1.0
    assert np.abs(a).max() <= 1e-13 * hs * (1e3 if m.meta.get("offset") else 1)
    # the boundary term is the returned bnormal: closure = edge sums + bnormal
    a2 = _outward_sums(m, t, n)
    a2[t.bnode] += b
    np.testing.assert_allclose(a, a2, rtol=0, atol=1e-13 * hs * (1e3 if m.meta.get("offset") else 1))
    # planted change of one edge value
    e = int(rng.integers(t.n_edges))
    delta = np.arange(1, d + 1, dtype=np.float64) * 0.125
    n2 = n.copy()
    n2[e] += delta
    a3 = oracle.closure(d, m.x, t, n2)
    j, k = t.edges[e]
    exp = a.copy()
    exp[j] += delta
    exp[k] -= delta
    np.testing.assert_allclose(a3, exp, rtol=0, atol=1e-13)
    moved = np.flatnonzero(np.abs(a3 - a).max(axis=1) > 1e-3)
    assert sorted(moved.tolist()) == sorted([int(j), int(k)])


def _cayley_menger(m):
    d = m.dim
    P = m.x[m.elems[:, :d + 1]]
    if d == 2:
        a = np.linalg.norm(P[:, 1] - P[:, 0], axis=1)
        b = np.linalg.norm(P[:, 2] - P[:, 1], axis=1)
        c = np.linalg.norm(P[:, 0] - P[:, 2], axis=1)
        s = 0.5 * (a + b + c)
        return np.sqrt(np.maximum(s * (s - a) * (s - b) * (s - c), 0))
    ne = P.shape[0]
    CM = np.ones((ne, 5, 5))
    CM[:, 0, 0] = 0
    for i in range(4):
        CM[:, i + 1, i + 1] = 0
        for j in range(4):
            if i != j:
                CM[:, i + 1, j + 1] = ((P[:, i] - P[:, j]) ** 2).sum(axis=1)
    return np.sqrt(np.linalg.det(CM) / 288.0)


def test_single_element_brute_force():
    """One element: every edge is a boundary edge, every node a boundary node.
    The dual volume of each node is exactly V_E/(D+1) (Sec. 4.2) and the
    closure holds with (1/D) n_B at every node (Sec. 3.2.3)."""
    for d in (2, 3):
        for seed in range(5):
            m = meshgen.single_simplex(d, seed=100 + seed)
            t, n, v, b = _metrics(m)
            assert t.n_edges == (3 if d == 2 else 6)
            assert t.bface.shape[0] == d + 1 and t.bnode.size == d + 1
            VE = _cayley_menger(m)[0]
            np.testing.assert_allclose(v, VE / (d + 1), rtol=1e-13)
            a = _outward_sums(m, t, n)
            a[t.bnode] += b
            assert np.abs(a).max() < 1e-14
            # each boundary face's n_B points away from the opposite node and has
            # the face's measure
            for B in range(t.bface.shape[0]):
                f = t.bface[B]
                opp = [i for i in range(d + 1) if i not in f][0]
                P = m.x[f]
                if d == 3:
                    nB = 0.5 * np.cross(P[1] - P[0], P[2] - P[0])
                else:
                    nB = np.array([P[0, 1] - P[1, 1], P[1, 0] - P[0, 0]])
                assert np.dot(nB, P[0] - m.x[opp]) > 0


# ----------------------------------------------------------------------------
# edges and boundary faces by brute force
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("builder", [
    lambda: meshgen.tri_square(5, jitter=0.2, seed=31),
    lambda: meshgen.kuhn_cube(3, jitter=0.2, seed=32),
    lambda: meshgen.single_simplex(3),
])
def test_topology_brute_force(builder):
    m = builder()
    d = m.dim
    t = oracle.topology(d, m.elems, m.x)
    pairs = [(0, 1), (0, 2), (1, 2)] if d == 2 else [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]
    es = sorted({tuple(sorted((int(e[p]), int(e[q])))) for e in m.elems for p, q in pairs})
    assert [tuple(r) for r in t.edges.tolist()] == es
    for E in range(m.n_elems):
        for l, (p, q) in enumerate(pairs):
            assert tuple(t.edges[t.elem2edge[E, l]]) == tuple(sorted((int(m.elems[E, p]), int(m.elems[E, q]))))
    count = {}
    for E in range(m.n_elems):
        for o in range(d + 1):
            f = tuple(sorted(int(m.elems[E, i]) for i in range(d + 1) if i != o))
            count.setdefault(f, []).append((E, o))
    bnd = sorted(f for f, owners in count.items() if len(owners) == 1)
    assert [tuple(sorted(r)) for r in t.bface.tolist()] == bnd
    for B, f in enumerate(bnd):
        E, o = count[f][0]
        assert t.bowner[B] == E * 4 + o
        cen = m.x[m.elems[E, :d + 1]].mean(axis=0)
        P = m.x[t.bface[B]]
        nB = 0.5 * np.cross(P[1] - P[0], P[2] - P[0]) if d == 3 else np.array([P[0, 1] - P[1, 1], P[1, 0] - P[0, 0]])
        assert np.dot(nB, P.mean(axis=0) - cen) > 0
        if d == 3:
            assert t.bface[B, 0] == min(f)
    assert t.bnode.tolist() == sorted({v for f in bnd for v in f})


def test_structured_counts_and_paper_grid_sizes():
    g = json.load(open(os.path.join(GOLDEN, "paper_grid_counts.json")))
    # count formulas (combinatorics of the two splits) checked on small grids
    for c in (1, 2, 5):
        m = meshgen.kuhn_cube(c, jitter=0.0)
        t = oracle.topology(3, m.elems, m.x)
        assert m.n_nodes == (c + 1) ** 3 and m.n_elems == 6 * c ** 3
        assert t.n_edges == 3 * c * (c + 1) ** 2 + 3 * c * c * (c + 1) + c ** 3
        assert t.bface.shape[0] == 12 * c * c
        assert t.bnode.size == (c + 1) ** 3 - max(c - 1, 0) ** 3
        m2 = meshgen.tri_square(c, jitter=0.0)
        t2 = oracle.topology(2, m2.elems, m2.x)
        assert m2.n_nodes == (c + 1) ** 2 and m2.n_elems == 2 * c * c
        assert t2.n_edges == 3 * c * c + 2 * c and t2.bface.shape[0] == 4 * c
    # the same formulas at the paper's grid sizes (Sec. 5)
    n2, n3 = g["tri_cells_per_side"], g["tet_cells_per_side"]
    assert (n2 + 1) ** 2 == g["tri_nodes"] and 2 * n2 * n2 == g["tri_elems"]
    assert (n3 + 1) ** 3 == g["tet_nodes"] and 6 * n3 ** 3 == g["tet_elems"]


def test_workload_sizes():
    # the 48^3 workload: counts from the formulas above
    m = meshgen.workload("kuhn48")
    t = oracle.topology(3, m.elems, m.x)
    assert (m.n_nodes, m.n_elems, t.n_edges, t.bface.shape[0], t.bnode.size) == (117649, 663552, 795024, 27648, 13826)
    m = meshgen.workload("tri16")
    t = oracle.topology(2, m.elems, m.x)
    assert (m.n_nodes, m.n_elems, t.n_edges) == (289, 512, 800)


# ----------------------------------------------------------------------------
# adjoint: analytic gradient vs central differences (zero truncation error,
# because L is affine in every single coordinate)
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("builder", [
    lambda: meshgen.tri_square(6, jitter=0.3, seed=41),
    lambda: meshgen.kuhn_cube(3, jitter=0.3, seed=42),
    lambda: meshgen.single_simplex(3),
    lambda: meshgen.single_simplex(2),
])
def test_adjoint_vs_central_differences(builder):
    m = builder()
    d = m.dim
    t = oracle.topology(d, m.elems, m.x)
    w, c = meshgen.generate.loss_weights(t.n_edges, m.n_nodes, d, seed=7)
    g = oracle.adjoint(d, m.x, m.elems, t, w, c)
    # the loss itself: L = sum w.n + sum c V from the forward outputs
    n, v, _ = oracle.direct(d, m.x, m.elems, t)
    L = oracle.loss(d, m.x, m.elems, t, w, c)
    assert abs(L - (np.sum(w * n) + np.sum(c * v))) <= 1e-13 * (np.abs(w * n).sum() + np.abs(c * v).sum())
    # full-loss central differences at every node and coordinate
    delta = 1e-6 * m.h
    gfd = np.zeros_like(g)
    for i in range(m.n_nodes):
        for q in range(d):
            xp = m.x.copy(); xp[i, q] += delta
            xm = m.x.copy(); xm[i, q] -= delta
            gfd[i, q] = (oracle.loss(d, xp, m.elems, t, w, c) - oracle.loss(d, xm, m.elems, t, w, c)) / (2 * delta)
    assert np.abs(g - gfd).max() <= 1e-7 * np.abs(g).max()
    # patch-local differences agree as well
    gp = oracle.fd_gradient(d, m.x, m.elems, t, w, c, np.arange(m.n_nodes), delta)
    assert np.abs(g - gp).max() <= 1e-7 * np.abs(g).max()


def test_adjoint_patch_fd_medium():
    m = meshgen.kuhn_cube(10, jitter=0.2, seed=43)
    t = oracle.topology(3, m.elems, m.x)
    w, c = meshgen.generate.loss_weights(t.n_edges, m.n_nodes, 3, seed=44)
    g = oracle.adjoint(3, m.x, m.elems, t, w, c)
    nodes = meshgen.generate.fd_nodes(m.n_nodes, 200, seed=45)
    gp = oracle.fd_gradient(3, m.x, m.elems, t, w, c, nodes, 1e-6 * m.h)
    assert np.abs(g[nodes] - gp).max() <= 1e-7 * np.abs(g).max()


# ----------------------------------------------------------------------------
# the sampled evaluation used at full grid sizes equals the full evaluation
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("builder", [
    lambda: meshgen.kuhn_cube(5, jitter=0.3, seed=61),
    lambda: meshgen.tri_square(7, jitter=0.3, seed=62),
    lambda: meshgen.kuhn_cube(4, jitter=0.2, seed=63, offset=1000.0),
])
def test_sampled_oracle_equals_full(builder):
    m = builder()
    t = oracle.topology(m.dim, m.elems, m.x)
    n, v, b = oracle.direct(m.dim, m.x, m.elems, t)
    w, c = meshgen.generate.hash_weights(t.edges, m.n_nodes, m.dim, 2502000778)
    g = oracle.adjoint(m.dim, m.x, m.elems, t, w, c)
    es = np.arange(0, t.n_edges, 2)
    sn, sv, sb, sg = oracle.sample(m.dim, m.x, m.elems, t.edges[es, 0], t.edges[es, 1], np.arange(m.n_nodes),
                                   2502000778)
    full_b = np.zeros((m.n_nodes, m.dim))
    full_b[t.bnode] = b
    assert np.abs(sn - n[es]).max() <= 1e-15 * m.h ** (m.dim - 1)
    assert np.abs(sv - v).max() <= 1e-15 * m.h ** m.dim
    assert np.abs(sb - full_b).max() <= 1e-15 * m.h ** (m.dim - 1)
    assert np.abs(sg - g).max() <= 1e-14 * np.abs(g).max()


# ----------------------------------------------------------------------------
# edge-loop residual (Sec. 2): what the metrics are for
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("builder", [
    lambda: meshgen.tri_square(10, jitter=0.3, seed=51),
    lambda: meshgen.kuhn_cube(5, jitter=0.3, seed=52),
    lambda: meshgen.kuhn_cube(4, jitter=0.2, seed=53, offset=1000.0),
])
def test_edge_residual_linear_exactness(builder):
    """For a linear flux F = A x + f0 the central-flux edge loop reproduces
    V_j div F = V_j tr(A) at every interior node (a consequence of closure and
    of sum_k 1/2 (x_k - x_j) (x) n_jk = V_j I, not of the residual's own code);
    a constant flux gives zero there; and the edge fluxes cancel in the total,
    leaving sum_b F_b . bnormal_b."""
    m = builder()
    d = m.dim
    t, n, v, b = _metrics(m)
    rng = np.random.Generator(np.random.PCG64(77))
    A = rng.standard_normal((d, d))
    f0 = rng.standard_normal(d)
    xr = m.x - m.x.mean(axis=0)                  # keep F of order one on the offset grid
    F = xr @ A.T + f0
    r = oracle.edge_residual(d, t, n, F, b)
    inner = np.ones(m.n_nodes, bool)
    inner[t.bnode] = False
    scale = np.abs(F).max() * m.h ** (d - 1)
    assert np.abs(r[inner] - v[inner] * np.trace(A)).max() <= 1e-12 * scale
    r0 = oracle.edge_residual(d, t, n, np.tile(f0, (m.n_nodes, 1)), b)
    assert np.abs(r0[inner]).max() <= 1e-12 * np.abs(f0).max() * m.h ** (d - 1)
    total = float(np.sum(F[t.bnode] * b))
    assert abs(r.sum() - total) <= 1e-11 * scale * m.n_nodes


# ----------------------------------------------------------------------------
# adjoint with boundary-normal weights: L += sum_b bw_b . bnormal_b
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("builder", [
    lambda: meshgen.tri_square(5, jitter=0.3, seed=61),
    lambda: meshgen.kuhn_cube(3, jitter=0.3, seed=62),
    lambda: meshgen.single_simplex(3),
])
def test_adjoint_with_boundary_weights(builder):
    """The boundary-weight part of L equals sum_b bw_b . bnormal_b with the
    forward's own boundary normals (a separate loop), and the analytic
    gradient matches full-loss central differences."""
    m = builder()
    d = m.dim
    t = oracle.topology(d, m.elems, m.x)
    w, c = meshgen.generate.loss_weights(t.n_edges, m.n_nodes, d, seed=8)
    rng = np.random.Generator(np.random.PCG64(63))
    bw = rng.standard_normal((len(t.bnode), d))
    n, v, b = oracle.direct(d, m.x, m.elems, t)
    L0 = oracle.loss(d, m.x, m.elems, t, w, c)
    L1 = oracle.loss(d, m.x, m.elems, t, w, c, bw)
    assert abs((L1 - L0) - np.sum(bw * b)) <= 1e-13 * np.abs(bw * b).sum()
    g = oracle.adjoint(d, m.x, m.elems, t, w, c, bw)
    g0 = oracle.adjoint(d, m.x, m.elems, t, w, c)
    assert np.abs(g - g0).max() > 0                    # the boundary weights do move the gradient
    delta = 1e-6 * (m.h if m.n_elems > 1 else 1.0)
    gfd = np.zeros_like(g)
    for i in range(m.n_nodes):
        for q in range(d):
            xp = m.x.copy(); xp[i, q] += delta
            xm = m.x.copy(); xm[i, q] -= delta
            gfd[i, q] = (oracle.loss(d, xp, m.elems, t, w, c, bw) - oracle.loss(d, xm, m.elems, t, w, c, bw)) / (2 * delta)
    assert np.abs(g - gfd).max() <= 1e-7 * np.abs(g).max()
    gp = oracle.fd_gradient(d, m.x, m.elems, t, w, c, np.arange(m.n_nodes), delta, bw)
    assert np.abs(g - gp).max() <= 1e-7 * np.abs(g).max()

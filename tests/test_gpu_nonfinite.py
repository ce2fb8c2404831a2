"""Non-finite inputs on the tiled scatter and the atomic path.

A NaN or an infinity in a coordinate, an edge weight w, a node weight c or a
boundary-normal weight makes the tiled scatter write NaN to every component
of every output whose elements or boundary faces read it (the dependency
set, computed here from the connectivity alone), and leaves every other
output finite and within the FP64 contract of the oracle's value (the
FP32-based MIXED form at its own accuracy).  Plain FP64 arithmetic, as in
the oracle and the atomic path, can leave single components finite (a cross
product component that does not read the bad coordinate), so the atomic
path is compared per node."""
import numpy as np
import pytest

import meshgen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"

MESHES = {
    "tri12": lambda: meshgen.tri_square(12, jitter=0.25, seed=611),
    "kuhn6": lambda: meshgen.kuhn_cube(6, jitter=0.2, seed=612),
    "kuhn5_off": lambda: meshgen.kuhn_cube(5, jitter=0.2, seed=613, offset=1000.0),
}


def _plant(m, t, seed):
    """Clean inputs plus copies with one NaN coordinate (an interior node),
    one infinite coordinate (a boundary node), one NaN edge weight and one
    infinite node weight, at seeded positions."""
    rng = np.random.Generator(np.random.PCG64(seed))
    w, c = meshgen.generate.loss_weights(t.n_edges, m.n_nodes, m.dim, seed=seed + 1)
    bw = rng.standard_normal((t.bnode.size, m.dim))
    interior = np.setdiff1d(np.arange(m.n_nodes), t.bnode)
    x = m.x.copy()
    x[int(rng.choice(interior)), int(rng.integers(m.dim))] = np.nan
    x[int(rng.choice(t.bnode)), 0] = np.inf
    w2, c2, bw2 = w.copy(), c.copy(), bw.copy()
    w2[int(rng.integers(t.n_edges)), int(rng.integers(m.dim))] = np.nan
    c2[int(rng.integers(m.n_nodes))] = -np.inf
    bw2[int(rng.integers(t.bnode.size)), 0] = np.nan
    return x, w2, c2, bw2


def _structural(m, t, x, w, c, bw=None):
    """Targets that depend on a non-finite input, from the connectivity alone:
    an element with a non-finite coordinate reaches every edge and node it
    touches; its gradient terms also take the w of its edges and the c of its
    nodes; a boundary face reaches its edges and its nodes' boundary normals
    through its coordinates, and the gradient of its nodes through those, the
    w of its edges and the boundary-normal weights of its nodes.  Returns
    boolean masks over edges, nodes (V), boundary nodes and nodes (grad)."""
    d = m.dim
    el = m.elems[:, :d + 1]
    bad_x = ~np.isfinite(x).all(axis=1)
    bad_w = ~np.isfinite(w).all(axis=1)
    bad_c = ~np.isfinite(c) if c is not None else np.zeros(m.n_nodes, bool)
    ex = bad_x[el].any(axis=1)
    ea = ex | bad_w[t.elem2edge].any(axis=1) | bad_c[el].any(axis=1)
    me = np.zeros(t.n_edges, bool)
    me[t.elem2edge[ex].ravel()] = True
    mv = np.zeros(m.n_nodes, bool)
    mv[el[ex].ravel()] = True
    mg = np.zeros(m.n_nodes, bool)
    mg[el[ea].ravel()] = True
    bf = t.bface
    fx = bad_x[bf].any(axis=1)
    # the edges of a boundary face, as edge ids
    key = {(int(a), int(b)): k for k, (a, b) in enumerate(t.edges)}
    fe = np.array([[key[tuple(sorted((int(f[i]), int(f[j]))))] for i in range(d) for j in range(i + 1, d)]
                   for f in bf])
    fa = fx | bad_w[fe].any(axis=1)
    if bw is not None:
        bwn = np.zeros(m.n_nodes, bool)
        bwn[t.bnode] = ~np.isfinite(bw).all(axis=1)
        fa |= bwn[bf].any(axis=1)
    bnode_of = np.full(m.n_nodes, -1)
    bnode_of[t.bnode] = np.arange(t.bnode.size)
    mb = np.zeros(t.bnode.size, bool)
    mb[bnode_of[bf[fx].ravel()]] = True
    mg[bf[fa].ravel()] = True
    return me, mv, mb, mg


def _check(got, ref, mask, tol):
    """Non-finite exactly on the masked targets (every component), finite
    and within tol of the oracle elsewhere."""
    got = np.asarray(got)
    bad = ~np.isfinite(got)
    want = np.broadcast_to(mask.reshape(mask.shape + (1,) * (got.ndim - 1)), got.shape)
    assert mask.any()
    assert np.array_equal(bad, want), (np.flatnonzero(bad != want)[:10], bad.sum(), want.sum())
    ok = ~want
    assert np.isfinite(ref[ok]).all()
    assert np.abs(got[ok] - ref[ok]).max() <= tol


@pytest.mark.parametrize("prec", ["dw", "mixed", "fp64"])
@pytest.mark.parametrize("name", list(MESHES))
def test_tiled_nonfinite(name, prec):
    from paper_2502_00778_gb300 import api
    m = MESHES[name]()
    d = m.dim
    t = oracle.topology(d, m.elems, m.x)
    xb, w, c, bw = _plant(m, t, 620 + d)
    topo = api.edge_build(torch.from_numpy(m.elems).to(DEV), torch.from_numpy(m.x).to(DEV))
    api.plan_build(topo, 64)
    xt = torch.from_numpy(xb).to(DEV)
    n, v, b, g = api.edge_metrics_fused(topo, xt, torch.from_numpy(w).to(DEV), torch.from_numpy(c).to(DEV), prec,
                                        path="tiled", bw=torch.from_numpy(bw).to(DEV))
    with np.errstate(invalid="ignore", over="ignore"):
        rn, rv, rb = oracle.direct(d, xb, m.elems, t)
        rg = oracle.adjoint(d, xb, m.elems, t, w, c, bw)
    me, mv, mb, mg = _structural(m, t, xb, w, c, bw)
    h = m.h
    s = 1e-12 if prec != "mixed" else 2e-6
    sg = 1e-12 if prec != "mixed" else 1e-5
    _check(n.cpu().numpy(), rn, me, s * h ** (d - 1))
    _check(v.cpu().numpy(), rv, mv, s * h ** d)
    _check(b.cpu().numpy(), rb, mb, s * h ** (d - 1))
    _check(g.cpu().numpy(), rg, mg, sg * np.abs(rg[~mg]).max())
    # the separate forward pass of the same path
    n2, v2, b2 = api.edge_metrics(topo, xt, prec, "tiled")
    assert torch.equal(torch.isfinite(n2), torch.isfinite(n)) and torch.equal(torch.isfinite(v2), torch.isfinite(v))


def test_autograd_nan_upstream_gradient():
    """A NaN in the upstream gradient of n reaches the coordinate gradient of
    exactly the nodes whose elements contain that edge, on the tiled and the
    atomic path alike."""
    from paper_2502_00778_gb300 import api
    m = MESHES["kuhn6"]()
    t = oracle.topology(3, m.elems, m.x)
    topo = api.edge_build(torch.from_numpy(m.elems).to(DEV), torch.from_numpy(m.x).to(DEV))
    api.plan_build(topo, 64)
    w, c = meshgen.generate.loss_weights(t.n_edges, m.n_nodes, 3, seed=631)
    e = 17
    w[e, 1] = np.nan
    with np.errstate(invalid="ignore"):
        rg = oracle.adjoint(3, m.x, m.elems, t, w, c)
    mg = _structural(m, t, m.x, w, c)[3]
    assert np.array_equal(~np.isfinite(rg).all(axis=1), mg)
    for path, prec in (("tiled", "dw"), ("atomic", "fp64")):
        x = torch.from_numpy(m.x).to(DEV).requires_grad_(True)
        n, v, b = api.EdgeMetrics.apply(x, topo, prec, path)
        gx, = torch.autograd.grad((n, v), (x,), (torch.from_numpy(w).to(DEV), torch.from_numpy(c).to(DEV)))
        gx = gx.cpu().numpy()
        if path == "tiled":
            _check(gx, rg, mg, 1e-12 * np.abs(rg[~mg]).max())
        else:
            assert np.array_equal(~np.isfinite(gx).all(axis=1), mg)
            assert np.abs(gx[~mg] - rg[~mg]).max() <= 1e-12 * np.abs(rg[~mg]).max()

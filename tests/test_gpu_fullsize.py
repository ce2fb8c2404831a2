"""Full-size checks in the benchmark's configuration.

160^3 x 6 tets, offset 1e3 (the benchmark workload), in the benchmark's
launch configuration (fused tiled scatter, one launch per step, at the tile
sizes the autotuner picks there: 256 nodes for DW and FP64, which run
512-thread CTAs with the L2 prefetch of the next tile, 128 for MIXED; the
ordered gather path for comparison): edge_build is checked through properties that characterise
the sorted unique edge list exactly; the metrics and the adjoint are checked
at 2000 sampled edges and nodes, each computed by the oracle alone from the
elements around it.  96^3 x 6 (the adjoint workload): the full gradient
against the oracle's analytic gradient and central differences on 1000 nodes.
"""
import os

import numpy as np
import pytest

import meshgen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"
SEED = 2502000778


def _mesh(name):
    cache = os.environ.get("EM_MESH_CACHE") or os.path.join(os.path.dirname(os.path.dirname(__file__)), "_build",
                                                          "meshcache")
    return meshgen.generate.cached_workload(name, cache_dir=cache)


@pytest.fixture(scope="module")
def big():
    from paper_2502_00778_gb300 import api
    m = _mesh("kuhn160_off1e3")
    x = torch.from_numpy(m.x).to(DEV)
    el = torch.from_numpy(m.elems).to(DEV)
    topo = api.edge_build(el, x)
    api.plan_build(topo, 256)
    return m, x, topo


# tile_nodes per (form, path) as the benchmark's autotuner picks them
TILE = {("dw", "tiled"): 256, ("fp64", "tiled"): 256, ("mixed", "tiled"): 128, ("dw", "gather"): 128}


def test_edge_build_properties_160(big):
    m, x, topo = big
    n = 160
    e = topo.edges.cpu().numpy().astype(np.int64)
    assert e.shape[0] == 3 * n * (n + 1) ** 2 + 3 * n * n * (n + 1) + n ** 3
    assert np.all(e[:, 0] < e[:, 1])
    key = e[:, 0] * m.n_nodes + e[:, 1]
    assert np.all(np.diff(key) > 0)                      # sorted, unique
    e2e = topo.elem2edge.cpu().numpy()
    pairs = [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]
    used = np.zeros(e.shape[0], bool)
    for l, (p, q) in enumerate(pairs):
        a, b = m.elems[:, p].astype(np.int64), m.elems[:, q].astype(np.int64)
        lo, hi = np.minimum(a, b), np.maximum(a, b)
        assert np.array_equal(e[e2e[:, l], 0], lo) and np.array_equal(e[e2e[:, l], 1], hi)
        used[e2e[:, l]] = True
    assert used.all()                                    # exactly the element edges
    assert topo.n_bfaces == 12 * n * n
    assert topo.n_bnodes == (n + 1) ** 3 - (n - 1) ** 3


@pytest.mark.parametrize("prec,path", [("dw", "tiled"), ("fp64", "tiled"), ("mixed", "tiled"), ("dw", "gather")])
def test_sampled_parity_160(big, prec, path):
    from paper_2502_00778_gb300 import api
    m, x, topo = big
    e = topo.edges.cpu().numpy()
    rng = np.random.Generator(np.random.PCG64(SEED + 31))
    es = np.sort(rng.choice(e.shape[0], 2000, replace=False))
    bn = topo.bnode.cpu().numpy()
    ns = np.unique(np.concatenate([rng.choice(m.n_nodes, 1500, replace=False), rng.choice(bn, 500, replace=False)]))
    w, c = meshgen.generate.hash_weights(e, m.n_nodes, 3, SEED)
    wt, ct = torch.from_numpy(w).to(DEV), torch.from_numpy(c).to(DEV)
    api.plan_build(topo, TILE[(prec, path)])
    n, v, b, g = api.edge_metrics_fused(topo, x, wt, ct, prec, path=path)
    rn, rv, rb, rg = oracle.sample(3, m.x, m.elems, e[es, 0], e[es, 1], ns, SEED)
    h = m.h
    # FP64 contract; the FP32 element-math form at its stated accuracy
    tn, tv, tg = (1e-12, 1e-12, 1e-12) if prec != "mixed" else (2e-6, 2e-6, 1e-5)
    assert np.abs(n.cpu().numpy()[es] - rn).max() <= tn * h * h
    assert np.abs(v.cpu().numpy()[ns] - rv).max() <= tv * h ** 3
    bfull = np.zeros((m.n_nodes, 3))
    bfull[bn] = b.cpu().numpy()
    assert np.abs(bfull[ns] - rb).max() <= tn * h * h
    gg = g.cpu().numpy()
    assert np.abs(gg[ns] - rg).max() <= tg * np.abs(gg).max()
    if prec == "mixed":
        return
    # properties at every node: closure and the volume sum
    a = np.zeros((m.n_nodes, 3))
    nn = n.cpu().numpy()
    np.add.at(a, e[:, 0], nn)
    np.add.at(a, e[:, 1], -nn)
    a[bn] += bfull[bn]
    assert np.abs(a).max() <= 1e-12 * h * h
    assert abs(v.cpu().numpy().sum() - 1.0) <= 1e-11


def test_atomic_fp64_sampled_160(big):
    from paper_2502_00778_gb300 import api
    m, x, topo = big
    e = topo.edges.cpu().numpy()
    rng = np.random.Generator(np.random.PCG64(SEED + 32))
    es = np.sort(rng.choice(e.shape[0], 500, replace=False))
    n, v, b = api.edge_metrics(topo, x, "fp64", "atomic")
    rn, rv, rb, rg = oracle.sample(3, m.x, m.elems, e[es, 0], e[es, 1], np.array([0], np.int32), SEED)
    assert np.abs(n.cpu().numpy()[es] - rn).max() <= 1e-12 * m.h ** 2


def test_adjoint_96_fd():
    """Adjoint workload: full oracle gradient, and central differences with
    step 1e-6 h on 1000 seeded nodes (L is affine in each coordinate, so the
    difference carries rounding error only)."""
    from paper_2502_00778_gb300 import api
    m = _mesh("kuhn96")
    x = torch.from_numpy(m.x).to(DEV)
    topo = api.edge_build(torch.from_numpy(m.elems).to(DEV), x)
    api.plan_build(topo, 128)
    t = oracle.topology(3, m.elems, m.x)
    assert np.array_equal(topo.edges.cpu().numpy(), t.edges)
    w, c = meshgen.generate.loss_weights(t.n_edges, m.n_nodes, 3, seed=SEED + 5)
    wt, ct = torch.from_numpy(w).to(DEV), torch.from_numpy(c).to(DEV)
    rg = oracle.adjoint(3, m.x, m.elems, t, w, c)
    tol = 1e-12 * np.abs(rg).max()
    for prec, path, tile in [("dw", "tiled", 128), ("fp64", "tiled", 128), ("dw", "gather", 128),
                             ("fp64", "gather", 128), ("dw", "tiled", 256), ("fp64", "atomic", 128)]:
        api.plan_build(topo, tile)
        g = api.edge_metrics_adjoint(topo, x, wt, ct, prec, path).cpu().numpy()
        assert np.abs(g - rg).max() <= tol, (prec, path, tile)
    nodes = meshgen.generate.fd_nodes(m.n_nodes, 1000, seed=SEED + 6)
    gfd = oracle.fd_gradient(3, m.x, m.elems, t, w, c, nodes, 1e-6 * m.h)
    assert np.abs(g[nodes] - gfd).max() <= 1e-7 * np.abs(rg).max()


def test_paper_2d_grid_size():
    """The paper's 2D grid size (255^2 x 2 = 130,050 triangles, 65,536 nodes):
    the tiled fused DW step and the CSR path against the full oracle."""
    from paper_2502_00778_gb300 import api
    m = _mesh("tri255")
    assert (m.n_nodes, m.n_elems) == (65536, 130050)
    x = torch.from_numpy(m.x).to(DEV)
    topo = api.edge_build(torch.from_numpy(m.elems).to(DEV), x)
    t = oracle.topology(2, m.elems, m.x)
    assert np.array_equal(topo.edges.cpu().numpy(), t.edges)
    rn, rv, rb = oracle.direct(2, m.x, m.elems, t)
    w, c = meshgen.generate.loss_weights(t.n_edges, m.n_nodes, 2, seed=SEED + 9)
    rg = oracle.adjoint(2, m.x, m.elems, t, w, c)
    api.plan_build(topo, 128)
    n, v, b, g = api.edge_metrics_fused(topo, x, torch.from_numpy(w).to(DEV), torch.from_numpy(c).to(DEV), "dw",
                                        path="tiled")
    h = m.h
    assert np.abs(n.cpu().numpy() - rn).max() <= 1e-12 * h
    assert np.abs(v.cpu().numpy() - rv).max() <= 1e-12 * h * h
    assert np.abs(b.cpu().numpy() - rb).max() <= 1e-12 * h
    assert np.abs(g.cpu().numpy() - rg).max() <= 1e-12 * np.abs(rg).max()
    n2, v2, b2 = api.edge_metrics(topo, x, "fp64", "csr")
    assert np.array_equal(n2.cpu().numpy(), rn) and np.array_equal(v2.cpu().numpy(), rv)

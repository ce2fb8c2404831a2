"""Tiled gather path (EM_PATH_GATHER): FP64 and DW forms against the oracle
at the FP64 contract, MIXED at FP32 level, bit-reproducibility, and several
tile sizes (halos, multi-chunk tiles, ragged last tile)."""
import numpy as np
import pytest

import oracle
from _helpers import SMALL_MESHES, assert_close_g, assert_close_n, assert_close_v, hscale, loss_weights, mesh, \
    oracle_fwd, oracle_topo

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"
_topos = {}


def _setup(name, tile_nodes=128):
    from paper_2502_00778_gb300 import api
    key = (name, tile_nodes)
    if key not in _topos:
        m = mesh(name)
        x = torch.from_numpy(m.x).to(DEV)
        topo = api.edge_build(torch.from_numpy(m.elems).to(DEV), x)
        api.plan_build(topo, tile_nodes)
        _topos[key] = (m, x, topo)
    return _topos[key]


@pytest.mark.parametrize("prec", ["fp64", "dw"])
@pytest.mark.parametrize("name", list(SMALL_MESHES))
def test_forward_contract(name, prec):
    from paper_2502_00778_gb300 import api
    m, x, topo = _setup(name)
    n, v, b = api.edge_metrics(topo, x, prec, "gather")
    rn, rv, rb = oracle_fwd(name)
    assert_close_n(n.cpu().numpy(), rn, m)
    assert_close_v(v.cpu().numpy(), rv, m)
    assert_close_n(b.cpu().numpy(), rb, m, "bnormal")


def _or_too_big(fn):
    """Run fn; a tile whose shared-memory need exceeds the GPU limit must be
    refused with a clear error (never a fault): return None then."""
    from paper_2502_00778_gb300 import EMError
    try:
        return fn()
    except EMError as ex:
        assert "shared memory" in str(ex) and "tile_nodes" in str(ex), str(ex)
        return None


@pytest.mark.parametrize("tile", [32, 64, 128, 256, 512, 2048])
@pytest.mark.parametrize("name", ["tri_odd", "kuhn7_off", "kuhn11_nomorton", "kuhn48"])
def test_tile_sizes(name, tile):
    from paper_2502_00778_gb300 import api, EMError
    try:
        m, x, topo = _setup(name, tile)
    except EMError as ex:       # tiles beyond the 16-bit local index range are refused at plan build
        assert "16-bit" in str(ex) and tile > 256, str(ex)
        return
    rn, rv, rb = oracle_fwd(name)
    r = _or_too_big(lambda: api.edge_metrics(topo, x, "dw", "gather"))
    if r is not None:
        n, v, b = r
        assert_close_n(n.cpu().numpy(), rn, m)
        assert_close_v(v.cpu().numpy(), rv, m)
        assert_close_n(b.cpu().numpy(), rb, m, "bnormal")
    elif tile <= 128:
        raise AssertionError("tiles of <= 128 nodes must fit in shared memory")
    w, c = loss_weights(name)
    g = _or_too_big(lambda: api.edge_metrics_adjoint(topo, x, torch.from_numpy(w).to(DEV),
                                                     torch.from_numpy(c).to(DEV), "dw", "gather"))
    if g is not None:
        rg = oracle.adjoint(m.dim, m.x, m.elems, oracle_topo(name), w, c)
        assert_close_g(g.cpu().numpy(), rg)


@pytest.mark.parametrize("name", ["tri16", "kuhn48", "kuhn7_off"])
def test_forward_mixed(name):
    from paper_2502_00778_gb300 import api
    m, x, topo = _setup(name)
    n, v, b = api.edge_metrics(topo, x, "mixed", "gather")
    rn, rv, rb = oracle_fwd(name)
    h = hscale(m)
    en = np.abs(n.cpu().numpy() - rn).max() / h ** (m.dim - 1)
    ev = np.abs(v.cpu().numpy() - rv).max() / h ** m.dim
    eb = np.abs(b.cpu().numpy() - rb).max() / h ** (m.dim - 1)
    assert en < 2e-6 and ev < 2e-6 and eb < 2e-6, (en, ev, eb)


@pytest.mark.parametrize("prec", ["fp64", "dw"])
@pytest.mark.parametrize("name", ["tri16", "tri_odd", "single2", "single3", "kuhn5", "kuhn7_off", "kuhn48"])
def test_adjoint_contract(name, prec):
    from paper_2502_00778_gb300 import api
    m, x, topo = _setup(name)
    w, c = loss_weights(name)
    g = api.edge_metrics_adjoint(topo, x, torch.from_numpy(w).to(DEV), torch.from_numpy(c).to(DEV), prec, "gather")
    rg = oracle.adjoint(m.dim, m.x, m.elems, oracle_topo(name), w, c)
    assert_close_g(g.cpu().numpy(), rg)


def test_adjoint_mixed(name="kuhn48"):
    from paper_2502_00778_gb300 import api
    m, x, topo = _setup(name)
    w, c = loss_weights(name)
    g = api.edge_metrics_adjoint(topo, x, torch.from_numpy(w).to(DEV), torch.from_numpy(c).to(DEV), "mixed", "gather")
    rg = oracle.adjoint(m.dim, m.x, m.elems, oracle_topo(name), w, c)
    assert np.abs(g.cpu().numpy() - rg).max() / np.abs(rg).max() < 1e-5


@pytest.mark.parametrize("prec", ["fp64", "dw", "mixed"])
@pytest.mark.parametrize("name", ["tri_odd", "kuhn7_off", "kuhn48"])
def test_fused_equals_separate_and_is_deterministic(name, prec):
    from paper_2502_00778_gb300 import api
    m, x, topo = _setup(name)
    w, c = loss_weights(name)
    wt, ct = torch.from_numpy(w).to(DEV), torch.from_numpy(c).to(DEV)
    n1, v1, b1, g1 = api.edge_metrics_fused(topo, x, wt, ct, prec)
    n2, v2, b2 = api.edge_metrics(topo, x, prec, "gather")
    g2 = api.edge_metrics_adjoint(topo, x, wt, ct, prec, "gather")
    n3, v3, b3, g3 = api.edge_metrics_fused(topo, x, wt, ct, prec)
    for a, bb, cc in [(n1, n2, n3), (v1, v2, v3), (b1, b2, b3), (g1, g2, g3)]:
        assert torch.equal(a, bb) and torch.equal(a, cc)
    if prec != "mixed":
        rn, rv, rb = oracle_fwd(name)
        assert_close_n(n1.cpu().numpy(), rn, m)
        assert_close_g(g1.cpu().numpy(), oracle.adjoint(m.dim, m.x, m.elems, oracle_topo(name), w, c))


def test_adjoint_without_c(name="kuhn5"):
    from paper_2502_00778_gb300 import api
    m, x, topo = _setup(name)
    w, c = loss_weights(name)
    g = api.edge_metrics_adjoint(topo, x, torch.from_numpy(w).to(DEV), None, "dw", "gather")
    rg = oracle.adjoint(m.dim, m.x, m.elems, oracle_topo(name), w, np.zeros_like(c))
    assert_close_g(g.cpu().numpy(), rg)


def test_gather_autograd(name="kuhn7_off"):
    from paper_2502_00778_gb300 import api
    m, x, topo = _setup(name)
    w, c = loss_weights(name)
    xr = x.clone().requires_grad_(True)
    n, v, b = api.EdgeMetrics.apply(xr, topo, "dw", "gather")
    L = (n * torch.from_numpy(w).to(DEV)).sum() + (v * torch.from_numpy(c).to(DEV)).sum()
    L.backward()
    assert_close_g(xr.grad.cpu().numpy(), oracle.adjoint(m.dim, m.x, m.elems, oracle_topo(name), w, c))

"""Atomic-scatter path (FP64, mixed, compensated FP32) against the oracle."""
import numpy as np
import pytest

from _helpers import SMALL_MESHES, assert_close_g, assert_close_n, assert_close_v, loss_weights, mesh, oracle_fwd, \
    oracle_topo, hscale
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _setup(name):
    from paper_2502_00778_gb300 import api
    m = mesh(name)
    x = torch.from_numpy(m.x).to(DEV)
    topo = api.edge_build(torch.from_numpy(m.elems).to(DEV), x)
    return m, x, topo


@pytest.mark.parametrize("name", list(SMALL_MESHES))
def test_forward_fp64(name):
    from paper_2502_00778_gb300 import api
    m, x, topo = _setup(name)
    n, v, b = api.edge_metrics(topo, x, "fp64", "atomic")
    rn, rv, rb = oracle_fwd(name)
    assert_close_n(n.cpu().numpy(), rn, m)
    assert_close_v(v.cpu().numpy(), rv, m)
    assert_close_n(b.cpu().numpy(), rb, m, "bnormal")


@pytest.mark.parametrize("prec", ["mixed", "mixed_comp32"])
@pytest.mark.parametrize("name", ["tri16", "kuhn48", "kuhn7_off"])
def test_forward_mixed_error_is_fp32_level(name, prec):
    from paper_2502_00778_gb300 import api
    m, x, topo = _setup(name)
    n, v, b = api.edge_metrics(topo, x, prec, "atomic")
    rn, rv, rb = oracle_fwd(name)
    h = hscale(m)
    en = np.abs(n.cpu().numpy() - rn).max() / h ** (m.dim - 1)
    ev = np.abs(v.cpu().numpy() - rv).max() / h ** m.dim
    assert en < 2e-6 and ev < 2e-6, (en, ev)
    assert_close_n(b.cpu().numpy(), rb, m, "bnormal")   # boundary normals stay FP64


@pytest.mark.parametrize("name", ["tri16", "tri_odd", "single2", "single3", "kuhn5", "kuhn7_off", "kuhn48"])
def test_adjoint_fp64(name):
    from paper_2502_00778_gb300 import api
    m, x, topo = _setup(name)
    w, c = loss_weights(name)
    g = api.edge_metrics_adjoint(topo, x, torch.from_numpy(w).to(DEV), torch.from_numpy(c).to(DEV), "fp64", "atomic")
    rg = oracle.adjoint(m.dim, m.x, m.elems, oracle_topo(name), w, c)
    assert_close_g(g.cpu().numpy(), rg)


def test_adjoint_mixed_error(name="kuhn48"):
    from paper_2502_00778_gb300 import api
    m, x, topo = _setup(name)
    w, c = loss_weights(name)
    g = api.edge_metrics_adjoint(topo, x, torch.from_numpy(w).to(DEV), torch.from_numpy(c).to(DEV), "mixed", "atomic")
    rg = oracle.adjoint(m.dim, m.x, m.elems, oracle_topo(name), w, c)
    err = np.abs(g.cpu().numpy() - rg).max() / np.abs(rg).max()
    assert err < 1e-5, err


def test_autograd_function(name="kuhn5"):
    from paper_2502_00778_gb300 import api
    m, x, topo = _setup(name)
    w, c = loss_weights(name)
    xr = x.clone().requires_grad_(True)
    n, v, b = api.EdgeMetrics.apply(xr, topo, "fp64", "atomic")
    L = (n * torch.from_numpy(w).to(DEV)).sum() + (v * torch.from_numpy(c).to(DEV)).sum()
    L.backward()
    rg = oracle.adjoint(m.dim, m.x, m.elems, oracle_topo(name), w, c)
    assert_close_g(xr.grad.cpu().numpy(), rg)


@pytest.mark.parametrize("name", list(SMALL_MESHES))
def test_traditional_dual_faces(name):
    """The traditional dual-face construction on the GPU (the paper's
    comparison algorithm) against the oracle's, and against the proposed
    formula's n_jk, which it equals up to rounding."""
    from paper_2502_00778_gb300 import api
    m = mesh(name)
    x = torch.from_numpy(m.x).to(DEV)
    topo = api.edge_build(torch.from_numpy(m.elems).to(DEV), x)
    nt = api.edge_areas_traditional(topo, x).cpu().numpy()
    assert_close_n(nt, oracle.traditional(m.dim, m.x, m.elems, oracle_topo(name)), m, "traditional n")
    rn, _, _ = oracle_fwd(name)
    assert_close_n(nt, rn, m, "traditional vs proposed n")


@pytest.mark.parametrize("name", ["tri16", "kuhn5", "kuhn7_off", "single3"])
def test_adjoint_boundary_weights(name):
    """L = sum w.n + sum c V + sum bw.bnormal: the atomic and tiled adjoints
    and the fused tiled pass against the oracle, and autograd through all
    three outputs."""
    from paper_2502_00778_gb300 import api
    m, x, topo = _setup(name)
    w, c = loss_weights(name)
    t = oracle_topo(name)
    rng = np.random.Generator(np.random.PCG64(17))
    bw = rng.standard_normal((len(t.bnode), m.dim))
    wt, ct, bt = (torch.from_numpy(a).to(DEV) for a in (w, c, bw))
    rg = oracle.adjoint(m.dim, m.x, m.elems, t, w, c, bw)
    g = api.edge_metrics_adjoint(topo, x, wt, ct, "fp64", "atomic", bw=bt)
    assert_close_g(g.cpu().numpy(), rg)
    api.plan_build(topo, 64)
    for prec in ("fp64", "dw"):
        g = api.edge_metrics_adjoint(topo, x, wt, ct, prec, "tiled", bw=bt)
        assert_close_g(g.cpu().numpy(), rg)
        _, _, _, g = api.edge_metrics_fused(topo, x, wt, ct, prec, path="tiled", bw=bt)
        assert_close_g(g.cpu().numpy(), rg)
    g = api.edge_metrics_adjoint(topo, x, wt, ct, "mixed", "tiled", bw=bt)
    assert np.abs(g.cpu().numpy() - rg).max() <= 1e-5 * np.abs(rg).max()
    xr = x.clone().requires_grad_(True)
    n, v, b = api.EdgeMetrics.apply(xr, topo, "fp64", "atomic")
    L = (n * wt).sum() + (v * ct).sum() + (b * bt).sum()
    L.backward()
    assert_close_g(xr.grad.cpu().numpy(), rg)
    from paper_2502_00778_gb300 import EMError
    with pytest.raises(EMError):
        api.edge_metrics_adjoint(topo, x, wt, ct, "dw", "gather", bw=bt)

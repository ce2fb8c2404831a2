"""Edge-based dual volume (Sec. 4.1) on the GPU: bit-identical to the
oracle's serial edge loop for the same n, and equal to the element-based
volume within the FP64 contract (flat boundary faces)."""
import numpy as np
import pytest

import oracle
from _helpers import SMALL_MESHES, assert_close_v, hscale, mesh, oracle_fwd, oracle_topo

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.mark.parametrize("name", list(SMALL_MESHES))
def test_edge_volume(name):
    from paper_2502_00778_gb300 import api
    m = mesh(name)
    x = torch.from_numpy(m.x).to(DEV)
    topo = api.edge_build(torch.from_numpy(m.elems).to(DEV), x)
    rn, rv, rb = oracle_fwd(name)
    v = api.edge_volume(topo, x, torch.from_numpy(rn).to(DEV)).cpu().numpy()
    assert np.array_equal(v, oracle.edge_volume(m.dim, m.x, oracle_topo(name), rn))
    n, _, _ = api.edge_metrics(topo, x, "fp64", "csr")
    assert_close_v(api.edge_volume(topo, x, n).cpu().numpy(), rv, m)


@pytest.mark.parametrize("name", list(SMALL_MESHES))
def test_edge_residual(name):
    """Edge-loop residual (Sec. 2): bit-identical to the oracle's serial edge
    loop for the same inputs, and V_j div F at interior nodes for a linear F
    with the GPU's own metrics."""
    from paper_2502_00778_gb300 import api
    m = mesh(name)
    t = oracle_topo(name)
    x = torch.from_numpy(m.x).to(DEV)
    topo = api.edge_build(torch.from_numpy(m.elems).to(DEV), x)
    rn, rv, rb = oracle_fwd(name)
    rng = np.random.Generator(np.random.PCG64(91))
    A = rng.standard_normal((m.dim, m.dim))
    F = (m.x - m.x.mean(axis=0)) @ A.T + rng.standard_normal(m.dim)
    Ft = torch.from_numpy(F).to(DEV)
    r = api.edge_residual(topo, Ft, torch.from_numpy(rn).to(DEV), torch.from_numpy(rb).to(DEV)).cpu().numpy()
    assert np.array_equal(r, oracle.edge_residual(m.dim, t, rn, F, rb))
    n, v, b = api.edge_metrics(topo, x, "fp64", "csr")
    r2 = api.edge_residual(topo, Ft, n, b).cpu().numpy()
    inner = np.ones(m.n_nodes, bool)
    inner[t.bnode] = False
    scale = np.abs(F).max() * hscale(m) ** (m.dim - 1)
    if inner.any():                              # single elements have no interior node
        assert np.abs(r2[inner] - rv[inner] * np.trace(A)).max() <= 1e-12 * scale

"""edge_build on the GPU is bit-exact against the oracle's topology."""
import numpy as np
import pytest

import meshgen
import oracle
from _helpers import SMALL_MESHES, mesh, oracle_topo

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _gpu_topo(m):
    from paper_2502_00778_gb300 import api
    dev = torch.device("cuda:0")
    return api.edge_build(torch.from_numpy(m.elems).to(dev), torch.from_numpy(m.x).to(dev))


@pytest.mark.parametrize("name", list(SMALL_MESHES))
def test_edge_build_bit_exact(name):
    m = mesh(name)
    t = oracle_topo(name)
    g = _gpu_topo(m)
    assert np.array_equal(g.edges.cpu().numpy(), t.edges)
    assert np.array_equal(g.elem2edge.cpu().numpy(), t.elem2edge)
    assert np.array_equal(g.bface.cpu().numpy(), t.bface)
    assert np.array_equal(g.bface_owner.cpu().numpy(), t.bowner)
    assert np.array_equal(g.bnode.cpu().numpy(), t.bnode)
    # CSR: slots of each edge, ascending
    nle = 6 if m.dim == 3 else 3
    ptr = g.edge_ptr.cpu().numpy()
    slot = g.edge_slot.cpu().numpy()
    assert ptr[0] == 0 and ptr[-1] == nle * m.n_elems
    flat = t.elem2edge.ravel()
    order = np.lexsort((np.arange(flat.size), flat))
    assert np.array_equal(slot, order)


def test_edge_build_errors():
    from paper_2502_00778_gb300 import api, EMError
    m = meshgen.kuhn_cube(2, jitter=0.0)
    dev = torch.device("cuda:0")
    el = m.elems.copy()
    el[3, 1] = m.n_nodes + 5          # out of range id
    with pytest.raises(EMError, match="BAD_ID"):
        api.edge_build(torch.from_numpy(el).to(dev), torch.from_numpy(m.x).to(dev))
    el = m.elems.copy()
    el[2, 2] = el[2, 0]               # repeated node
    with pytest.raises(EMError, match="BAD_ID"):
        api.edge_build(torch.from_numpy(el).to(dev), torch.from_numpy(m.x).to(dev))
    # a face shared by three elements
    el = np.concatenate([m.elems, m.elems[:1]], 0)
    with pytest.raises(EMError, match="TOPOLOGY"):
        api.edge_build(torch.from_numpy(el).to(dev), torch.from_numpy(m.x).to(dev))
    # degenerate element (all four nodes coplanar)
    x = m.x.copy()
    e0 = m.elems[0]
    x[e0[3]] = x[e0[0]] + 0.5 * (x[e0[1]] - x[e0[0]]) + 0.5 * (x[e0[2]] - x[e0[0]])
    with pytest.raises(EMError, match="DEGENERATE"):
        api.check_elements(3, torch.from_numpy(m.elems).to(dev), torch.from_numpy(x).to(dev))
    assert api.check_elements(3, torch.from_numpy(m.elems).to(dev), torch.from_numpy(m.x).to(dev)) == (0, 0)

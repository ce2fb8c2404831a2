"""Edge-based dual volume (Sec. 4.1) on the GPU: bit-identical to the
oracle's serial edge loop for the same n, and equal to the element-based
volume within the FP64 contract (flat boundary faces)."""
import numpy as np
import pytest

import oracle
from _helpers import SMALL_MESHES, assert_close_v, mesh, oracle_fwd, oracle_topo

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

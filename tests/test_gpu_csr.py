"""CSR gather path (EM_PATH_CSR, FP64): every output is the same floating-point
expression as in the oracle's serial loops, so the results are bit-identical."""
import numpy as np
import pytest

from _helpers import SMALL_MESHES, mesh, oracle_fwd

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.mark.parametrize("name", list(SMALL_MESHES))
def test_csr_bit_identical_to_oracle(name):
    from paper_2502_00778_gb300 import api
    m = mesh(name)
    x = torch.from_numpy(m.x).to(DEV)
    topo = api.edge_build(torch.from_numpy(m.elems).to(DEV), x)
    n, v, b = api.edge_metrics(topo, x, "fp64", "csr")
    rn, rv, rb = oracle_fwd(name)
    assert np.array_equal(n.cpu().numpy(), rn)
    assert np.array_equal(v.cpu().numpy(), rv)
    assert np.array_equal(b.cpu().numpy(), rb)
    n2, v2, b2 = api.edge_metrics(topo, x, "fp64", "csr")
    assert torch.equal(n, n2) and torch.equal(v, v2) and torch.equal(b, b2)

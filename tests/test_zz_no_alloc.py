"""The allocation-free forward, em_edge_metrics_noalloc.

Some callers cannot allocate device memory while they run -- a solver
plug-in whose host application owns all device memory through its own pool,
or a process held to a fixed device-memory cap -- so they cannot hand the
library a freshly allocated workspace.  For them the library keeps the
scratch of one forward form (the compensated-FP32 atomic scatter) in a fixed
array of its own.  These tests call that entry point through the C ABI, twice
in a row on the same grid (the shared array must be cleared on every call),
and compare it with the workspace form it mirrors, em_edge_metrics(ATOMIC,
MIXED_COMP32), at the tolerance used for that form elsewhere in the suite.
The file is named to be collected last."""
import ctypes

import numpy as np
import pytest

from _helpers import hscale, mesh, oracle_fwd

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"
TOL = 2e-6   # relative to h^(D-1) (vectors) and h^D (volumes), as for the compensated-FP32 form


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


@pytest.mark.parametrize("name", ["tri16", "kuhn48", "kuhn7_off"])
def test_noalloc_matches_workspace_form_on_two_calls(name):
    from paper_2502_00778_gb300 import api, load
    from paper_2502_00778_gb300._lib import check
    L = load()
    m = mesh(name)
    x = torch.from_numpy(m.x).to(DEV)
    topo = api.edge_build(torch.from_numpy(m.elems).to(DEV), x)
    n0, v0, b0 = api.edge_metrics(topo, x, "mixed_comp32", "atomic")
    ms = topo.em_mesh()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    h = hscale(m)
    rn, rv, rb = oracle_fwd(name)
    n = torch.empty_like(n0)
    v = torch.empty_like(v0)
    b = torch.empty_like(b0)
    for call in range(2):
        for t in (n, v, b):
            t.fill_(float("nan"))
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        check(L.em_edge_metrics_noalloc(ctypes.byref(ms), _p(x), _p(n), _p(v), _p(b), stream))
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info()[0]
        if call == 1:
            # the first call may load the module (and commit its array); the
            # second must not change the device's free memory at all
            assert free1 == free0
        assert (n - n0).abs().max().item() <= TOL * h ** (m.dim - 1)
        assert (v - v0).abs().max().item() <= TOL * h ** m.dim
        assert (b - b0).abs().max().item() <= TOL * h ** (m.dim - 1)
        assert np.abs(n.cpu().numpy() - rn).max() <= TOL * h ** (m.dim - 1)


def test_noalloc_rejects_grids_beyond_its_scratch():
    from paper_2502_00778_gb300 import api, load
    L = load()
    m = mesh("kuhn5")
    x = torch.from_numpy(m.x).to(DEV)
    topo = api.edge_build(torch.from_numpy(m.elems).to(DEV), x)
    ms = topo.em_mesh()
    ms.n_edges = 3_000_000            # 4 * (6 * 3e6 + ...) bytes > 64 MiB: refused before any device work
    out = torch.empty(8, dtype=torch.float64, device=DEV)
    st = L.em_edge_metrics_noalloc(ctypes.byref(ms), _p(x), _p(out), _p(out), _p(out), ctypes.c_void_p(0))
    assert st == -1
    buf = ctypes.create_string_buffer(256)
    L.em_last_error(buf, 256)
    assert b"scratch" in buf.value

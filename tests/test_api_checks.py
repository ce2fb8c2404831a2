"""The Python binding refuses tensors that do not fit the grid before it
passes any pointer to the library (no GPU needed): a wrong number of
elements, an output that is not contiguous float64, a batched input whose
memory would be used as is in another dtype, a tensor on another device.
The library reads and writes through plain pointers, so any of these would
otherwise make a kernel access memory outside the tensor."""
import pytest

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def api():
    import __graft_entry__  # noqa: F401  (puts the repository root on the path)
    from paper_2502_00778_gb300 import api as a, build
    build.build()
    return a


N_NODES, N_ELEMS, N_EDGES, N_BF, N_BN, D = 27, 48, 98, 48, 26, 3


@pytest.fixture
def topo(api):
    """A host-side topology with the sizes of a 2^3 x 6 Kuhn grid (the
    contents are never read: every call below fails its checks first)."""
    i32 = dict(dtype=torch.int32)
    t = api.Topology(D, torch.zeros((N_ELEMS, 4), **i32), torch.zeros((N_EDGES, 2), **i32),
                     torch.zeros((N_ELEMS, 6), **i32), None, None, torch.zeros((N_BF, 3), **i32),
                     torch.zeros(N_BF, **i32), torch.zeros(N_BN, **i32), N_NODES)
    t.plan = torch.zeros(256, dtype=torch.uint8)
    return t


def f64(*shape):
    return torch.zeros(shape, dtype=torch.float64)


def inputs():
    return f64(N_NODES, D), f64(N_EDGES, D), f64(N_NODES)


def test_sizes_are_checked_before_anything_reaches_the_library(api, topo):
    x, w, c = inputs()
    with pytest.raises(ValueError, match=r"x has 78 elements; this grid needs 81"):
        api.edge_metrics(topo, f64(N_NODES - 1, D))
    with pytest.raises(ValueError, match=r"w has"):
        api.edge_metrics_adjoint(topo, x, f64(N_EDGES - 1, D), c)
    with pytest.raises(ValueError, match=r"c has"):
        api.edge_metrics_fused(topo, x, w, f64(N_NODES + 1))
    with pytest.raises(ValueError, match=r"bw has"):
        api.edge_metrics_fused(topo, x, w, c, bw=f64(N_BN + 1, D))
    with pytest.raises(ValueError, match=r"x has"):
        api.edge_metrics_partial(topo, f64(2 * N_NODES, D), (0, 1))
    with pytest.raises(ValueError, match=r"n_edge has"):
        api.edge_volume(topo, x, f64(N_EDGES, 2))
    with pytest.raises(ValueError, match=r"F has"):
        api.edge_residual(topo, f64(N_NODES), f64(N_EDGES, D), f64(N_BN, D))
    with pytest.raises(ValueError, match=r"bnormal has"):
        api.edge_residual(topo, x, f64(N_EDGES, D), f64(N_BN - 1, D))


def test_outputs_must_fit_and_be_contiguous_float64(api, topo):
    x, w, c = inputs()
    n, v, b, g = f64(N_EDGES, D), f64(N_NODES), f64(N_BN, D), f64(N_NODES, D)
    with pytest.raises(ValueError, match=r"vol has"):
        api.edge_metrics(topo, x, out=(n, f64(N_NODES - 1), b))
    with pytest.raises(ValueError, match=r"n_edge must be a contiguous float64"):
        api.edge_metrics(topo, x, out=(n.to(torch.float32), v, b))
    with pytest.raises(ValueError, match=r"grad must be a contiguous float64"):
        api.edge_metrics_fused(topo, x, w, c, out=(n, v, b, f64(D, N_NODES).t()))
    with pytest.raises(ValueError, match=r"grad has"):
        api.edge_metrics_adjoint(topo, x, w, c, out=f64(N_NODES))
    with pytest.raises(ValueError, match=r"n_edge has"):
        api.edge_areas_traditional(topo, x, out=f64(N_EDGES - 1, D))


def test_batched_inputs_are_used_as_is(api, topo):
    x, w, c = inputs()
    with pytest.raises(ValueError, match=r"xs\[0\] must be a contiguous float64"):
        api.Batch([topo], [x.to(torch.float32)], [w], [c])
    with pytest.raises(ValueError, match=r"ws\[0\] has"):
        api.Batch([topo], [x], [f64(N_EDGES + 1, D)], [c])
    with pytest.raises(ValueError, match=r"one x, w and c per grid"):
        api.Batch([topo], [x], [w, w], [c])


def test_fitting_host_tensors_pass_the_size_checks(api, topo):
    """With every size right, the next check is the device: host tensors are
    refused as such, still before any pointer reaches the library."""
    x, w, c = inputs()
    with pytest.raises(ValueError, match=r"CUDA tensors"):
        api.edge_metrics_fused(topo, x, w, c)
    with pytest.raises(ValueError, match=r"CUDA tensors"):
        api.edge_metrics(topo, x, out=(f64(N_EDGES, D), f64(N_NODES), f64(N_BN, D)))


def test_tensors_on_another_device_are_refused(api, topo):
    x, w, c = inputs()
    meta = torch.zeros((N_EDGES, D), dtype=torch.float64, device="meta")
    with pytest.raises(ValueError, match=r"w is on meta"):
        api.edge_metrics_adjoint(topo, x, meta, c)

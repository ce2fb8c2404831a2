"""Edge cases of the GPU paths against the oracle.

* Tiles without elements: nodes that no element references, inserted inside
  the node numbering and appended after it, so that some tiles of a plan own
  only such nodes and others mix them with grid nodes.  Their volume and
  gradient are exactly 0, and every other output meets the FP64 contract on
  the atomic, gather and tiled paths.
* The tiled path's fixed-point headroom (an int32 limb-plane entry holds
  fewer than 1024 limbs, so an edge may have at most 340 elements and a node
  at most 170): a fan of tetrahedra around one axis edge puts the axis edge
  and its two end nodes at any valence, with congruent elements, so the
  rounding errors of the fixed-point sums add up instead of averaging out.
  Up to the node limit the tiled forms meet the contract; one element more
  and the tiled and batched paths refuse the grid, while the gather and
  atomic paths still meet it.  At 400 elements (slivers of aspect ratio 64,
  sums that cancel 60-fold) the double-word arithmetic of the DW form, about
  2^-48 per operation, stays within 1e-11 rather than 1e-12; the FP64 forms
  stay within the contract.
"""
import numpy as np
import pytest

import meshgen
import oracle
from _helpers import assert_close_g, assert_close_n, assert_close_v

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _grid_with_isolated_nodes(inserted=70, at=100, appended=130):
    """The 5^3 x 6 jittered Kuhn grid with `inserted` unreferenced nodes at
    ids [at, at + inserted) and `appended` more after the grid's nodes."""
    m = meshgen.kuhn_cube(5, jitter=0.3, seed=meshgen.SEED_BASE + 504)
    n0 = m.n_nodes
    el = m.elems.astype(np.int64)
    el = np.where(el >= at, el + inserted, el)
    rng = np.random.Generator(np.random.PCG64(meshgen.SEED_BASE + 40))
    x = np.empty((n0 + inserted + appended, 3))
    x[:at] = m.x[:at]
    x[at + inserted:n0 + inserted] = m.x[at:]
    x[at:at + inserted] = rng.uniform(2.0, 3.0, (inserted, 3))      # away from the grid
    x[n0 + inserted:] = rng.uniform(-3.0, -2.0, (appended, 3))
    iso = np.r_[np.arange(at, at + inserted), np.arange(n0 + inserted, n0 + inserted + appended)]
    mm = meshgen.generate.Mesh(name="kuhn5_isolated", dim=3, x=x, elems=el.astype(np.int32), h=m.h, meta={})
    return mm, iso


def _fan(k):
    """k tetrahedra (a, b, p_i, p_{i+1}) around the axis edge a = (0,0,0),
    b = (0,0,1), with p_i on the unit circle at height 1/2: edge ab and nodes
    a and b belong to all k elements; positively oriented."""
    th = 2.0 * np.pi * np.arange(k) / k
    x = np.zeros((k + 2, 3))
    x[1] = (0.0, 0.0, 1.0)
    x[2:, 0], x[2:, 1], x[2:, 2] = np.cos(th), np.sin(th), 0.5
    i = np.arange(k)
    el = np.stack([np.zeros(k, np.int64), np.ones(k, np.int64), 2 + i, 2 + (i + 1) % k], 1)
    a, b, c = (x[el[:, j]] - x[el[:, 0]] for j in (1, 2, 3))
    neg = np.einsum("ij,ij->i", a, np.cross(b, c)) < 0
    el[neg, 2], el[neg, 3] = el[neg, 3].copy(), el[neg, 2].copy()
    return meshgen.generate.Mesh(name=f"fan{k}", dim=3, x=x, elems=el.astype(np.int32), h=1.0, meta={})


def _weights(m, n_edges, seed):
    return meshgen.generate.loss_weights(n_edges, m.n_nodes, 3, seed=seed)


def _setup(m, tile_nodes):
    from paper_2502_00778_gb300 import api
    x = torch.from_numpy(m.x).to(DEV)
    topo = api.edge_build(torch.from_numpy(m.elems).to(DEV), x)
    api.plan_build(topo, tile_nodes)
    ot = oracle.topology(3, m.elems, m.x)
    w, c = _weights(m, topo.n_edges, meshgen.SEED_BASE + 41)
    ref = oracle.direct(3, m.x, m.elems, ot) + (oracle.adjoint(3, m.x, m.elems, ot, w, c),)
    return x, topo, torch.from_numpy(w).to(DEV), torch.from_numpy(c).to(DEV), ref


def _check(m, got, ref):
    assert_close_n(got[0].cpu().numpy(), ref[0], m)
    assert_close_v(got[1].cpu().numpy(), ref[1], m)
    assert_close_n(got[2].cpu().numpy(), ref[2], m, "bnormal")
    if len(got) > 3:
        assert_close_g(got[3].cpu().numpy(), ref[3])


# (path, precision): every form that takes a plan, plus the plan-free atomic path
FORMS = [("atomic", "fp64"), ("gather", "dw"), ("tiled", "dw"), ("tiled", "fp64"), ("tiled", "mixed")]


@pytest.mark.parametrize("tile_nodes", [64, 128])
@pytest.mark.parametrize("path,prec", FORMS)
def test_tiles_without_elements(path, prec, tile_nodes):
    from paper_2502_00778_gb300 import api
    m, iso = _grid_with_isolated_nodes()
    x, topo, w, c, ref = _setup(m, tile_nodes)
    assert api.plan_tiles(topo) * tile_nodes >= m.n_nodes
    assert np.all(ref[1][iso] == 0.0) and np.all(ref[3][iso] == 0.0)
    if path == "atomic":
        got = api.edge_metrics(topo, x, prec, "atomic") + (
            api.edge_metrics_adjoint(topo, x, w, c, prec, "atomic"),)
    else:
        got = api.edge_metrics_fused(topo, x, w, c, prec, path=path)
    if prec == "mixed":   # FP32-level form: outputs at FP32 accuracy, exact zeros still exact
        for g, r in zip(got, ref):
            g = g.cpu().numpy()
            assert np.abs(g - r).max() <= 1e-5 * max(np.abs(r).max(), 1e-300)
    else:
        _check(m, got, ref)
    assert np.all(got[1].cpu().numpy()[iso] == 0.0)
    assert np.all(got[3].cpu().numpy()[iso] == 0.0)
    # separate forward on the same plan
    if path != "atomic":
        fwd = api.edge_metrics(topo, x, prec, path)
        assert np.all(fwd[1].cpu().numpy()[iso] == 0.0)


@pytest.mark.parametrize("k", [40, 100, 168])
def test_tiled_up_to_the_node_valence_limit(k):
    """k elements at nodes a and b (limit 170) and at edge ab (limit 340):
    accepted, FP64 contract on the tiled DW and FP64 forms, bit-reproducible."""
    from paper_2502_00778_gb300 import api
    from paper_2502_00778_gb300._lib import PLAN_INFO
    m = _fan(k)
    x, topo, w, c, ref = _setup(m, 64)
    assert topo.plan_info[PLAN_INFO["max_node_valence"]] == k
    assert topo.plan_info[PLAN_INFO["max_edge_valence"]] == k
    for prec in ("dw", "fp64"):
        got = api.edge_metrics_fused(topo, x, w, c, prec, path="tiled")
        _check(m, got, ref)
        again = api.edge_metrics_fused(topo, x, w, c, prec, path="tiled")
        for g, a in zip(got, again):
            assert torch.equal(g, a)


@pytest.mark.parametrize("k", [171, 400])
def test_above_the_valence_limits(k):
    """171 elements at a node (limit 170), 400 at an edge (limit 340): the
    tiled and batched paths refuse the grid before any launch; the gather
    and atomic paths still meet the FP64 contract."""
    from paper_2502_00778_gb300 import api, EMError
    m = _fan(k)
    x, topo, w, c, ref = _setup(m, 64)
    with pytest.raises(EMError, match="headroom"):
        api.edge_metrics_fused(topo, x, w, c, "dw", path="tiled")
    with pytest.raises(EMError, match="headroom"):
        api.edge_metrics(topo, x, "dw", "tiled")
    with pytest.raises(EMError, match="headroom"):
        b = api.Batch([topo], [x], [w], [c], "dw")
        b.run()
    _check(m, api.edge_metrics_fused(topo, x, w, c, "fp64", path="gather"), ref)
    _check(m, api.edge_metrics(topo, x, "fp64", "atomic") + (
        api.edge_metrics_adjoint(topo, x, w, c, "fp64", "atomic"),), ref)
    got = api.edge_metrics_fused(topo, x, w, c, "dw", path="gather")
    if k <= 171:
        _check(m, got, ref)
    else:            # double-word arithmetic on slivers: see the module docstring
        for g, r in zip(got, ref):
            assert np.abs(g.cpu().numpy() - r).max() <= 1e-11 * np.abs(r).max()

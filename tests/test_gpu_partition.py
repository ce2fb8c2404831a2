"""One grid split into contiguous element ranges (the multi-GPU partition of
a single grid): each range's contributions come from the CUDA kernels
(em_edge_metrics_partial), and the sum of the partial arrays over the ranges
must equal the oracle's full result at the FP64 contract.  Run once in one
process (ranges one after the other) and once as two processes on cuda:0
that exchange their partial sums through gloo (the kernels of the two
processes never wait on each other)."""
import os
import socket

import numpy as np
import pytest

from _helpers import TOL_G, TOL_N, TOL_V, hscale, loss_weights, mesh, oracle_fwd, oracle_topo

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _oracle_grad(name):
    import oracle
    m = mesh(name)
    w, c = loss_weights(name)
    return oracle.adjoint(m.dim, m.x, m.elems, oracle_topo(name), w, c)


@pytest.mark.parametrize("name,ranges", [
    ("kuhn48", 2),
    ("kuhn48", [0, 0, 1, 200_000, 200_001, 663_552]),   # uneven, with an empty and one-element ranges
    ("tri16", 3),
    ("kuhn7_off", 4),
])
def test_partials_sum_to_the_oracle(name, ranges):
    from paper_2502_00778_gb300 import api, sharding
    m = mesh(name)
    x = torch.from_numpy(m.x).to(DEV)
    topo = api.edge_build(torch.from_numpy(m.elems).to(DEV), x)
    w, c = loss_weights(name)
    wt, ct = torch.from_numpy(w).to(DEV), torch.from_numpy(c).to(DEV)
    if isinstance(ranges, int):
        bounds = sharding.element_ranges(m.n_elems, ranges)
    else:
        bounds = list(zip(ranges[:-1], ranges[1:]))
    assert bounds[0][0] == 0 and bounds[-1][1] == m.n_elems
    tot = None
    for lo, hi in bounds:
        parts = api.edge_metrics_partial(topo, x, (lo, hi), wt, ct, "fp64")
        tot = list(parts) if tot is None else [a + b for a, b in zip(tot, parts)]
    torch.cuda.synchronize()
    rn, rv, rb = oracle_fwd(name)
    rg = _oracle_grad(name)
    h = hscale(m)
    assert np.abs(tot[0].cpu().numpy() - rn).max() <= TOL_N * h ** (m.dim - 1)
    assert np.abs(tot[1].cpu().numpy() - rv).max() <= TOL_V * h ** m.dim
    assert np.abs(tot[2].cpu().numpy() - rb).max() <= TOL_N * h ** (m.dim - 1)
    assert np.abs(tot[3].cpu().numpy() - rg).max() <= TOL_G * np.abs(rg).max()


def test_one_range_is_the_atomic_path():
    """The whole grid as one range gives the ordinary atomic FP64 results."""
    from paper_2502_00778_gb300 import api
    m = mesh("kuhn5")
    x = torch.from_numpy(m.x).to(DEV)
    topo = api.edge_build(torch.from_numpy(m.elems).to(DEV), x)
    n, v, b, g = api.edge_metrics_partial(topo, x, (0, m.n_elems))
    n0, v0, b0 = api.edge_metrics(topo, x, "fp64", "atomic")
    h = hscale(m)
    assert g is None
    assert (n - n0).abs().max().item() <= 1e-14 * h ** 2
    assert (v - v0).abs().max().item() <= 1e-14 * h ** 3
    assert (b - b0).abs().max().item() <= 1e-14 * h ** 2


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    try:
        import sys
        root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
        sys.path.insert(0, root)
        sys.path.insert(0, os.path.join(root, "tests"))
        os.environ["MASTER_ADDR"] = "127.0.0.1"
        os.environ["MASTER_PORT"] = str(port)
        import torch as T
        import torch.distributed as dist
        from _helpers import loss_weights as lw, mesh as mk
        from paper_2502_00778_gb300 import api, sharding
        dist.init_process_group("gloo", rank=rank, world_size=world)
        m = mk("kuhn48")
        x = T.from_numpy(m.x).to(DEV)
        topo = api.edge_build(T.from_numpy(m.elems).to(DEV), x)
        w, c = lw("kuhn48")
        parts = sharding.partitioned_metrics(topo, x, T.from_numpy(w).to(DEV), T.from_numpy(c).to(DEV))
        out = [a.cpu().numpy() for a in parts]
        dist.destroy_process_group()
        q.put((rank, out))
    except Exception as ex:  # reported to the parent
        q.put((rank, repr(ex)))


def test_two_processes_exchange_partials_through_gloo():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
    for r in range(2):
        assert not isinstance(res[r], str), res[r]
    m = mesh("kuhn48")
    rn, rv, rb = oracle_fwd("kuhn48")
    rg = _oracle_grad("kuhn48")
    h = hscale(m)
    for r in range(2):
        n, v, b, g = res[r]
        assert np.abs(n - rn).max() <= TOL_N * h ** 2
        assert np.abs(v - rv).max() <= TOL_V * h ** 3
        assert np.abs(b - rb).max() <= TOL_N * h ** 2
        assert np.abs(g - rg).max() <= TOL_G * np.abs(rg).max()
    assert np.array_equal(res[0][0], res[1][0])   # every rank holds the same summed arrays

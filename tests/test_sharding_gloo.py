"""Multi-rank logic on CPU (gloo, world sizes 2 and 3): batch sharding and
the single-grid element partition with its one exchange (all-reduce of the
whole partial arrays, or of the interface entries only), checked against the
unpartitioned result.  The per-rank compute here is the oracle: what is
tested is the partition / exchange logic."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    try:
        os.environ["MASTER_ADDR"] = "127.0.0.1"
        os.environ["MASTER_PORT"] = str(port)
        import sys
        sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
        import meshgen
        import oracle
        from paper_2502_00778_gb300 import sharding
        dist.init_process_group("gloo", rank=rank, world_size=world)

        # --- batch of independent grids -----------------------------------
        grids = meshgen.batched_set(7, nmin=2, nmax=6)
        sizes = [g.n_elems for g in grids]
        parts = sharding.shard_grids(sizes, world)
        mine = torch.tensor([1 if i in parts[rank] else 0 for i in range(len(grids))])
        allp = [torch.zeros_like(mine) for _ in range(world)]
        dist.all_gather(allp, mine)
        cover = torch.stack(allp).sum(0)
        assert torch.all(cover == 1), "every grid on exactly one rank"
        vol = torch.zeros(1, dtype=torch.float64)
        for i in parts[rank]:
            g = grids[i]
            t = oracle.topology(3, g.elems, g.x)
            vol += oracle.direct(3, g.x, g.elems, t)[1].sum()
        dist.all_reduce(vol)
        assert abs(vol.item() - len(grids)) < 1e-12      # each grid is a unit cube

        # --- one grid split into element ranges ----------------------------
        m = meshgen.kuhn_cube(6, jitter=0.2, seed=77)
        t = oracle.topology(3, m.elems, m.x)
        lo, hi = sharding.element_ranges(m.n_elems, world)[rank]
        sub = oracle.Topology(3, t.edges, t.elem2edge[lo:hi], t.bface[sharding.owned_boundary_faces(t.bowner, lo, hi)],
                              None, t.bnode)
        n, v, b = oracle.direct(3, m.x, m.elems[lo:hi], sub)
        parts_t = [torch.from_numpy(np.ascontiguousarray(a)) for a in (n, v, b)]
        for a in parts_t:
            dist.all_reduce(a)
        rn, rv, rb = oracle.direct(3, m.x, m.elems, t)
        h = m.h
        assert np.abs(parts_t[0].numpy() - rn).max() <= 1e-13 * h * h
        assert np.abs(parts_t[1].numpy() - rv).max() <= 1e-13 * h ** 3
        assert np.abs(parts_t[2].numpy() - rb).max() <= 1e-13 * h * h
        dist.destroy_process_group()
        q.put((rank, "ok"))
    except Exception as ex:  # report to the parent
        q.put((rank, repr(ex)))


def test_sharding_two_ranks_gloo():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=240) for _ in procs]
    for p in procs:
        p.join(timeout=60)
    assert sorted(res) == [(0, "ok"), (1, "ok")], res


def test_shard_grids_balance():
    from paper_2502_00778_gb300 import sharding
    sizes = [3072 * k for k in (1, 8, 27, 64, 125, 216, 343, 512, 3, 9)]
    for w in (1, 2, 3, 4, 8):
        parts = sharding.shard_grids(sizes, w)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(sizes)))
        loads = [sum(sizes[i] for i in p) for p in parts]
        assert max(loads) <= sum(sizes) / w + max(sizes)    # LPT bound
    assert sharding.element_ranges(10, 3) == [(0, 4), (4, 7), (7, 10)]


def _grid_topology(n=5, seed=78):
    import meshgen
    import oracle
    m = meshgen.kuhn_cube(n, jitter=0.2, seed=seed)
    return m, oracle.topology(3, m.elems, m.x)


def test_interface_targets_against_plain_loops():
    """The interface sets of a 3-way element partition, against per-range
    Python sets built element by element and face by face."""
    from paper_2502_00778_gb300 import sharding
    m, t = _grid_topology()
    ranges = sharding.element_ranges(m.n_elems, 3)
    iface = sharding.interface_targets(3, m.elems, t.elem2edge, t.bface, t.bowner, t.bnode, ranges)
    bpos = {int(node): k for k, node in enumerate(t.bnode)}
    sets = []
    for lo, hi in ranges:
        es, vs, bs = set(), set(), set()
        for e in range(lo, hi):
            es.update(int(k) for k in t.elem2edge[e])
            vs.update(int(k) for k in m.elems[e, :4])
        for f in range(len(t.bface)):
            if lo <= t.bowner[f] // 4 < hi:
                bs.update(bpos[int(k)] for k in t.bface[f])
        sets.append((es, vs, bs))
    for k, key in enumerate(("edges", "nodes", "bnodes")):
        count = {}
        for s in sets:
            for i in s[k]:
                count[i] = count.get(i, 0) + 1
        assert list(iface[key]) == sorted(i for i, c in count.items() if c > 1), key
        for r in range(3):
            assert list(iface["touched"][r][k]) == sorted(sets[r][k]), (key, r)
    # contiguous ranges of Morton-ordered elements leave most targets interior
    assert 0 < len(iface["edges"]) < 0.6 * len(t.edges)


def _interface_worker(rank, world, port, q):
    try:
        os.environ["MASTER_ADDR"] = "127.0.0.1"
        os.environ["MASTER_PORT"] = str(port)
        import sys
        sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
        import oracle
        from paper_2502_00778_gb300 import sharding
        dist.init_process_group("gloo", rank=rank, world_size=world)
        m, t = _grid_topology()
        ranges = sharding.element_ranges(m.n_elems, world)
        iface = sharding.interface_targets(3, m.elems, t.elem2edge, t.bface, t.bowner, t.bnode, ranges)
        lo, hi = ranges[rank]
        sub = oracle.Topology(3, t.edges, t.elem2edge[lo:hi], t.bface[sharding.owned_boundary_faces(t.bowner, lo, hi)],
                              None, t.bnode)
        n, v, b = oracle.direct(3, m.x, m.elems[lo:hi], sub)
        parts = [torch.from_numpy(np.ascontiguousarray(a)) for a in (n, v, b)] + [None]
        sent = sharding.exchange_interface(parts, iface)
        assert sent == 3 * len(iface["edges"]) + len(iface["nodes"]) + 3 * len(iface["bnodes"])
        assert sent < 0.6 * (n.size + v.size + b.size)
        rn, rv, rb = oracle.direct(3, m.x, m.elems, t)
        te, tv, tb = iface["touched"][rank]
        h = m.h
        assert np.abs(parts[0].numpy()[te] - rn[te]).max() <= 1e-13 * h * h
        assert np.abs(parts[1].numpy()[tv] - rv[tv]).max() <= 1e-13 * h ** 3
        assert np.abs(parts[2].numpy()[tb] - rb[tb]).max() <= 1e-13 * h * h
        # interface targets are final on every rank; what only others touch stays 0
        assert np.abs(parts[0].numpy()[iface["edges"]] - rn[iface["edges"]]).max() <= 1e-13 * h * h
        others = np.setdiff1d(np.arange(len(t.edges)), np.union1d(te, iface["edges"]))
        assert np.all(parts[0].numpy()[others] == 0.0)
        dist.destroy_process_group()
        q.put((rank, "ok"))
    except Exception as ex:  # report to the parent
        q.put((rank, repr(ex)))


def test_interface_exchange_three_ranks_gloo():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_interface_worker, args=(r, 3, port, q)) for r in range(3)]
    for p in procs:
        p.start()
    res = [q.get(timeout=240) for _ in procs]
    for p in procs:
        p.join(timeout=60)
    assert sorted(res) == [(0, "ok"), (1, "ok"), (2, "ok")], res

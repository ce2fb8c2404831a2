"""Multi-rank logic on CPU (gloo, world size 2): batch sharding and the
single-grid element partition with its one interface exchange (all-reduce of
partial sums), checked against the unpartitioned result.  The per-rank
compute here is the oracle: what is tested is the partition / exchange logic."""
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

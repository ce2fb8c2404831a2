"""How the work shards over several GPUs (one process per GPU).

Two units shard naturally, and neither needs a collective on the data path
except the one exchange of a partitioned grid:

* a batch of independent grids (deforming-mesh or adaptation sequences):
  each rank takes a subset of the grids, balanced by element count with the
  longest-processing-time rule (largest grid first, onto the least loaded
  rank); ranks run em_batched_fwd_adj on their own subsets;
* one large grid: each rank takes a contiguous range of elements (a Morton
  range when the elements are Morton ordered), computes the contributions of
  its elements to the global edge / node arrays, and the partial arrays are
  summed once over all ranks: either whole (one all-reduce per array, every
  rank ends with every value) or over the interface only (the entries of the
  edges and nodes that more than one range touches, packed into one buffer
  and all-reduced; every rank ends with the values of the targets its range
  touches).  The metrics are sums of per-element terms (plus per-boundary-face
  terms assigned to the rank of the face's owner element), so the summed
  partials equal the single-GPU result up to rounding order.
"""
from __future__ import annotations

import heapq


def shard_grids(sizes, world_size):
    """Assign grids (by element count) to ranks: returns a list of index lists,
    one per rank, every grid exactly once, each list in ascending order."""
    if world_size < 1:
        raise ValueError("world_size must be >= 1")
    heap = [(0, r) for r in range(world_size)]
    out = [[] for _ in range(world_size)]
    for i in sorted(range(len(sizes)), key=lambda k: (-sizes[k], k)):
        load, r = heapq.heappop(heap)
        out[r].append(i)
        heapq.heappush(heap, (load + sizes[i], r))
    return [sorted(o) for o in out]


def element_ranges(n_elems, world_size):
    """Contiguous element ranges [lo, hi) per rank, sizes differing by <= 1."""
    base, extra = divmod(n_elems, world_size)
    out, lo = [], 0
    for r in range(world_size):
        hi = lo + base + (1 if r < extra else 0)
        out.append((lo, hi))
        lo = hi
    return out


def owned_boundary_faces(bface_owner, lo, hi):
    """Boundary faces whose owner element lies in [lo, hi)."""
    import numpy as np
    e = np.asarray(bface_owner) // 4
    return np.nonzero((e >= lo) & (e < hi))[0]


def interface_targets(dim, elems, elem2edge, bface, bface_owner, bnode, ranges):
    """The targets of a partitioned grid that more than one element range
    touches, and the targets each range touches (host-side numpy, once per
    partition; every rank derives the same sets from the same arrays).

    A range touches the edges and the nodes of its elements (n; V and the
    gradient) and the boundary nodes of the boundary faces its elements own
    (bnormal); a face's edges and nodes are its owner element's, so its
    contributions to n and the gradient land on targets of the range too.
    Returns {"edges", "nodes", "bnodes"}: ascending interface ids (boundary
    nodes as positions in `bnode`), and "touched": per range, the same three
    id arrays."""
    import numpy as np
    elems = np.asarray(elems)
    e2e = np.asarray(elem2edge)
    bface = np.asarray(bface).reshape(-1, dim)
    own = np.asarray(bface_owner).astype(np.int64) // 4
    bnode = np.asarray(bnode).astype(np.int64)
    pos = np.full(int(bnode.max()) + 1 if bnode.size else 0, -1, np.int64)
    pos[bnode] = np.arange(bnode.size)
    touched = []
    for lo, hi in ranges:
        te = np.unique(e2e[lo:hi].ravel()).astype(np.int64)
        tv = np.unique(elems[lo:hi, :dim + 1].ravel()).astype(np.int64)
        faces = np.nonzero((own >= lo) & (own < hi))[0]
        tb = np.unique(pos[bface[faces].ravel()]) if faces.size else np.zeros(0, np.int64)
        touched.append((te, tv, tb))

    def shared(k):
        if not touched:
            return np.zeros(0, np.int64)
        ids, count = np.unique(np.concatenate([t[k] for t in touched]), return_counts=True)
        return ids[count > 1]

    return {"edges": shared(0), "nodes": shared(1), "bnodes": shared(2), "touched": touched}


def exchange_interface(parts, iface, group=None):
    """The one exchange of a partitioned grid over its interface: the partial
    (n, V, bnormal, grad) entries of the interface targets (`iface` from
    interface_targets) are packed into one buffer, summed over the ranks of
    `group` with one all-reduce, and written back in place.  Afterwards every
    rank holds the final value of each target its range touches and of each
    interface target; entries that only other ranks touch stay as they were
    (0).  Every rank must pass the same kinds of arrays (None where a kind is
    not computed).  Without an initialised process group nothing is summed.
    Returns the number of values exchanged."""
    import torch
    import torch.distributed as dist
    n, v, b, g = (list(parts) + [None] * 4)[:4]
    sel = []
    for a, key in ((n, "edges"), (v, "nodes"), (b, "bnodes"), (g, "nodes")):
        if a is not None and len(iface[key]):
            sel.append((a, torch.as_tensor(iface[key], dtype=torch.long, device=a.device)))
    if not sel:
        return 0
    buf = torch.cat([a.index_select(0, i).reshape(-1) for a, i in sel])
    if dist.is_available() and dist.is_initialized():
        if dist.get_backend(group) == "gloo" and buf.is_cuda:   # gloo reduces host copies
            t = buf.cpu()
            dist.all_reduce(t, group=group)
            buf.copy_(t)
        else:
            dist.all_reduce(buf, group=group)
    off = 0
    for a, i in sel:
        k = i.numel() * (a[0].numel() if a.dim() > 1 else 1)
        a.index_copy_(0, i, buf[off:off + k].view((i.numel(),) + tuple(a.shape[1:])))
        off += k
    return buf.numel()


def reduce_partials(parts, group=None):
    """Sum one rank's partial metric arrays (from api.edge_metrics_partial)
    over all ranks of `group` in place: the one exchange step of a partitioned
    grid.  Without an initialised process group (one process holding every
    range) it returns the arrays unchanged.  None entries are skipped."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return parts
    gloo = dist.get_backend(group) == "gloo"
    for a in parts:
        if a is None:
            continue
        if gloo and a.is_cuda:   # gloo reduces host copies
            t = a.cpu()
            dist.all_reduce(t, group=group)
            a.copy_(t)
        else:
            dist.all_reduce(a, group=group)
    return parts


def partitioned_metrics(topo, x, w=None, c=None, precision="fp64", rank=None, world_size=None, group=None,
                        exchange="all", iface=None):
    """The metrics of one grid computed by `world_size` ranks, each on its
    contiguous element range (this rank's range through the CUDA kernels),
    summed over the ranks: equals the single-rank result up to rounding
    order.  rank / world_size default to the process group's.

    exchange="all" sums the whole arrays (every rank ends with every value);
    exchange="interface" sums only the interface entries (exchange_interface;
    every rank ends with the values of the targets its range touches).
    `iface` (from interface_targets on this partition) is derived from the
    topology's arrays when not given."""
    from . import api
    import torch.distributed as dist
    if rank is None or world_size is None:
        if dist.is_available() and dist.is_initialized():
            rank, world_size = dist.get_rank(group), dist.get_world_size(group)
        else:
            rank, world_size = 0, 1
    ranges = element_ranges(topo.n_elems, world_size)
    lo, hi = ranges[rank]
    parts = api.edge_metrics_partial(topo, x, (lo, hi), w, c, precision)
    if exchange == "all":
        return reduce_partials(parts, group)
    if exchange != "interface":
        raise ValueError("exchange must be 'all' or 'interface'")
    if iface is None:
        host = lambda t: t.cpu().numpy()  # noqa: E731
        iface = interface_targets(topo.dim, host(topo.elems), host(topo.elem2edge), host(topo.bface),
                                  host(topo.bface_owner), host(topo.bnode), ranges)
    exchange_interface(parts, iface, group)
    return parts


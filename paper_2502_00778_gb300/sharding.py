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
  summed once over all ranks (all-reduce, or reduce-scatter onto the owner
  of each edge / node).  The metrics are sums of per-element terms (plus
  per-boundary-face terms assigned to the rank of the face's owner element),
  so the summed partials equal the single-GPU result up to rounding order.
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


def partitioned_metrics(topo, x, w=None, c=None, precision="fp64", rank=None, world_size=None, group=None):
    """The metrics of one grid computed by `world_size` ranks, each on its
    contiguous element range (this rank's range through the CUDA kernels),
    summed over the ranks: equals the single-rank result up to rounding
    order.  rank / world_size default to the process group's."""
    from . import api
    import torch.distributed as dist
    if rank is None or world_size is None:
        if dist.is_available() and dist.is_initialized():
            rank, world_size = dist.get_rank(group), dist.get_world_size(group)
        else:
            rank, world_size = 0, 1
    lo, hi = element_ranges(topo.n_elems, world_size)[rank]
    parts = api.edge_metrics_partial(topo, x, (lo, hi), w, c, precision)
    return reduce_partials(parts, group)


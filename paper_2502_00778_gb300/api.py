"""Python binding of the edge-metrics library: argument marshalling only.

PyTorch provides device memory and the current CUDA stream; every step of
the computation runs in the library's CUDA kernels.  Tensors passed in must
live on the GPU; nothing here falls back to a CPU implementation.
"""
from __future__ import annotations

import ctypes

import torch

from . import _lib
from ._lib import EmMesh, PATH, PREC, check, load

__all__ = ["Topology", "edge_build", "plan_build", "edge_metrics", "edge_metrics_adjoint", "edge_metrics_fused",
           "check_elements", "EdgeMetrics", "workspace"]


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


class _Workspace:
    """Grow-only device workspace shared by calls on one device."""

    def __init__(self):
        self.buf = {}

    def get(self, nbytes, device):
        key = str(device)
        b = self.buf.get(key)
        if b is None or b.numel() < nbytes:
            b = torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)
            self.buf[key] = b
        return b


workspace = _Workspace()


def _require_cuda(*ts):
    for t in ts:
        if t is not None and not t.is_cuda:
            raise ValueError("edge-metrics tensors must be CUDA tensors")


def _check_sizes(topo, **named):
    """Host-side checks before any launch.  The library reads and writes its
    arrays through plain pointers, so a tensor with the wrong number of
    elements would make a kernel access memory outside it; a tensor whose
    memory the library uses as is (an output written in place, or a batched
    input whose address is kept) must be contiguous float64; and every tensor
    must live on the grid's device.  `named` maps a name to (tensor or None,
    the number of elements the grid needs, whether its memory is used as is)."""
    dev = topo.elems.device
    for name, (t, count, as_is) in named.items():
        if t is None:
            continue
        if t.numel() != count:
            raise ValueError(f"{name} has {t.numel()} elements; this grid needs {count}")
        if as_is and (t.dtype != torch.float64 or not t.is_contiguous()):
            raise ValueError(f"{name} must be a contiguous float64 tensor: the library uses its memory as is")
        if t.device != dev:
            raise ValueError(f"{name} is on {t.device}; the grid's arrays are on {dev}")


class Topology:
    """Integer topology from em_edge_build (+ optional gather plan)."""

    def __init__(self, dim, elems, edges, elem2edge, edge_ptr, edge_slot, bface, bface_owner, bnode, n_nodes):
        self.dim = dim
        self.n_nodes = n_nodes
        self.elems = elems
        self.edges = edges
        self.elem2edge = elem2edge
        self.edge_ptr = edge_ptr
        self.edge_slot = edge_slot
        self.bface = bface
        self.bface_owner = bface_owner
        self.bnode = bnode
        self.plan = None
        self.plan_info = None
        self.tile_nodes = None

    @property
    def n_elems(self):
        return self.elems.shape[0]

    @property
    def n_edges(self):
        return self.edges.shape[0]

    @property
    def n_bfaces(self):
        return self.bface.shape[0]

    @property
    def n_bnodes(self):
        return self.bnode.shape[0]

    def em_mesh(self) -> EmMesh:
        m = EmMesh()
        m.dim = self.dim
        m.n_nodes, m.n_elems, m.n_edges = self.n_nodes, self.n_elems, self.n_edges
        m.n_bfaces, m.n_bnodes = self.n_bfaces, self.n_bnodes
        m.elems = self.elems.data_ptr()
        m.elem2edge = self.elem2edge.data_ptr()
        m.edges = self.edges.data_ptr()
        m.edge_ptr = self.edge_ptr.data_ptr() if self.edge_ptr is not None else None
        m.edge_slot = self.edge_slot.data_ptr() if self.edge_slot is not None else None
        m.bface = self.bface.data_ptr() if self.n_bfaces else None
        m.bface_owner = self.bface_owner.data_ptr() if self.n_bfaces else None
        m.bnode = self.bnode.data_ptr() if self.n_bnodes else None
        m.plan = self.plan.data_ptr() if self.plan is not None else None
        m.plan_bytes = self.plan.numel() if self.plan is not None else 0
        if self.plan_info is not None:
            for i, v in enumerate(self.plan_info):
                m.plan_info[i] = v
        return m


def edge_build(elems: torch.Tensor, x: torch.Tensor, csr: bool = True) -> Topology:
    """Edges, element->edge map, CSR, boundary faces and nodes (bit-exact)."""
    L = load()
    _require_cuda(elems, x)
    elems = elems.contiguous().to(torch.int32)
    x = x.contiguous().to(torch.float64)
    ne = elems.shape[0]
    nv, dim = x.shape
    nle = 6 if dim == 3 else 3
    dev = elems.device
    wsb = ctypes.c_size_t(0)
    counts = (ctypes.c_int64 * 3)()
    null = ctypes.c_void_p(0)
    check(L.em_edge_build(dim, nv, ne, _ptr(elems), _ptr(x), null, ctypes.byref(wsb), null, 0, null, null, null, null,
                          null, 0, null, 0, counts, _stream()))
    ws = workspace.get(wsb.value, dev)
    cap_e = nle * ne
    cap_b = (dim + 1) * ne
    edges = torch.empty((cap_e, 2), dtype=torch.int32, device=dev)
    e2e = torch.empty((ne, nle), dtype=torch.int32, device=dev)
    eptr = torch.empty(cap_e + 1, dtype=torch.int32, device=dev) if csr else None
    eslot = torch.empty(nle * ne, dtype=torch.int32, device=dev) if csr else None
    bface = torch.empty((cap_b, dim), dtype=torch.int32, device=dev)
    bown = torch.empty(cap_b, dtype=torch.int32, device=dev)
    bnode = torch.empty(nv, dtype=torch.int32, device=dev)
    check(L.em_edge_build(dim, nv, ne, _ptr(elems), _ptr(x), _ptr(ws), ctypes.byref(wsb), _ptr(edges), cap_e,
                          _ptr(e2e), _ptr(eptr), _ptr(eslot), _ptr(bface), _ptr(bown), cap_b, _ptr(bnode), nv,
                          counts, _stream()))
    n_e, n_b, n_bn = counts[0], counts[1], counts[2]
    topo = Topology(dim, elems, edges[:n_e].clone(), e2e, eptr[:n_e + 1].clone() if csr else None, eslot,
                    bface[:n_b].clone(), bown[:n_b].clone(), bnode[:n_bn].clone(), nv)
    return topo


def plan_build(topo: Topology, tile_nodes: int = 0) -> Topology:
    """Build the tiled gather plan (EM_PATH_GATHER) into topo.plan."""
    L = load()
    dev = topo.elems.device
    wsb = ctypes.c_size_t(0)
    pb = ctypes.c_size_t(0)
    null = ctypes.c_void_p(0)
    args = (topo.dim, topo.n_nodes, topo.n_elems, _ptr(topo.elems), _ptr(topo.elem2edge), topo.n_edges,
            _ptr(topo.edges), topo.n_bfaces, _ptr(topo.bface) if topo.n_bfaces else null,
            _ptr(topo.bface_owner) if topo.n_bfaces else null, topo.n_bnodes,
            _ptr(topo.bnode) if topo.n_bnodes else null, int(tile_nodes))
    info = (ctypes.c_int64 * _lib.PLAN_INFO_LEN)()
    # 1: scratch for the count pass; 2: exact plan and scratch sizes; 3: build
    check(L.em_plan_build(*args, null, ctypes.byref(wsb), null, ctypes.byref(pb), info, _stream()))
    ws = workspace.get(wsb.value, dev)
    check(L.em_plan_build(*args, _ptr(ws), ctypes.byref(wsb), null, ctypes.byref(pb), info, _stream()))
    ws = workspace.get(wsb.value, dev)
    plan = torch.empty(max(pb.value, 256), dtype=torch.uint8, device=dev)
    check(L.em_plan_build(*args, _ptr(ws), ctypes.byref(wsb), _ptr(plan), ctypes.byref(pb), info, _stream()))
    topo.plan = plan
    topo.plan_info = list(info)
    topo.tile_nodes = info[0]
    return topo


def plan_tiles(topo: Topology) -> int:
    n = ctypes.c_int64(0)
    check(load().em_plan_tiles(_ptr(topo.plan), ctypes.byref(n), _stream()))
    return n.value


def _mesh_ref(topo):
    m = topo.em_mesh()
    return m, ctypes.byref(m)


def edge_metrics(topo: Topology, x: torch.Tensor, precision: str = "fp64", path: str = "atomic", out=None):
    """Forward: (n_edge [Ne,dim], vol [Nv], bnormal [Nbn,dim]) as float64 CUDA tensors."""
    L = load()
    d = topo.dim
    n0, v0, b0 = out if out is not None else (None, None, None)
    _check_sizes(topo, x=(x, topo.n_nodes * d, False), n_edge=(n0, topo.n_edges * d, True),
                 vol=(v0, topo.n_nodes, True), bnormal=(b0, topo.n_bnodes * d, True))
    _require_cuda(x)
    x = x.contiguous().to(torch.float64)
    dim, dev = topo.dim, x.device
    if out is None:
        n = torch.empty((topo.n_edges, dim), dtype=torch.float64, device=dev)
        v = torch.empty(topo.n_nodes, dtype=torch.float64, device=dev)
        b = torch.empty((topo.n_bnodes, dim), dtype=torch.float64, device=dev)
    else:
        n, v, b = out
    m, mr = _mesh_ref(topo)
    wsb = ctypes.c_size_t(0)
    null = ctypes.c_void_p(0)
    pr, pa = PREC[precision], PATH[path]
    check(L.em_edge_metrics(mr, pr, pa, _ptr(x), _ptr(n), _ptr(v), _ptr(b), null, ctypes.byref(wsb), _stream()))
    ws = workspace.get(wsb.value, dev)
    check(L.em_edge_metrics(mr, pr, pa, _ptr(x), _ptr(n), _ptr(v), _ptr(b), _ptr(ws), ctypes.byref(wsb), _stream()))
    return n, v, b


def edge_metrics_adjoint(topo: Topology, x, w, c=None, precision: str = "fp64", path: str = "atomic", out=None,
                         bw=None):
    """grad_x = d/dx (sum w.n + sum c V + sum bw.bnormal), float64 [Nv, dim];
    bw (boundary-normal weights, [n_bnodes, dim] in topo.bnode order) is
    optional and supported on the atomic and tiled paths."""
    L = load()
    d = topo.dim
    _check_sizes(topo, x=(x, topo.n_nodes * d, False), w=(w, topo.n_edges * d, False), c=(c, topo.n_nodes, False),
                 bw=(bw, topo.n_bnodes * d, False), grad=(out, topo.n_nodes * d, True))
    _require_cuda(x, w, c, bw)
    x = x.contiguous().to(torch.float64)
    w = w.contiguous().to(torch.float64)
    c = c.contiguous().to(torch.float64) if c is not None else None
    bw = bw.contiguous().to(torch.float64) if bw is not None else None
    g = out if out is not None else torch.empty((topo.n_nodes, topo.dim), dtype=torch.float64, device=x.device)
    m, mr = _mesh_ref(topo)
    wsb = ctypes.c_size_t(0)
    null = ctypes.c_void_p(0)
    pr, pa = PREC[precision], PATH[path]
    check(L.em_edge_metrics_adjoint(mr, pr, pa, _ptr(x), _ptr(w), _ptr(c), _ptr(bw), _ptr(g), null,
                                    ctypes.byref(wsb), _stream()))
    ws = workspace.get(wsb.value, x.device)
    check(L.em_edge_metrics_adjoint(mr, pr, pa, _ptr(x), _ptr(w), _ptr(c), _ptr(bw), _ptr(g), _ptr(ws),
                                    ctypes.byref(wsb), _stream()))
    return g


def edge_metrics_fused(topo: Topology, x, w, c=None, precision: str = "fp64", out=None, path: str = "gather",
                       bw=None):
    """Forward outputs and the adjoint in one pass (plan required; path
    "gather" = deterministic ordered gather, "tiled" = shared-memory scatter;
    bw as in edge_metrics_adjoint, tiled path only)."""
    L = load()
    d = topo.dim
    n0, v0, b0, g0 = out if out is not None else (None, None, None, None)
    _check_sizes(topo, x=(x, topo.n_nodes * d, False), w=(w, topo.n_edges * d, False), c=(c, topo.n_nodes, False),
                 bw=(bw, topo.n_bnodes * d, False), n_edge=(n0, topo.n_edges * d, True),
                 vol=(v0, topo.n_nodes, True), bnormal=(b0, topo.n_bnodes * d, True),
                 grad=(g0, topo.n_nodes * d, True))
    _require_cuda(x, w, c, bw)
    x = x.contiguous().to(torch.float64)
    w = w.contiguous().to(torch.float64)
    c = c.contiguous().to(torch.float64) if c is not None else None
    bw = bw.contiguous().to(torch.float64) if bw is not None else None
    dim, dev = topo.dim, x.device
    if out is None:
        n = torch.empty((topo.n_edges, dim), dtype=torch.float64, device=dev)
        v = torch.empty(topo.n_nodes, dtype=torch.float64, device=dev)
        b = torch.empty((topo.n_bnodes, dim), dtype=torch.float64, device=dev)
        g = torch.empty((topo.n_nodes, dim), dtype=torch.float64, device=dev)
    else:
        n, v, b, g = out
    m, mr = _mesh_ref(topo)
    wsb = ctypes.c_size_t(0)
    null = ctypes.c_void_p(0)
    pr, pa = PREC[precision], PATH[path]
    args = (_ptr(x), _ptr(w), _ptr(c), _ptr(bw), _ptr(n), _ptr(v), _ptr(b), _ptr(g))
    check(L.em_edge_metrics_fused(mr, pr, pa, *args, null, ctypes.byref(wsb), _stream()))
    ws = workspace.get(wsb.value, dev)
    check(L.em_edge_metrics_fused(mr, pr, pa, *args, _ptr(ws), ctypes.byref(wsb), _stream()))
    return n, v, b, g


def edge_metrics_partial(topo: Topology, x, elem_range, w=None, c=None, precision: str = "fp64", forward=True):
    """One rank's share of a grid split into element ranges: the
    contributions of elements [lo, hi) (and of the boundary faces they own)
    to the global n [Ne, dim], V [Nv], bnormal [Nbn, dim] and, when w is
    given, dL/dx [Nv, dim].  Returns (n, V, bnormal, grad), None for what was
    not asked for.  Summing the tuples of ranges that cover the grid gives the
    full result up to rounding order (sharding.reduce_partials)."""
    L = load()
    d = topo.dim
    _check_sizes(topo, x=(x, topo.n_nodes * d, False), w=(w, topo.n_edges * d, False), c=(c, topo.n_nodes, False))
    _require_cuda(x, w, c)
    lo, hi = (int(v) for v in elem_range)
    x = x.contiguous().to(torch.float64)
    w = w.contiguous().to(torch.float64) if w is not None else None
    c = c.contiguous().to(torch.float64) if c is not None else None
    dev = x.device
    n = v = b = g = None
    if forward:
        n = torch.empty((topo.n_edges, topo.dim), dtype=torch.float64, device=dev)
        v = torch.empty(topo.n_nodes, dtype=torch.float64, device=dev)
        b = torch.empty((topo.n_bnodes, topo.dim), dtype=torch.float64, device=dev)
    if w is not None:
        g = torch.empty((topo.n_nodes, topo.dim), dtype=torch.float64, device=dev)
    m, mr = _mesh_ref(topo)
    check(L.em_edge_metrics_partial(mr, PREC[precision], lo, hi, _ptr(x), _ptr(w), _ptr(c), _ptr(n), _ptr(v),
                                    _ptr(b), _ptr(g), _stream()))
    return n, v, b, g


def edge_volume(topo: Topology, x, n_edge):
    """Edge-based dual volume (Sec. 4.1) from lumped directed-area vectors."""
    L = load()
    _check_sizes(topo, x=(x, topo.n_nodes * topo.dim, False), n_edge=(n_edge, topo.n_edges * topo.dim, False))
    _require_cuda(x, n_edge)
    x = x.contiguous().to(torch.float64)
    n_edge = n_edge.contiguous().to(torch.float64)
    v = torch.empty(topo.n_nodes, dtype=torch.float64, device=x.device)
    m, mr = _mesh_ref(topo)
    wsb = ctypes.c_size_t(0)
    null = ctypes.c_void_p(0)
    check(L.em_edge_volume(mr, _ptr(x), _ptr(n_edge), _ptr(v), null, ctypes.byref(wsb), _stream()))
    ws = workspace.get(wsb.value, x.device)
    check(L.em_edge_volume(mr, _ptr(x), _ptr(n_edge), _ptr(v), _ptr(ws), ctypes.byref(wsb), _stream()))
    return v


def edge_areas_traditional(topo: Topology, x, out=None):
    """n_jk by the traditional dual-face construction (Sec. 3.1), FP64 atomics."""
    L = load()
    _check_sizes(topo, x=(x, topo.n_nodes * topo.dim, False), n_edge=(out, topo.n_edges * topo.dim, True))
    _require_cuda(x)
    x = x.contiguous().to(torch.float64)
    n = out if out is not None else torch.empty((topo.n_edges, topo.dim), dtype=torch.float64, device=x.device)
    m, mr = _mesh_ref(topo)
    check(L.em_edge_areas_traditional(mr, _ptr(x), _ptr(n), _stream()))
    return n


def edge_residual(topo: Topology, F, n_edge, bnormal):
    """Edge-loop residual with central fluxes (Sec. 2) for nodal fluxes F."""
    L = load()
    d = topo.dim
    _check_sizes(topo, F=(F, topo.n_nodes * d, False), n_edge=(n_edge, topo.n_edges * d, False),
                 bnormal=(bnormal, topo.n_bnodes * d, False))
    _require_cuda(F, n_edge, bnormal)
    F = F.contiguous().to(torch.float64)
    n_edge = n_edge.contiguous().to(torch.float64)
    bnormal = bnormal.contiguous().to(torch.float64)
    res = torch.empty(topo.n_nodes, dtype=torch.float64, device=F.device)
    m, mr = _mesh_ref(topo)
    wsb = ctypes.c_size_t(0)
    null = ctypes.c_void_p(0)
    check(L.em_edge_residual(mr, _ptr(F), _ptr(n_edge), _ptr(bnormal), _ptr(res), null, ctypes.byref(wsb), _stream()))
    ws = workspace.get(wsb.value, F.device)
    check(L.em_edge_residual(mr, _ptr(F), _ptr(n_edge), _ptr(bnormal), _ptr(res), _ptr(ws), ctypes.byref(wsb),
                             _stream()))
    return res


def check_elements(dim: int, elems: torch.Tensor, x: torch.Tensor):
    """(bad-id count, degenerate count); raises EMError on either."""
    L = load()
    elems = elems.contiguous().to(torch.int32)
    x = x.contiguous().to(torch.float64)
    wsb = ctypes.c_size_t(0)
    counts = (ctypes.c_int64 * 2)()
    null = ctypes.c_void_p(0)
    check(L.em_check_elements(dim, x.shape[0], elems.shape[0], _ptr(elems), _ptr(x), null, ctypes.byref(wsb), counts,
                              _stream()))
    ws = workspace.get(wsb.value, elems.device)
    check(L.em_check_elements(dim, x.shape[0], elems.shape[0], _ptr(elems), _ptr(x), _ptr(ws), ctypes.byref(wsb),
                              counts, _stream()))
    return counts[0], counts[1]


class EdgeMetrics(torch.autograd.Function):
    """(n_edge, vol, bnormal) = EdgeMetrics.apply(x, topo, precision, path).

    backward calls the adjoint kernel with w = grad(n_edge), c = grad(vol)
    and bw = grad(bnormal) (the ordered-gather path takes its adjoint on the
    tiled path when bnormal carries a gradient)."""

    @staticmethod
    def forward(ctx, x, topo, precision="fp64", path="atomic"):
        ctx.topo, ctx.precision, ctx.path = topo, precision, path
        ctx.save_for_backward(x)
        ctx.set_materialize_grads(False)      # an unused output's gradient arrives as None
        n, v, b = edge_metrics(topo, x, precision, path)
        return n, v, b

    @staticmethod
    def backward(ctx, gn, gv, gb):
        (x,) = ctx.saved_tensors
        topo = ctx.topo
        if gn is None:
            gn = torch.zeros((topo.n_edges, topo.dim), dtype=torch.float64, device=x.device)
        adj_path = ctx.path if ctx.path in ("atomic", "gather", "tiled") else "atomic"
        if gb is not None and adj_path == "gather":
            adj_path = "tiled"
        g = edge_metrics_adjoint(topo, x, gn, gv, ctx.precision if ctx.precision != "mixed_comp32" else "mixed",
                                 adj_path, bw=gb)
        return g, None, None, None


class Batch:
    """Forward + adjoint of many grids of uneven size in one launch.

    All device-side descriptions (the em_batch_item array, the tile prefix
    sums, the outputs) are built once here and keep fixed addresses, so
    run() only enqueues the library call and a captured CUDA graph of run()
    can be replayed after the inputs (x, w, c) are updated in place.
    blocks: 0 one CTA per (grid, tile) item; > 0 that many persistent CTAs
    claiming items from a counter; -1 persistent, SMs x resident CTAs.
    """

    def __init__(self, topos, xs, ws, cs, precision: str = "dw", blocks: int = 0):
        L = load()
        if not topos:
            raise ValueError("empty batch")
        self.dim = topos[0].dim
        if any(t.dim != self.dim for t in topos):
            raise ValueError("all grids of a batch must have the same dimension")
        if any(t.plan is None for t in topos):
            raise ValueError("every grid needs a plan (plan_build)")
        if not (len(xs) == len(ws) == len(cs) == len(topos)):
            raise ValueError("one x, w and c per grid")
        dev = xs[0].device
        self.topos, self.xs, self.ws, self.cs = topos, xs, ws, cs
        self.precision = precision
        self.blocks = blocks
        self.outs = []
        self.recs = []
        items = (_lib.EmBatchItem * len(topos))()
        for i, (t, x, w, c) in enumerate(zip(topos, xs, ws, cs)):
            d = t.dim
            _check_sizes(t, **{f"xs[{i}]": (x, t.n_nodes * d, True), f"ws[{i}]": (w, t.n_edges * d, True),
                               f"cs[{i}]": (c, t.n_nodes, True)})
            o = (torch.empty((t.n_edges, d), dtype=torch.float64, device=dev),
                 torch.empty(t.n_nodes, dtype=torch.float64, device=dev),
                 torch.empty((t.n_bnodes, d), dtype=torch.float64, device=dev),
                 torch.empty((t.n_nodes, d), dtype=torch.float64, device=dev))
            self.outs.append(o)
            items[i].mesh = t.em_mesh()
            items[i].x, items[i].w = x.data_ptr(), w.data_ptr()
            items[i].c = c.data_ptr() if c is not None else None
            items[i].n_edge, items[i].vol = o[0].data_ptr(), o[1].data_ptr()
            items[i].bnormal, items[i].grad_x = o[2].data_ptr(), o[3].data_ptr()
            # this grid's tile records (scatter tiles), 32 bytes each
            nrec = sum(t.plan_info[_lib.PLAN_INFO[k]] for k in ("rec_edges", "rec_nodes", "rec_bnodes"))
            r = torch.empty(max(32 * nrec, 256), dtype=torch.uint8, device=dev)
            self.recs.append(r)
            items[i].rec = r.data_ptr()
        raw = bytes(items)
        self.items = torch.frombuffer(bytearray(raw), dtype=torch.uint8).to(dev)
        tiles = [t.plan_info[1] for t in topos]
        prefix = [0]
        for n in tiles:
            prefix.append(prefix[-1] + n)
        self.n_tiles = prefix[-1]
        self.prefix = torch.tensor(prefix, dtype=torch.int64, device=dev)
        self.max_info = (ctypes.c_int64 * _lib.PLAN_INFO_LEN)()
        for t in topos:
            for k, v in enumerate(t.plan_info):
                self.max_info[k] = max(self.max_info[k], v)
        self.status = torch.zeros(1, dtype=torch.int32, device=dev)
        wsb = ctypes.c_size_t(0)
        check(L.em_batched_fwd_adj(len(topos), None, None, self.n_tiles, self.max_info, self.dim, PREC[precision],
                                   blocks, None, None, ctypes.byref(wsb), _stream()))
        self.wsb = wsb.value
        self.wsbuf = torch.empty(max(self.wsb, 256), dtype=torch.uint8, device=dev)

    def run(self):
        """Enqueue the batched launch on the current stream."""
        wsb = ctypes.c_size_t(self.wsbuf.numel())
        check(load().em_batched_fwd_adj(len(self.topos), _ptr(self.items), _ptr(self.prefix), self.n_tiles,
                                        self.max_info, self.dim, PREC[self.precision], self.blocks, _ptr(self.status),
                                        _ptr(self.wsbuf), ctypes.byref(wsb), _stream()))

    def capture(self):
        """A CUDA graph of run(); replay() it after updating the inputs in place."""
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self.run()
        torch.cuda.current_stream().wait_stream(s)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.run()
        return g

    def check_status(self):
        st = int(self.status.item())
        if st != 0:
            raise _lib.EMError(st, "batched launch reported an item error")

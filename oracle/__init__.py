"""CPU oracle for the edge-based grid metrics (arXiv 2502.00778).

TEST INFRASTRUCTURE ONLY: a plain, serial, double-precision C implementation
written from the paper, loaded through ctypes.  Only the test-suite,
``__graft_entry__.smoke()`` and the benchmark's CPU-baseline / reference arm
may import this package; the GPU product path never does, and the two share
no code.  See ``oracle.c`` for the functions, the equations each follows and
the readings taken where the paper leaves a choice open.

Every function takes and returns numpy arrays:
  x      float64 [n_nodes, dim]
  elems  int32   [n_elems, 4]   (triangles: column 3 is -1)
"""
import ctypes
import os
import threading

import numpy as np

from . import build as _build

_lock = threading.Lock()
_lib = None

_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_f64p = ctypes.POINTER(ctypes.c_double)
_i64 = ctypes.c_int64


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            L = ctypes.CDLL(path)
            L.or_edges.restype = _i64
            L.or_edges.argtypes = [ctypes.c_int, _i64, _i32p, _i64, _i32p, _i32p]
            L.or_bfaces.restype = _i64
            L.or_bfaces.argtypes = [ctypes.c_int, _i64, _i32p, _f64p, _i64, _i32p, _i32p]
            L.or_bnodes.restype = _i64
            L.or_bnodes.argtypes = [ctypes.c_int, _i64, _i64, _i32p, _i32p]
            L.or_direct.restype = None
            L.or_direct.argtypes = [ctypes.c_int, _i64, _f64p, _i64, _i32p, _i32p, _i64, _i32p, _i64, _i32p,
                                    _f64p, _f64p, _f64p]
            L.or_traditional.restype = None
            L.or_traditional.argtypes = [ctypes.c_int, _i64, _f64p, _i64, _i32p, _i32p, _i64, _f64p]
            L.or_edge_volume.restype = None
            L.or_edge_volume.argtypes = [ctypes.c_int, _i64, _f64p, _i64, _i32p, _f64p, _f64p]
            L.or_edge_residual.restype = None
            L.or_edge_residual.argtypes = [ctypes.c_int, _i64, _i64, _i32p, _f64p, _f64p, _i64, _i32p, _f64p, _f64p]
            L.or_closure.restype = None
            L.or_closure.argtypes = [ctypes.c_int, _i64, _f64p, _i64, _i32p, _f64p, _i64, _i32p, _f64p]
            L.or_adjoint.restype = None
            L.or_adjoint.argtypes = [ctypes.c_int, _i64, _f64p, _i64, _i32p, _i32p, _i64, _i32p, _i64, _i32p,
                                     _f64p, _f64p, _f64p, _f64p]
            L.or_loss_subset.restype = ctypes.c_double
            L.or_loss_subset.argtypes = [ctypes.c_int, _f64p, _i32p, _i32p, _i64, _i64p, _i64, _i32p, _i32p,
                                         _i64, _i64p, _f64p, _f64p, _f64p]
            L.or_fd_gradient.restype = None
            L.or_fd_gradient.argtypes = [ctypes.c_int, _i64, _f64p, _i64, _i32p, _i32p, _i64, _i32p, _i64, _i32p,
                                         _f64p, _f64p, _f64p, _i64, _i64p, ctypes.c_double, _f64p]
            L.or_sample.restype = None
            L.or_sample.argtypes = [ctypes.c_int, _i64, _f64p, _i64, _i32p, _i64, _i32p, _i32p, _f64p, _i64, _i32p,
                                    _f64p, _f64p, ctypes.c_uint64, _f64p]
            _lib = L
    return _lib


def _p(a, t):
    return a.ctypes.data_as(t)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def nloc(dim):
    return 6 if dim == 3 else 3


class Topology:
    """Oracle-side topology: edges, element->edge map, boundary faces and nodes."""

    def __init__(self, dim, edges, elem2edge, bface, bowner, bnode):
        self.dim = dim
        self.edges = edges
        self.elem2edge = elem2edge
        self.bface = bface
        self.bowner = bowner
        self.bnode = bnode

    @property
    def n_edges(self):
        return self.edges.shape[0]


def edges(dim, elems):
    elems = _c(elems, np.int32)
    ne = elems.shape[0]
    nl = nloc(dim)
    cap = ne * nl
    e = np.empty((max(cap, 1), 2), np.int32)
    e2e = np.empty((ne, nl), np.int32)
    m = lib().or_edges(dim, ne, _p(elems, _i32p), cap, _p(e, _i32p), _p(e2e, _i32p))
    assert m >= 0
    return e[:m].copy(), e2e


def bfaces(dim, elems, x):
    elems = _c(elems, np.int32)
    x = _c(x, np.float64)
    ne = elems.shape[0]
    cap = ne * (dim + 1)
    bf = np.empty((max(cap, 1), dim), np.int32)
    bo = np.empty(max(cap, 1), np.int32)
    m = lib().or_bfaces(dim, ne, _p(elems, _i32p), _p(x, _f64p), cap, _p(bf, _i32p), _p(bo, _i32p))
    assert m >= 0
    return bf[:m].copy(), bo[:m].copy()


def bnodes(dim, n_nodes, bface):
    bface = _c(bface, np.int32)
    out = np.empty(max(n_nodes, 1), np.int32)
    m = lib().or_bnodes(dim, n_nodes, bface.shape[0], _p(bface, _i32p), _p(out, _i32p))
    return out[:m].copy()


def topology(dim, elems, x):
    e, e2e = edges(dim, elems)
    bf, bo = bfaces(dim, elems, x)
    bn = bnodes(dim, x.shape[0], bf)
    return Topology(dim, e, e2e, bf, bo, bn)


def direct(dim, x, elems, topo):
    """Proposed algorithm: returns (n_edge [Ne,dim], vol [Nv], bnormal [Nbn,dim])."""
    x = _c(x, np.float64)
    elems = _c(elems, np.int32)
    nv = x.shape[0]
    n = np.empty((topo.n_edges, dim))
    v = np.empty(nv)
    bfull = np.empty((nv, dim))
    lib().or_direct(dim, nv, _p(x, _f64p), elems.shape[0], _p(elems, _i32p), _p(topo.elem2edge, _i32p),
                    topo.n_edges, _p(topo.edges, _i32p), topo.bface.shape[0], _p(topo.bface, _i32p),
                    _p(n, _f64p), _p(v, _f64p), _p(bfull, _f64p))
    return n, v, bfull[topo.bnode.astype(np.int64)]


def traditional(dim, x, elems, topo):
    x = _c(x, np.float64)
    elems = _c(elems, np.int32)
    n = np.empty((topo.n_edges, dim))
    lib().or_traditional(dim, x.shape[0], _p(x, _f64p), elems.shape[0], _p(elems, _i32p),
                         _p(topo.elem2edge, _i32p), topo.n_edges, _p(n, _f64p))
    return n


def edge_volume(dim, x, topo, n_edge):
    x = _c(x, np.float64)
    n_edge = _c(n_edge, np.float64)
    v = np.empty(x.shape[0])
    lib().or_edge_volume(dim, x.shape[0], _p(x, _f64p), topo.n_edges, _p(topo.edges, _i32p), _p(n_edge, _f64p),
                         _p(v, _f64p))
    return v


def edge_residual(dim, topo, n_edge, F, bnormal):
    """Edge-loop residual with central fluxes (Sec. 2) and the boundary term
    F_j . bnormal_j; `bnormal` is [n_bnodes][dim] in topo.bnode order."""
    n_edge = _c(n_edge, np.float64)
    F = _c(F, np.float64)
    bnormal = _c(bnormal, np.float64)
    bn = _c(topo.bnode, np.int32)
    res = np.empty(F.shape[0])
    lib().or_edge_residual(dim, F.shape[0], topo.n_edges, _p(topo.edges, _i32p), _p(n_edge, _f64p), _p(F, _f64p),
                           bn.shape[0], _p(bn, _i32p), _p(bnormal, _f64p), _p(res, _f64p))
    return res


def closure(dim, x, topo, n_edge):
    x = _c(x, np.float64)
    n_edge = _c(n_edge, np.float64)
    a = np.empty((x.shape[0], dim))
    lib().or_closure(dim, x.shape[0], _p(x, _f64p), topo.n_edges, _p(topo.edges, _i32p), _p(n_edge, _f64p),
                     topo.bface.shape[0], _p(topo.bface, _i32p), _p(a, _f64p))
    return a


def _bw_node(topo, n_nodes, dim, bw):
    """Boundary-normal weights given per boundary node (topo.bnode order) as a
    per-node array, zero at interior nodes; None stays None."""
    if bw is None:
        return None
    out = np.zeros((n_nodes, dim))
    out[np.asarray(topo.bnode)] = np.asarray(bw, dtype=np.float64).reshape(-1, dim)
    return out


def adjoint(dim, x, elems, topo, w, c, bw=None):
    """dL/dx for L = sum_e w_e.n_e + sum_i c_i V_i (+ sum_b bw_b.bnormal_b)."""
    x = _c(x, np.float64)
    elems = _c(elems, np.int32)
    w = _c(w, np.float64)
    c = _c(c, np.float64)
    bn = _bw_node(topo, x.shape[0], dim, bw)
    g = np.empty((x.shape[0], dim))
    lib().or_adjoint(dim, x.shape[0], _p(x, _f64p), elems.shape[0], _p(elems, _i32p), _p(topo.elem2edge, _i32p),
                     topo.n_edges, _p(topo.edges, _i32p), topo.bface.shape[0], _p(topo.bface, _i32p),
                     _p(w, _f64p), _p(c, _f64p), None if bn is None else _p(bn, _f64p), _p(g, _f64p))
    return g


_lib_omp = None


def lib_omp():
    """The multi-core CPU baseline (oracle_omp.c): the oracle's element
    arithmetic with its loops split over OpenMP threads.  A timing baseline,
    not a parity reference (its summation order follows the thread
    schedule)."""
    global _lib_omp
    with _lock:
        if _lib_omp is None:
            L = ctypes.CDLL(_build.build_omp())
            L.or_fused_omp.restype = None
            L.or_fused_omp.argtypes = [ctypes.c_int, ctypes.c_int, _i64, _f64p, _i64, _i32p, _i32p, _i64, _i32p,
                                       _i64, _i32p, _f64p, _f64p, _f64p, _f64p, _f64p, _f64p]
            L.or_omp_max_threads.restype = ctypes.c_int
            L.or_omp_max_threads.argtypes = []
            _lib_omp = L
    return _lib_omp


def fused_omp(dim, x, elems, topo, w, c, threads=0):
    """Forward (n, V, bnormal) and dL/dx on `threads` cores (0: all the
    OpenMP runtime offers); returns (n, V, bnormal, grad)."""
    x = _c(x, np.float64)
    elems = _c(elems, np.int32)
    w = _c(w, np.float64)
    c = _c(c, np.float64)
    nv = x.shape[0]
    n = np.empty((topo.n_edges, dim))
    v = np.empty(nv)
    bfull = np.empty((nv, dim))
    g = np.empty((nv, dim))
    lib_omp().or_fused_omp(int(threads), dim, nv, _p(x, _f64p), elems.shape[0], _p(elems, _i32p),
                           _p(topo.elem2edge, _i32p), topo.n_edges, _p(topo.edges, _i32p), topo.bface.shape[0],
                           _p(topo.bface, _i32p), _p(w, _f64p), _p(c, _f64p), _p(n, _f64p), _p(v, _f64p),
                           _p(bfull, _f64p), _p(g, _f64p))
    return n, v, bfull[topo.bnode.astype(np.int64)], g


def omp_threads():
    return int(lib_omp().or_omp_max_threads())


def loss_subset(dim, x, elems, topo, sel, bsel, w, c, bw=None):
    x = _c(x, np.float64)
    elems = _c(elems, np.int32)
    sel = _c(sel, np.int64)
    bsel = _c(bsel, np.int64)
    w = _c(w, np.float64)
    c = _c(c, np.float64)
    bn = _bw_node(topo, x.shape[0], dim, bw)
    return lib().or_loss_subset(dim, _p(x, _f64p), _p(elems, _i32p), _p(topo.elem2edge, _i32p), sel.shape[0],
                                _p(sel, _i64p), topo.n_edges, _p(topo.edges, _i32p), _p(topo.bface, _i32p),
                                bsel.shape[0], _p(bsel, _i64p), _p(w, _f64p), _p(c, _f64p),
                                None if bn is None else _p(bn, _f64p))


def loss(dim, x, elems, topo, w, c, bw=None):
    return loss_subset(dim, x, elems, topo, np.arange(elems.shape[0]), np.arange(topo.bface.shape[0]), w, c, bw)


def fd_gradient(dim, x, elems, topo, w, c, nodes, delta, bw=None):
    x = np.array(x, dtype=np.float64, order="C", copy=True)
    elems = _c(elems, np.int32)
    w = _c(w, np.float64)
    c = _c(c, np.float64)
    nodes = _c(nodes, np.int64)
    bn = _bw_node(topo, x.shape[0], dim, bw)
    g = np.empty((nodes.shape[0], dim))
    lib().or_fd_gradient(dim, x.shape[0], _p(x, _f64p), elems.shape[0], _p(elems, _i32p), _p(topo.elem2edge, _i32p),
                         topo.n_edges, _p(topo.edges, _i32p), topo.bface.shape[0], _p(topo.bface, _i32p),
                         _p(w, _f64p), _p(c, _f64p), None if bn is None else _p(bn, _f64p), nodes.shape[0],
                         _p(nodes, _i64p), float(delta), _p(g, _f64p))
    return g


def sample(dim, x, elems, edge_j, edge_k, nodes, seed):
    """n at the sampled edges (j<k), and V, bnormal, dL/dx at the sampled
    nodes, each computed from the elements around it; L uses the counter-based
    weights w(j,k), c(v) (SplitMix64 of the node ids, see or_hash_w)."""
    x = _c(x, np.float64)
    elems = _c(elems, np.int32)
    ej = _c(edge_j, np.int32)
    ek = _c(edge_k, np.int32)
    nd = _c(nodes, np.int32)
    n = np.empty((ej.shape[0], dim))
    v = np.empty(nd.shape[0])
    b = np.empty((nd.shape[0], dim))
    g = np.empty((nd.shape[0], dim))
    lib().or_sample(dim, x.shape[0], _p(x, _f64p), elems.shape[0], _p(elems, _i32p), ej.shape[0], _p(ej, _i32p),
                    _p(ek, _i32p), _p(n, _f64p), nd.shape[0], _p(nd, _i32p), _p(v, _f64p), _p(b, _f64p),
                    ctypes.c_uint64(seed), _p(g, _f64p))
    return n, v, b, g

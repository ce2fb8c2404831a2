"""The C-ABI library loads and exports every function include/*.h declares;
argument errors are reported as status codes (no GPU needed for these)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^\s*(?:int|size_t|void)\s+(em_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__  # noqa: F401  (build helper lives at the repo root)
    from paper_2502_00778_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 10, names
    for n in names:
        assert hasattr(lib, n), f"{n} declared in include/ but not exported"


def test_version_and_error_paths(lib):
    import paper_2502_00778_gb300 as p
    L = p.load()
    assert L.em_version() == 200
    # NULL mesh -> EM_ERR_ARG, no device work
    st = L.em_edge_metrics(None, 0, 0, None, None, None, None, None, None, None)
    assert st == -1
    buf = ctypes.create_string_buffer(256)
    assert L.em_last_error(buf, 256) == -1
    assert b"mesh" in buf.value
    # unsupported dimension
    sz = ctypes.c_size_t(0)
    cnt = (ctypes.c_int64 * 3)()
    st = L.em_edge_build(4, 10, 10, None, None, None, ctypes.byref(sz), None, 0, None, None, None, None, None, 0,
                         None, 0, cnt, None)
    assert st == -1
    # bad path / precision pairs are rejected before any device work
    m = p._lib.EmMesh()
    m.dim, m.n_nodes, m.n_elems, m.n_edges = 3, 4, 1, 6
    m.elems = m.elem2edge = m.edges = 4096  # never dereferenced: validation fails first
    st = L.em_edge_metrics(ctypes.byref(m), 1, 0, None, None, None, None, None, ctypes.byref(sz), None)
    assert st == -1
    st = L.em_edge_metrics(ctypes.byref(m), 0, 1, None, None, None, None, None, ctypes.byref(sz), None)
    assert st == -1   # gather path without a plan
    st = L.em_edge_metrics(ctypes.byref(m), 0, 9, None, None, None, None, None, ctypes.byref(sz), None)
    assert st == -1


def test_workspace_queries_need_no_device(lib):
    import paper_2502_00778_gb300 as p
    L = p.load()
    sz = ctypes.c_size_t(0)
    cnt = (ctypes.c_int64 * 3)()
    st = L.em_edge_build(3, 1000, 5000, None, None, None, ctypes.byref(sz), None, 0, None, None, None, None, None, 0,
                         None, 0, cnt, None)
    assert st == 0 and sz.value > 5000 * 6 * 24


def test_newer_entry_points_reject_bad_arguments(lib):
    """Argument errors of the residual, traditional, adjoint-with-weights and
    batched entry points come back as EM_ERR_ARG with a message, before any
    device work."""
    import paper_2502_00778_gb300 as p
    L = p.load()
    buf = ctypes.create_string_buffer(256)
    sz = ctypes.c_size_t(0)
    assert L.em_edge_residual(None, None, None, None, None, None, ctypes.byref(sz), None) == -1
    L.em_last_error(buf, 256)
    assert b"mesh" in buf.value
    assert L.em_edge_areas_traditional(None, None, None, None) == -1
    m = p._lib.EmMesh()
    m.dim, m.n_nodes, m.n_elems, m.n_edges = 3, 4, 1, 6
    m.elems = m.elem2edge = m.edges = 4096   # never dereferenced: validation fails first
    assert L.em_edge_areas_traditional(ctypes.byref(m), None, None, None) == -1   # x and n_edge NULL
    m.plan = 4096
    fake = ctypes.c_void_p(4096)
    st = L.em_edge_metrics_adjoint(ctypes.byref(m), 1, 1, fake, fake, fake, fake, fake, None, ctypes.byref(sz), None)
    assert st == -1
    L.em_last_error(buf, 256)
    assert b"boundary-normal" in buf.value      # weights are refused on the ordered-gather path
    big = ctypes.c_size_t(1 << 20)
    info = (ctypes.c_int64 * p._lib.PLAN_INFO_LEN)()
    st = L.em_batched_fwd_adj(0, None, None, 1, info, 3, 1, 0, None, fake, ctypes.byref(big), None)
    assert st == -1
    st = L.em_batched_fwd_adj(1, fake, fake, 0, info, 3, 1, 0, fake, fake, ctypes.byref(big), None)
    assert st == -1                             # no work items
    L.em_last_error(buf, 256)
    assert b"n_items" in buf.value
    st = L.em_batched_fwd_adj(1, fake, fake, 1, info, 3, 1, -2, fake, fake, ctypes.byref(big), None)
    assert st == -1                             # unknown launch shape
    L.em_last_error(buf, 256)
    assert b"blocks" in buf.value


def test_partial_entry_point_rejects_bad_arguments(lib):
    """em_edge_metrics_partial validates its range, precision and outputs
    before any device work."""
    import paper_2502_00778_gb300 as p
    L = p.load()
    buf = ctypes.create_string_buffer(256)
    m = p._lib.EmMesh()
    m.dim, m.n_nodes, m.n_elems, m.n_edges = 3, 4, 1, 6
    m.elems = m.elem2edge = m.edges = 4096   # never dereferenced: validation fails first
    fake = ctypes.c_void_p(4096)
    null = None
    # range outside [0, n_elems]
    assert L.em_edge_metrics_partial(ctypes.byref(m), 0, 0, 2, fake, null, null, fake, fake, fake, null, null) == -1
    L.em_last_error(buf, 256)
    assert b"range" in buf.value
    assert L.em_edge_metrics_partial(ctypes.byref(m), 0, 1, 0, fake, null, null, fake, fake, fake, null, null) == -1
    # forms other than FP64 and MIXED
    assert L.em_edge_metrics_partial(ctypes.byref(m), 1, 0, 1, fake, null, null, fake, fake, fake, null, null) == -1
    L.em_last_error(buf, 256)
    assert b"EM_PREC_FP64" in buf.value
    # forward outputs only in part, adjoint without w, nothing asked
    assert L.em_edge_metrics_partial(ctypes.byref(m), 0, 0, 1, fake, null, null, fake, null, null, null, null) == -1
    assert L.em_edge_metrics_partial(ctypes.byref(m), 0, 0, 1, fake, null, null, null, null, null, fake, null) == -1
    L.em_last_error(buf, 256)
    assert b"needs w" in buf.value
    assert L.em_edge_metrics_partial(ctypes.byref(m), 0, 0, 1, fake, null, null, null, null, null, null, null) == -1


def test_empty_grids_are_refused_before_device_work(lib):
    """A grid needs at least one node, one element and one edge: zero counts
    fail with EM_ERR_ARG before any device call."""
    import paper_2502_00778_gb300 as p
    L = p.load()
    buf = ctypes.create_string_buffer(256)
    sz = ctypes.c_size_t(0)
    cnt = (ctypes.c_int64 * 3)()
    for nv, ne in ((10, 0), (0, 10)):
        st = L.em_edge_build(3, nv, ne, None, None, None, ctypes.byref(sz), None, 0, None, None, None, None, None, 0,
                             None, 0, cnt, None)
        assert st == -1
    psz = ctypes.c_size_t(0)
    info = (ctypes.c_int64 * p._lib.PLAN_INFO_LEN)()
    st = L.em_plan_build(3, 10, 0, None, None, 6, None, 0, None, None, 0, None, 128, None, ctypes.byref(sz), None,
                         ctypes.byref(psz), info, None)
    assert st == -1
    m = p._lib.EmMesh()
    m.elems = m.elem2edge = m.edges = 4096   # never dereferenced: validation fails first
    fake = ctypes.c_void_p(4096)
    for nv, ne, nedges in ((4, 0, 6), (0, 1, 6), (4, 1, 0)):
        m.dim, m.n_nodes, m.n_elems, m.n_edges = 3, nv, ne, nedges
        st = L.em_edge_metrics(ctypes.byref(m), 0, 0, fake, fake, fake, fake, None, ctypes.byref(sz), None)
        assert st == -1
        L.em_last_error(buf, 256)
        assert b"positive" in buf.value
        st = L.em_edge_metrics_partial(ctypes.byref(m), 0, 0, 0, fake, None, None, fake, fake, fake, None, None)
        assert st == -1
        L.em_last_error(buf, 256)
        assert b"positive" in buf.value

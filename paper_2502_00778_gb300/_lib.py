"""ctypes declarations of the C ABI in include/edgemetrics.h.

Loading never falls back to anything: if the compiled library is missing the
import of the functions that need it raises.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libedgemetrics.so")

EM_OK = 0
ERRORS = {
    -1: "EM_ERR_ARG", -2: "EM_ERR_WORKSPACE", -3: "EM_ERR_CUDA", -4: "EM_ERR_BAD_ID",
    -5: "EM_ERR_DEGENERATE", -6: "EM_ERR_TIMEOUT", -7: "EM_ERR_CAPACITY", -8: "EM_ERR_TOPOLOGY",
}

PLAN_INFO_LEN = 32
PLAN_INFO = {"tile_nodes": 0, "tiles": 1, "max_edge_valence": 13, "max_node_valence": 14, "rec_nodes": 20,
             "rec_edges": 21, "rec_bnodes": 22}

PREC = {"fp64": 0, "dw": 1, "mixed": 2, "mixed_comp32": 3}
PATH = {"atomic": 0, "gather": 1, "csr": 2, "tiled": 3}

_c = ctypes
_vp = _c.c_void_p
_i64 = _c.c_int64
_i64p = _c.POINTER(_c.c_int64)
_szp = _c.POINTER(_c.c_size_t)


class EmMesh(_c.Structure):
    _fields_ = [
        ("dim", _c.c_int),
        ("n_nodes", _i64), ("n_elems", _i64), ("n_edges", _i64), ("n_bfaces", _i64), ("n_bnodes", _i64),
        ("elems", _vp), ("elem2edge", _vp), ("edges", _vp), ("edge_ptr", _vp), ("edge_slot", _vp),
        ("bface", _vp), ("bface_owner", _vp), ("bnode", _vp),
        ("plan", _vp), ("plan_bytes", _c.c_size_t),
        ("plan_info", _c.c_int64 * PLAN_INFO_LEN),
    ]


class EmBatchItem(_c.Structure):
    _fields_ = [
        ("mesh", EmMesh),
        ("x", _vp), ("w", _vp), ("c", _vp),
        ("n_edge", _vp), ("vol", _vp), ("bnormal", _vp), ("grad_x", _vp),
        ("rec", _vp),
    ]


SIGNATURES = {
    "em_version": ([], _c.c_int),
    "em_kernel_launches": ([], _c.c_int64),
    "em_last_error": ([_c.c_char_p, _c.c_size_t], _c.c_int),
    "em_edge_build": ([_c.c_int, _i64, _i64, _vp, _vp, _vp, _szp, _vp, _i64, _vp, _vp, _vp, _vp, _vp, _i64, _vp, _i64,
                       _i64p, _vp], _c.c_int),
    "em_plan_build": ([_c.c_int, _i64, _i64, _vp, _vp, _i64, _vp, _i64, _vp, _vp, _i64, _vp, _c.c_int, _vp, _szp,
                       _vp, _szp, _i64p, _vp], _c.c_int),
    "em_edge_metrics": ([_c.POINTER(EmMesh), _c.c_int, _c.c_int, _vp, _vp, _vp, _vp, _vp, _szp, _vp], _c.c_int),
    "em_edge_metrics_adjoint": ([_c.POINTER(EmMesh), _c.c_int, _c.c_int, _vp, _vp, _vp, _vp, _vp, _vp, _szp, _vp],
                                _c.c_int),
    "em_edge_metrics_fused": ([_c.POINTER(EmMesh), _c.c_int, _c.c_int, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp,
                               _szp, _vp], _c.c_int),
    "em_edge_metrics_noalloc": ([_c.POINTER(EmMesh), _vp, _vp, _vp, _vp, _vp], _c.c_int),
    "em_edge_metrics_partial": ([_c.POINTER(EmMesh), _c.c_int, _i64, _i64, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp],
                                _c.c_int),
    "em_edge_volume": ([_c.POINTER(EmMesh), _vp, _vp, _vp, _vp, _szp, _vp], _c.c_int),
    "em_edge_areas_traditional": ([_c.POINTER(EmMesh), _vp, _vp, _vp], _c.c_int),
    "em_edge_residual": ([_c.POINTER(EmMesh), _vp, _vp, _vp, _vp, _vp, _szp, _vp], _c.c_int),
    "em_check_elements": ([_c.c_int, _i64, _i64, _vp, _vp, _vp, _szp, _i64p, _vp], _c.c_int),
    "em_batched_fwd_adj": ([_c.c_int, _vp, _vp, _i64, _i64p, _c.c_int, _c.c_int, _c.c_int, _vp, _vp, _szp, _vp],
                           _c.c_int),
    "em_plan_tiles": ([_vp, _i64p, _vp], _c.c_int),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load the compiled library (raises OSError if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise OSError(f"edge-metrics CUDA library not built: {path} (run __graft_entry__.build())")
        L = _c.CDLL(path)
        for name, (args, res) in SIGNATURES.items():  # noqa: B007
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


class EMError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


def check(status):
    if status != EM_OK:
        buf = _c.create_string_buffer(512)
        load().em_last_error(buf, 512)
        raise EMError(status, buf.value.decode(errors="replace"))
    return status

// C-ABI entry points: argument validation, dispatch, thread-local last error.
#include <atomic>
#include <cstring>
#include <string>

#include "em_common.cuh"
#include "em_kernels.cuh"

namespace em {

namespace {
thread_local int t_status = EM_OK;
thread_local std::string t_msg;
std::atomic<int64_t> g_launches{0};
}  // namespace

void note_launches(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

void set_error(int code, const std::string& msg) {
    t_status = code;
    t_msg = msg;
}

int fail(int code, const std::string& msg) {
    set_error(code, msg);
    return code;
}

static int ok() {
    t_status = EM_OK;
    t_msg.clear();
    return EM_OK;
}

static int check_mesh(const em_mesh* m, bool need_e2e = true) {
    if (!m) return fail(EM_ERR_ARG, "mesh is NULL");
    if (m->dim != 2 && m->dim != 3) return fail(EM_ERR_ARG, "mesh->dim must be 2 or 3");
    if (m->n_nodes <= 0 || m->n_elems <= 0 || m->n_edges <= 0 || m->n_bfaces < 0 || m->n_bnodes < 0)
        return fail(EM_ERR_ARG, "mesh sizes must be positive");
    if (m->n_nodes >= INT32_MAX || m->n_elems >= INT32_MAX || m->n_edges >= INT32_MAX)
        return fail(EM_ERR_ARG, "mesh sizes must be below 2^31 - 1");
    if (!m->elems || (need_e2e && !m->elem2edge) || !m->edges) return fail(EM_ERR_ARG, "mesh arrays are NULL");
    if (m->n_bfaces && (!m->bface || !m->bface_owner)) return fail(EM_ERR_ARG, "boundary face arrays are NULL");
    if (m->n_bnodes && !m->bnode) return fail(EM_ERR_ARG, "bnode is NULL");
    if (reinterpret_cast<uintptr_t>(m->elems) & 15) return fail(EM_ERR_ARG, "elems must be 16-byte aligned");
    return EM_OK;
}

}  // namespace em

using namespace em;

extern "C" {

int em_version(void) { return EM_VERSION; }

int64_t em_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

int em_last_error(char* buf, size_t n) {
    if (buf && n) {
        size_t k = t_msg.size() < n - 1 ? t_msg.size() : n - 1;
        memcpy(buf, t_msg.data(), k);
        buf[k] = 0;
    }
    return t_status;
}

int em_edge_build(int dim, int64_t n_nodes, int64_t n_elems, const int32_t* elems, const double* x, void* ws,
                  size_t* ws_bytes, int32_t* edges, int64_t edges_cap, int32_t* elem2edge, int32_t* edge_ptr,
                  int32_t* edge_slot, int32_t* bface, int32_t* bface_owner, int64_t bface_cap, int32_t* bnode,
                  int64_t bnode_cap, int64_t* counts, void* stream) {
    if (elems && (reinterpret_cast<uintptr_t>(elems) & 15)) return fail(EM_ERR_ARG, "elems must be 16-byte aligned");
    int st = edge_build_impl(dim, n_nodes, n_elems, elems, x, ws, ws_bytes, edges, edges_cap, elem2edge, edge_ptr,
                             edge_slot, bface, bface_owner, bface_cap, bnode, bnode_cap, counts, as_stream(stream));
    return st == EM_OK ? ok() : st;
}

int em_check_elements(int dim, int64_t n_nodes, int64_t n_elems, const int32_t* elems, const double* x, void* ws,
                      size_t* ws_bytes, int64_t* counts, void* stream) {
    bool query;
    EM_TRY(check_ws(ws, ws_bytes, check_elements_ws_bytes(), &query));
    if (query) return ok();
    if (elems && (reinterpret_cast<uintptr_t>(elems) & 15)) return fail(EM_ERR_ARG, "elems must be 16-byte aligned");
    int st = check_elements_impl(dim, n_nodes, n_elems, elems, x, ws, counts, as_stream(stream));
    return st == EM_OK ? ok() : st;
}

int em_edge_metrics(const em_mesh* mesh, int precision, int path, const double* x, double* n_edge, double* vol,
                    double* bnormal, void* ws, size_t* ws_bytes, void* stream) {
    EM_TRY(check_mesh(mesh));
    size_t need = 0;
    if (path == EM_PATH_ATOMIC) {
        if (precision != EM_PREC_FP64 && precision != EM_PREC_MIXED && precision != EM_PREC_MIXED_COMP32)
            return fail(EM_ERR_ARG, "atomic path supports FP64, MIXED and MIXED_COMP32");
        need = atomic_fwd_ws_bytes(mesh, precision);
    } else if (path == EM_PATH_GATHER || path == EM_PATH_TILED) {
        if (precision != EM_PREC_FP64 && precision != EM_PREC_DW && precision != EM_PREC_MIXED)
            return fail(EM_ERR_ARG, "gather/tiled paths support FP64, DW and MIXED");
        if (!mesh->plan) return fail(EM_ERR_ARG, "gather/tiled paths need a plan from em_plan_build");
        need = gather_ws_bytes(mesh, path == EM_PATH_TILED ? GATHER_SCATTER : 0);
    } else if (path == EM_PATH_CSR) {
        if (precision != EM_PREC_FP64) return fail(EM_ERR_ARG, "CSR path supports FP64 only");
        if (!mesh->edge_ptr || !mesh->edge_slot) return fail(EM_ERR_ARG, "CSR path needs edge_ptr and edge_slot");
        need = csr_fwd_ws_bytes(mesh);
    } else {
        return fail(EM_ERR_ARG, "unknown path");
    }
    bool query;
    EM_TRY(check_ws(ws, ws_bytes, need, &query));
    if (query) return ok();
    if (!x) return fail(EM_ERR_ARG, "x is NULL");
    cudaStream_t s = as_stream(stream);
    int st;
    if (path == EM_PATH_ATOMIC) {
        st = atomic_fwd(mesh, precision, x, n_edge, vol, bnormal, ws, s);
    } else if (path == EM_PATH_GATHER || path == EM_PATH_TILED) {
        if (!n_edge || !vol || (mesh->n_bnodes && !bnormal)) return fail(EM_ERR_ARG, "gather path needs all outputs");
        st = gather_run(mesh, precision, GATHER_FWD | (path == EM_PATH_TILED ? GATHER_SCATTER : 0), x, nullptr,
                        nullptr, n_edge, vol, bnormal, nullptr, ws, s);
    } else {
        if (!n_edge || !vol || (mesh->n_bnodes && !bnormal)) return fail(EM_ERR_ARG, "CSR path needs all outputs");
        st = csr_fwd(mesh, x, n_edge, vol, bnormal, ws, s);
    }
    return st == EM_OK ? ok() : st;
}

int em_edge_metrics_adjoint(const em_mesh* mesh, int precision, int path, const double* x, const double* w,
                            const double* c, const double* bw, double* grad_x, void* ws, size_t* ws_bytes,
                            void* stream) {
    EM_TRY(check_mesh(mesh));
    size_t need = 0;
    if (path == EM_PATH_ATOMIC) {
        if (precision != EM_PREC_FP64 && precision != EM_PREC_MIXED)
            return fail(EM_ERR_ARG, "atomic adjoint supports FP64 and MIXED");
    } else if (path == EM_PATH_GATHER || path == EM_PATH_TILED) {
        if (precision != EM_PREC_FP64 && precision != EM_PREC_DW && precision != EM_PREC_MIXED)
            return fail(EM_ERR_ARG, "gather/tiled adjoint supports FP64, DW and MIXED");
        if (!mesh->plan) return fail(EM_ERR_ARG, "gather/tiled paths need a plan from em_plan_build");
        need = gather_ws_bytes(mesh, path == EM_PATH_TILED ? GATHER_SCATTER : 0);
    } else {
        return fail(EM_ERR_ARG, "adjoint supports the ATOMIC, GATHER and TILED paths");
    }
    if (bw && path == EM_PATH_GATHER)
        return fail(EM_ERR_ARG, "boundary-normal weights are supported by the TILED and ATOMIC paths");
    const size_t bw_off = (need + 255) & ~size_t(255);
    need = bw_off + bw_ws_bytes(mesh);
    bool query;
    EM_TRY(check_ws(ws, ws_bytes, need, &query));
    if (query) return ok();
    if (!x || !w || !grad_x) return fail(EM_ERR_ARG, "x, w and grad_x must not be NULL");
    cudaStream_t s = as_stream(stream);
    BwAux aux;
    EM_TRY(bw_prepare(mesh, bw, static_cast<char*>(ws) + bw_off, &aux, s));
    int st;
    if (path == EM_PATH_ATOMIC) {
        st = atomic_adj(mesh, precision, x, w, c, grad_x, s);
        if (st == EM_OK) st = atomic_bw_adj(mesh, x, aux, grad_x, s);
    } else {
        st = gather_run(mesh, precision, GATHER_ADJ | (path == EM_PATH_TILED ? GATHER_SCATTER : 0), x, w, c, nullptr,
                        nullptr, nullptr, grad_x, ws, s, &aux);
    }
    return st == EM_OK ? ok() : st;
}

int em_edge_metrics_fused(const em_mesh* mesh, int precision, int path, const double* x, const double* w,
                          const double* c, const double* bw, double* n_edge, double* vol, double* bnormal,
                          double* grad_x, void* ws, size_t* ws_bytes, void* stream) {
    EM_TRY(check_mesh(mesh));
    if (path != EM_PATH_GATHER && path != EM_PATH_TILED) return fail(EM_ERR_ARG, "fused pass: GATHER or TILED path");
    if (precision != EM_PREC_FP64 && precision != EM_PREC_DW && precision != EM_PREC_MIXED)
        return fail(EM_ERR_ARG, "fused pass supports FP64, DW and MIXED");
    if (!mesh->plan) return fail(EM_ERR_ARG, "fused pass needs a plan from em_plan_build");
    if (bw && path == EM_PATH_GATHER)
        return fail(EM_ERR_ARG, "boundary-normal weights are supported by the TILED and ATOMIC paths");
    const size_t bw_off = (gather_ws_bytes(mesh, path == EM_PATH_TILED ? GATHER_SCATTER : 0) + 255) & ~size_t(255);
    bool query;
    EM_TRY(check_ws(ws, ws_bytes, bw_off + bw_ws_bytes(mesh), &query));
    if (query) return ok();
    if (!x || !w || !grad_x || !n_edge || !vol || (mesh->n_bnodes && !bnormal))
        return fail(EM_ERR_ARG, "fused pass needs x, w and all outputs");
    cudaStream_t s = as_stream(stream);
    BwAux aux;
    EM_TRY(bw_prepare(mesh, bw, static_cast<char*>(ws) + bw_off, &aux, s));
    int st = gather_run(mesh, precision, GATHER_FWD | GATHER_ADJ | (path == EM_PATH_TILED ? GATHER_SCATTER : 0), x, w,
                        c, n_edge, vol, bnormal, grad_x, ws, s, &aux);
    return st == EM_OK ? ok() : st;
}

int em_edge_volume(const em_mesh* mesh, const double* x, const double* n_edge, double* vol, void* ws,
                   size_t* ws_bytes, void* stream) {
    if (!mesh) return fail(EM_ERR_ARG, "mesh is NULL");
    if (mesh->dim != 2 && mesh->dim != 3) return fail(EM_ERR_ARG, "mesh->dim must be 2 or 3");
    if (mesh->n_nodes <= 0 || mesh->n_edges <= 0 || !mesh->edges) return fail(EM_ERR_ARG, "mesh needs edges");
    bool query;
    EM_TRY(check_ws(ws, ws_bytes, edge_volume_ws_bytes(mesh), &query));
    if (query) return ok();
    if (!x || !n_edge || !vol) return fail(EM_ERR_ARG, "x, n_edge and vol must not be NULL");
    int st = edge_volume(mesh, x, n_edge, vol, ws, as_stream(stream));
    return st == EM_OK ? ok() : st;
}

int em_edge_areas_traditional(const em_mesh* mesh, const double* x, double* n_edge, void* stream) {
    if (!mesh) return fail(EM_ERR_ARG, "mesh is NULL");
    if (mesh->dim != 2 && mesh->dim != 3) return fail(EM_ERR_ARG, "mesh->dim must be 2 or 3");
    if (mesh->n_elems <= 0 || mesh->n_edges <= 0 || !mesh->elems || !mesh->elem2edge)
        return fail(EM_ERR_ARG, "mesh needs elems and elem2edge");
    if (!x || !n_edge) return fail(EM_ERR_ARG, "x and n_edge must not be NULL");
    int st = traditional_areas(mesh, x, n_edge, as_stream(stream));
    return st == EM_OK ? ok() : st;
}

int em_edge_residual(const em_mesh* mesh, const double* F, const double* n_edge, const double* bnormal, double* res,
                     void* ws, size_t* ws_bytes, void* stream) {
    if (!mesh) return fail(EM_ERR_ARG, "mesh is NULL");
    if (mesh->dim != 2 && mesh->dim != 3) return fail(EM_ERR_ARG, "mesh->dim must be 2 or 3");
    if (mesh->n_nodes <= 0 || mesh->n_edges <= 0 || !mesh->edges) return fail(EM_ERR_ARG, "mesh needs edges");
    if (mesh->n_bnodes < 0 || (mesh->n_bnodes && !mesh->bnode)) return fail(EM_ERR_ARG, "mesh needs bnode");
    bool query;
    EM_TRY(check_ws(ws, ws_bytes, edge_volume_ws_bytes(mesh), &query));
    if (query) return ok();
    if (!F || !n_edge || !res || (mesh->n_bnodes && !bnormal))
        return fail(EM_ERR_ARG, "F, n_edge, bnormal and res must not be NULL");
    int st = edge_residual(mesh, F, n_edge, bnormal, res, ws, as_stream(stream));
    return st == EM_OK ? ok() : st;
}

int em_edge_metrics_noalloc(const em_mesh* mesh, const double* x, double* n_edge, double* vol, double* bnormal,
                            void* stream) {
    EM_TRY(check_mesh(mesh));
    if (!x || !n_edge || !vol || (mesh->n_bnodes && !bnormal))
        return fail(EM_ERR_ARG, "x, n_edge, vol and bnormal must not be NULL");
    int st = atomic_fwd_noalloc(mesh, x, n_edge, vol, bnormal, as_stream(stream));
    return st == EM_OK ? ok() : st;
}

int em_edge_metrics_partial(const em_mesh* mesh, int precision, int64_t elem_begin, int64_t elem_end,
                            const double* x, const double* w, const double* c, double* n_edge, double* vol,
                            double* bnormal, double* grad_x, void* stream) {
    EM_TRY(check_mesh(mesh));
    if (precision != EM_PREC_FP64 && precision != EM_PREC_MIXED)
        return fail(EM_ERR_ARG, "partial metrics support EM_PREC_FP64 and EM_PREC_MIXED");
    if (elem_begin < 0 || elem_begin > elem_end || elem_end > mesh->n_elems)
        return fail(EM_ERR_ARG, "element range must satisfy 0 <= elem_begin <= elem_end <= n_elems");
    if (!x) return fail(EM_ERR_ARG, "x must not be NULL");
    const bool fwd = n_edge || vol || bnormal;
    if (fwd && (!n_edge || !vol || (mesh->n_bnodes && !bnormal)))
        return fail(EM_ERR_ARG, "partial forward needs n_edge, vol and bnormal together");
    if (grad_x && !w) return fail(EM_ERR_ARG, "partial adjoint needs w");
    if (!fwd && !grad_x) return fail(EM_ERR_ARG, "nothing to compute: give the forward outputs, grad_x or both");
    int st = atomic_partial(mesh, precision, elem_begin, elem_end, x, w, c, n_edge, vol, bnormal, grad_x,
                            as_stream(stream));
    return st == EM_OK ? ok() : st;
}

int em_plan_build(int dim, int64_t n_nodes, int64_t n_elems, const int32_t* elems, const int32_t* elem2edge,
                  int64_t n_edges, const int32_t* edges, int64_t n_bfaces, const int32_t* bface,
                  const int32_t* bface_owner, int64_t n_bnodes, const int32_t* bnode, int tile_nodes, void* ws,
                  size_t* ws_bytes, void* plan, size_t* plan_bytes, int64_t* plan_info, void* stream) {
    int st = plan_build_impl(dim, n_nodes, n_elems, elems, elem2edge, n_edges, edges, n_bfaces, bface, bface_owner,
                             n_bnodes, bnode, tile_nodes, ws, ws_bytes, plan, plan_bytes, plan_info,
                             as_stream(stream));
    return st == EM_OK ? ok() : st;
}

int em_plan_tiles(const void* plan, int64_t* n_tiles, void* stream) {
    int st = plan_tiles_impl(plan, n_tiles, as_stream(stream));
    return st == EM_OK ? ok() : st;
}

int em_batched_fwd_adj(int n_meshes, const em_batch_item* items, const int64_t* tile_prefix, int64_t n_items,
                       const int64_t* max_info, int dim, int precision, int blocks, int32_t* status, void* ws,
                       size_t* ws_bytes, void* stream) {
    int st = batched_impl(n_meshes, items, tile_prefix, n_items, max_info, dim, precision, blocks, status, ws,
                          ws_bytes, as_stream(stream));
    return st == EM_OK ? ok() : st;
}

}  // extern "C"

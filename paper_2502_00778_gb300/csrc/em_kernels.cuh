// Internal entry points shared between the translation units of the library.
#pragma once
#include "em_common.cuh"

namespace em {

// boundary-normal weights of the adjoint (L += sum_b bw_b . bnormal_b):
// node -> boundary-node map and the key of max |bw|, built in the workspace
struct BwAux {
    const double* bw;       // NULL: no boundary-normal term
    const int32_t* map;     // [n_nodes] boundary-node index or -1
    const unsigned* key;    // upper word of max |bw| (order-preserving)
};

int edge_build_impl(int dim, int64_t nv, int64_t ne, const int32_t* elems, const double* x, void* ws, size_t* ws_bytes,
                    int32_t* edges, int64_t edges_cap, int32_t* elem2edge, int32_t* edge_ptr, int32_t* edge_slot,
                    int32_t* bface, int32_t* bowner, int64_t bface_cap, int32_t* bnode, int64_t bnode_cap,
                    int64_t* counts, cudaStream_t s);
size_t check_elements_ws_bytes();
int check_elements_impl(int dim, int64_t nv, int64_t ne, const int32_t* elems, const double* x, void* ws,
                        int64_t* counts, cudaStream_t s);

size_t atomic_fwd_ws_bytes(const em_mesh* m, int prec);
int atomic_fwd(const em_mesh* m, int prec, const double* x, double* n, double* vol, double* bnormal, void* ws,
               cudaStream_t s);
int atomic_fwd_noalloc(const em_mesh* m, const double* x, double* n, double* vol, double* bnormal, cudaStream_t s);
int atomic_partial(const em_mesh* m, int prec, int64_t e0, int64_t e1, const double* x, const double* w,
                   const double* c, double* n, double* vol, double* bnormal, double* g, cudaStream_t s);
int atomic_adj(const em_mesh* m, int prec, const double* x, const double* w, const double* c, double* g,
               cudaStream_t s);

}  // namespace em

namespace em {

enum { GATHER_FWD = 1, GATHER_ADJ = 2, GATHER_SCATTER = 4 };

size_t gather_ws_bytes(const em_mesh* m, int what);
int gather_run(const em_mesh* m, int prec, int what, const double* x, const double* w, const double* c, double* n,
               double* vol, double* bnormal, double* g, void* ws, cudaStream_t s, const BwAux* bw = nullptr);

size_t csr_fwd_ws_bytes(const em_mesh* m);
size_t edge_volume_ws_bytes(const em_mesh* m);
int edge_volume(const em_mesh* m, const double* x, const double* n, double* vol, void* ws, cudaStream_t s);
size_t bw_ws_bytes(const em_mesh* m);
int bw_prepare(const em_mesh* m, const double* bw, void* ws, BwAux* aux, cudaStream_t s);
int atomic_bw_adj(const em_mesh* m, const double* x, const BwAux& aux, double* g, cudaStream_t s);
int traditional_areas(const em_mesh* m, const double* x, double* n, cudaStream_t s);
int edge_residual(const em_mesh* m, const double* F, const double* n, const double* bnormal, double* res, void* ws,
                  cudaStream_t s);
int csr_fwd(const em_mesh* m, const double* x, double* n, double* vol, double* bnormal, void* ws, cudaStream_t s);

int plan_build_impl(int dim, int64_t nv, int64_t ne, const int32_t* elems, const int32_t* elem2edge, int64_t n_edges,
                    const int32_t* edges, int64_t nbf, const int32_t* bface, const int32_t* bowner, int64_t nbn,
                    const int32_t* bnode, int tile_nodes, void* ws, size_t* ws_bytes, void* plan, size_t* plan_bytes,
                    int64_t* plan_info, cudaStream_t s);
int plan_tiles_impl(const void* plan, int64_t* n_tiles, cudaStream_t s);

// scatter tiles (em_scatter.cu): workspace = the tiles' partial-sum records
size_t scatter_ws_bytes(const em_mesh* m);
int scatter_run(const em_mesh* m, int prec, int what, const double* x, const double* w, const double* c, double* n,
                double* vol, double* bnormal, double* g, void* ws, cudaStream_t s, const BwAux* bw);

int batched_impl(int n_meshes, const em_batch_item* items, const int64_t* tile_prefix, int64_t n_items,
                 const int64_t* max_info, int dim, int precision, int blocks, int32_t* status, void* ws,
                 size_t* ws_bytes, cudaStream_t s);

}  // namespace em

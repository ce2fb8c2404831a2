/*
 * edgemetrics.h -- C ABI of the GB300 (sm_103a) edge-metrics library.
 *
 * The library computes, on triangular (dim = 2) and tetrahedral (dim = 3)
 * grids, the grid metrics of the edge-based finite-volume discretization
 * directly from element geometry, without forming median-dual control
 * volumes (H. Nishikawa, arXiv 2502.00778):
 *
 *   n_e      lumped directed-area vector of every edge e = {j,k}, j < k,
 *            pointing from j to k (Sec. 2).  Proposed algorithm, Sec. 3.2:
 *            n_jk = 2/(D(D+1)) sum_{E containing jk} n_j^E  plus
 *            n_B/(D(D+1)) for every boundary face B containing jk
 *            (Eq. efficient_njk_formula_general_D and the boundary
 *            correction after it), where n_j^E is the outward area vector of
 *            the face of E opposite j and n_B the outward area vector of B.
 *   V_i      median-dual volume of every node: sum over elements E of
 *            V_E/(D+1) (Sec. 4.2).
 *   b_i      boundary dual-face normal of every boundary node:
 *            (1/D) sum_{B containing i} n_B (Sec. 3.2.3, closure).
 *   dL/dx    gradient of L = sum_e w_e . n_e + sum_i c_i V_i with respect to
 *            the node coordinates (the adjoint of the above).
 *
 * Conventions shared by every entry point:
 *   - Every array argument is a DEVICE pointer owned by the caller unless
 *     stated otherwise; the library never allocates or frees caller memory.
 *   - Temporary storage is a caller-provided device workspace: call once with
 *     ws == NULL to receive the required size in *ws_bytes, then call again
 *     with a buffer of at least that size (256-byte aligned).
 *   - `stream` is a cudaStream_t passed as void*; NULL means the legacy
 *     default stream.  All work is enqueued on it.  Entry points that must
 *     return a count to the host (em_edge_build, em_plan_build) synchronize
 *     the stream before returning; all others are asynchronous.
 *   - Element connectivity is int32 [n_elems][4]; triangles use the first
 *     three entries and store -1 in the fourth.  Node ids are 0-based.
 *   - Coordinates are float64 [n_nodes][dim], row-major.
 *   - Node, element, edge and face counts must be below 2^31 - 1 (int32
 *     indices); byte offsets are size_t.
 *   - A grid has at least one node, one element and (once built) one edge:
 *     entry points that take a grid refuse zero counts with EM_ERR_ARG
 *     before any device work, since an empty grid has nothing to compute
 *     (em_check_elements alone accepts n_elems == 0 and reports no errors).
 *   - Every function returns an int status: EM_OK (0) or a negative EM_ERR_*
 *     code.  em_last_error() returns a message for the calling thread's last
 *     failure.  No C++ exception crosses the ABI and no kernel traps: device-
 *     side failures (bad ids, degenerate elements, timeouts) are reported
 *     through a status word that the host reads.
 */
#ifndef EDGEMETRICS_H
#define EDGEMETRICS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define EM_VERSION 200

/* status codes */
#define EM_OK               0
#define EM_ERR_ARG         -1   /* invalid argument (null pointer, bad size, unsupported dim/mode) */
#define EM_ERR_WORKSPACE   -2   /* workspace missing or smaller than required */
#define EM_ERR_CUDA        -3   /* a CUDA runtime call failed */
#define EM_ERR_BAD_ID      -4   /* element references a node id outside [0,n_nodes) or repeats a node */
#define EM_ERR_DEGENERATE  -5   /* an element has zero measure */
#define EM_ERR_TIMEOUT     -6   /* a bounded device-side wait gave up */
#define EM_ERR_CAPACITY    -7   /* an output capacity (edges_cap, ...) is too small */
#define EM_ERR_TOPOLOGY    -8   /* a face is shared by more than two elements */

/* arithmetic forms */
#define EM_PREC_FP64   0  /* native double-precision arithmetic and FP64 accumulation */
#define EM_PREC_DW     1  /* FP64-accurate results computed without FP64 instructions:
                             exact coordinate differences, FP32 double-word (error-free
                             transformation) products, exact integer accumulation */
#define EM_PREC_MIXED  2  /* FP32 element arithmetic on element-relative coordinates
                             (rounding ~1e-7 relative); accumulation exact (gather path)
                             or FP64 atomics (atomic path) */
#define EM_PREC_MIXED_COMP32 3 /* atomic path only: FP32 element arithmetic with
                             compensated FP32 (two-float) atomic accumulation */

/* summation paths */
#define EM_PATH_ATOMIC 0  /* element-centric scatter with global FP64 atomics
                             (summation order not reproducible) */
#define EM_PATH_GATHER 1  /* tiled gather: every output written once, exact integer
                             accumulation; bit-reproducible run to run */
#define EM_PATH_CSR    2  /* edge-centric CSR gather (per edge, its element slots in
                             ascending order; FP64 only); bit-reproducible */
#define EM_PATH_TILED  3  /* scatter tiles over the same node ranges as
                             EM_PATH_GATHER: every element is computed once, by
                             the tile of its lowest node, and adds its
                             contributions to the tile's accumulators with
                             shared-memory integer atomics on exact fixed-point
                             values (per-tile power-of-two scale); partial sums
                             of targets owned by later tiles are added to the
                             owners' outputs in a fixed order, so the results
                             are bit-reproducible run to run */

int em_version(void);

/* Number of CUDA kernels this library has enqueued in the calling process
 * (all threads, all devices) since it was loaded; a diagnostic for
 * benchmarks.  Memset and copy operations are not counted. */
int64_t em_kernel_launches(void);

/* Copies the calling thread's last error message (NUL-terminated, truncated
 * to n bytes) into buf; returns the last status code. */
int em_last_error(char* buf, size_t n);

/* ------------------------------------------------------------------------ */
/* Topology                                                                  */
/* ------------------------------------------------------------------------ */

/* em_edge_build -- integer topology of a grid (run once per connectivity).
 *
 * Edges (Sec. 2: edge(e,1) = j < edge(e,2) = k) are all element edges, sorted
 * lexicographically by (j,k); they are found by a radix sort of 64-bit
 * (min,max) keys and a unique pass.  Results are bit-exact.
 *
 *   elems        [n_elems][4] int32, read.
 *   x            [n_nodes][dim] float64, read: only used to orient boundary
 *                faces outward.
 *   edges        [edges_cap][2] int32, written: edges[e] = {j, k}, j < k.
 *   elem2edge    [n_elems][nle] int32, written (nle = 6 for tets, 3 for
 *                tris): edge id of local edge l, local edges taken over the
 *                STORED node order as (0,1),(0,2),(0,3),(1,2),(1,3),(2,3)
 *                (tris: (0,1),(0,2),(1,2)).
 *   edge_ptr     [edges_cap+1] int32 or NULL, written: CSR offsets of each
 *                edge's element slots.
 *   edge_slot    [n_elems*nle] int32 or NULL, written: slots e*nle+l, grouped
 *                by edge, ascending inside each edge.
 *   bface        [bface_cap][dim] int32, written: faces seen by exactly one
 *                element (the boundary elements of Sec. 3.2, taken as given in
 *                the paper), sorted by their sorted node ids, stored in the
 *                order that makes n_B outward (3D: first node = smallest id,
 *                n_B = 1/2 (x1-x0) x (x2-x0); 2D: n_B = (y0-y1, x1-x0)).
 *   bface_owner  [bface_cap] int32, written: elem*4 + local index of the
 *                owner's node opposite the face.
 *   bnode        [bnode_cap] int32, written: ascending ids of nodes on
 *                boundary faces.
 *   counts       HOST int64[3], written: n_edges, n_bfaces, n_bnodes.
 *
 * Capacities: edges_cap >= number of edges (at most nle*n_elems), bface_cap
 * >= number of boundary faces (at most (dim+1)*n_elems), bnode_cap >= number
 * of boundary nodes (at most n_nodes); otherwise EM_ERR_CAPACITY and the
 * needed counts are still written to `counts`.  Synchronizes `stream`.
 * Errors: EM_ERR_BAD_ID, EM_ERR_TOPOLOGY, EM_ERR_CAPACITY, EM_ERR_ARG,
 * EM_ERR_WORKSPACE, EM_ERR_CUDA. */
int em_edge_build(int dim, int64_t n_nodes, int64_t n_elems,
                  const int32_t* elems, const double* x,
                  void* ws, size_t* ws_bytes,
                  int32_t* edges, int64_t edges_cap,
                  int32_t* elem2edge,
                  int32_t* edge_ptr, int32_t* edge_slot,
                  int32_t* bface, int32_t* bface_owner, int64_t bface_cap,
                  int32_t* bnode, int64_t bnode_cap,
                  int64_t* counts,
                  void* stream);

/* host summary of a plan (em_plan_build's plan_info output, em_mesh.plan_info) */
#define EM_PLAN_INFO_LEN 32
#define EM_PLAN_INFO_TILE_NODES 0   /* nodes per tile */
#define EM_PLAN_INFO_TILES      1   /* number of tiles */
#define EM_PLAN_INFO_MAX_ELEMS  2   /* most elements in one tile */
#define EM_PLAN_INFO_MAX_NODES  3   /* most nodes (owned + halo) in one tile */
#define EM_PLAN_INFO_MAX_EDGES  4   /* most edges (owned + halo) in one tile */
#define EM_PLAN_INFO_MAX_OWNED_EDGES 5
#define EM_PLAN_INFO_MAX_BFACES 6
#define EM_PLAN_INFO_MAX_OWNED_BNODES 7
#define EM_PLAN_INFO_MAX_OWNED_NODES 8
#define EM_PLAN_INFO_CHECK      9   /* plan size in bytes, echoed for validation */
#define EM_PLAN_INFO_MAX_ESLOTS 10  /* most gather slots of one tile's owned edges */
#define EM_PLAN_INFO_MAX_NSLOTS 11  /* most gather slots of one tile's owned nodes */
#define EM_PLAN_INFO_MAX_BSLOTS 12  /* most gather slots of one tile's boundary nodes */
#define EM_PLAN_INFO_MAX_EDGE_VALENCE 13  /* most contributions to one edge (elements + boundary faces) */
#define EM_PLAN_INFO_MAX_NODE_VALENCE 14  /* most elements around one node */
/* scatter tiles (EM_PATH_TILED: each element computed once, by the tile of
 * its lowest node; partial sums for other tiles' targets go out as records) */
#define EM_PLAN_INFO_S_MAX_ELEMS  15  /* most elements of one scatter tile */
#define EM_PLAN_INFO_S_MAX_NODES  16  /* most local nodes (owned + halo) */
#define EM_PLAN_INFO_S_MAX_EDGES  17  /* most local edges (owned + halo) */
#define EM_PLAN_INFO_S_MAX_BNODES 18  /* most local boundary nodes (owned + halo) */
#define EM_PLAN_INFO_S_MAX_BFACES 19  /* most boundary faces of one scatter tile */
#define EM_PLAN_INFO_REC_NODES    20  /* node records (halo nodes of all tiles) */
#define EM_PLAN_INFO_REC_EDGES    21  /* edge records (halo edges of all tiles) */
#define EM_PLAN_INFO_REC_BNODES   22  /* boundary-node records */

/* em_plan_build -- tiled gather plan for EM_PATH_GATHER (run once per
 * connectivity, after em_edge_build).
 *
 * Nodes are cut into tiles of `tile_nodes` consecutive ids (a spatially
 * compact numbering, such as Morton order, keeps tiles compact).  A tile owns
 * its nodes, the edges whose lower end it owns and the boundary nodes among
 * its nodes; it processes every element and boundary face that touches one of
 * its nodes, so every output is produced by exactly one tile.
 *
 *   plan         device buffer of *plan_bytes bytes, written; call with
 *                plan == NULL to query the size (an upper bound from the
 *                counts; the bound needs no device work).
 *   tile_nodes   nodes per tile, 32..2048, multiple of 32 (0 = default 256).
 *   plan_info    HOST int64[EM_PLAN_INFO_LEN] or NULL, written on success:
 *                the summary to copy into em_mesh.plan_info.
 * Protocol (three calls, all synchronizing `stream`):
 *   1. ws == NULL            -> *ws_bytes = scratch for step 2;
 *   2. ws given, plan NULL   -> counts; *plan_bytes = exact plan size and
 *                               *ws_bytes = scratch for step 3;
 *   3. ws and plan given     -> builds the plan.
 * Errors: EM_ERR_ARG (bad sizes, a tile exceeding the 16-bit local index
 * limits: choose a smaller tile_nodes), EM_ERR_WORKSPACE, EM_ERR_CUDA.
 * The plan holds no device pointers: it is position-independent and may be
 * copied. */
int em_plan_build(int dim, int64_t n_nodes, int64_t n_elems, const int32_t* elems,
                  const int32_t* elem2edge,
                  int64_t n_edges, const int32_t* edges,
                  int64_t n_bfaces, const int32_t* bface, const int32_t* bface_owner,
                  int64_t n_bnodes, const int32_t* bnode,
                  int tile_nodes,
                  void* ws, size_t* ws_bytes,
                  void* plan, size_t* plan_bytes,
                  int64_t* plan_info,
                  void* stream);

/* ------------------------------------------------------------------------ */
/* Metrics                                                                   */
/* ------------------------------------------------------------------------ */

/* Mesh description passed to the metric entry points: device pointers from
 * em_edge_build (and em_plan_build for EM_PATH_GATHER). */
typedef struct em_mesh {
    int dim;
    int64_t n_nodes, n_elems, n_edges, n_bfaces, n_bnodes;
    const int32_t* elems;        /* [n_elems][4] */
    const int32_t* elem2edge;    /* [n_elems][nle] */
    const int32_t* edges;        /* [n_edges][2] */
    const int32_t* edge_ptr;     /* [n_edges+1], needed by EM_PATH_CSR only */
    const int32_t* edge_slot;    /* [n_elems*nle], needed by EM_PATH_CSR only */
    const int32_t* bface;        /* [n_bfaces][dim] */
    const int32_t* bface_owner;  /* [n_bfaces] */
    const int32_t* bnode;        /* [n_bnodes] */
    const void* plan;            /* from em_plan_build, needed by EM_PATH_GATHER only */
    size_t plan_bytes;
    int64_t plan_info[EM_PLAN_INFO_LEN]; /* host copy of the plan summary written by
                                    em_plan_build (GATHER path only); lets launches size
                                    their shared memory without reading the device */
} em_mesh;

/* em_edge_metrics -- forward: n_edge [n_edges][dim], vol [n_nodes],
 * bnormal [n_bnodes][dim] (all overwritten; any may be NULL to skip it on
 * the atomic path, all three are always produced on the gather paths).
 *   x          [n_nodes][dim] float64.
 *   precision  EM_PREC_*; path EM_PATH_*.  Supported pairs: ATOMIC with FP64,
 *              MIXED, MIXED_COMP32; GATHER and TILED with FP64, DW, MIXED; CSR
 *              with FP64.
 * Errors: EM_ERR_ARG (unsupported pair, missing plan/CSR), EM_ERR_WORKSPACE,
 * EM_ERR_CUDA.  Degenerate elements are not checked here (see
 * em_check_elements). */
int em_edge_metrics(const em_mesh* mesh, int precision, int path,
                    const double* x,
                    double* n_edge, double* vol, double* bnormal,
                    void* ws, size_t* ws_bytes, void* stream);

/* em_edge_metrics_adjoint -- grad_x [n_nodes][dim] (overwritten) =
 * d/dx ( sum_e w[e] . n_e + sum_i c[i] V_i + sum_b bw[b] . bnormal_b ),
 * w [n_edges][dim], c [n_nodes] (NULL: zero), bw [n_bnodes][dim] weights of
 * the boundary dual-face normals in mesh->bnode order (NULL: no such term;
 * not supported on the GATHER path).  The derivative of the paper's
 * equations (Eq. efficient_njk_formula_general_D with the boundary
 * correction, Sec. 4.2, Sec. 3.2.3).  Supported pairs: ATOMIC with FP64 or
 * MIXED; GATHER and TILED with FP64, DW, MIXED.  The workspace holds a
 * node -> boundary-node map used when bw is given. */
int em_edge_metrics_adjoint(const em_mesh* mesh, int precision, int path,
                            const double* x, const double* w, const double* c, const double* bw,
                            double* grad_x,
                            void* ws, size_t* ws_bytes, void* stream);

/* em_edge_metrics_fused -- forward outputs and the adjoint in one pass over
 * the grid (the adjoint does not depend on the forward outputs).  path:
 * EM_PATH_GATHER or EM_PATH_TILED (FP64, DW, MIXED); w, c, bw as in
 * em_edge_metrics_adjoint (bw only on the TILED path). */
int em_edge_metrics_fused(const em_mesh* mesh, int precision, int path,
                          const double* x, const double* w, const double* c, const double* bw,
                          double* n_edge, double* vol, double* bnormal, double* grad_x,
                          void* ws, size_t* ws_bytes, void* stream);

/* em_edge_volume -- the edge-based median-dual volume of Sec. 4.1,
 *   V_j = 1/(2D) sum_{edges {j,k}} (x_k - x_j) . n_jk,
 * from given lumped directed-area vectors n_edge [n_edges][dim] (for example
 * em_edge_metrics' output).  On a grid whose boundary faces are flat through
 * each of their nodes it equals the element-based volume, so it doubles as an
 * independent check of n_edge.  One thread per node sums its edges in
 * ascending edge id with explicitly rounded FP64 arithmetic, so the result is
 * the same floating-point expression as a serial edge loop.  vol [n_nodes] is
 * overwritten.  Needs only mesh->edges (and n_nodes, n_edges, dim); the
 * node-to-edge lists are built in the workspace. */
int em_edge_volume(const em_mesh* mesh, const double* x, const double* n_edge, double* vol,
                   void* ws, size_t* ws_bytes, void* stream);

/* em_edge_areas_traditional -- the directed-area vectors n_jk by the
 * TRADITIONAL construction the paper compares against (Sec. 3.1): in every
 * element, for every element edge, the dual-face part spanned by the edge
 * midpoint, the centroids of the two element faces that contain the edge and
 * the element centroid (2D: edge midpoint to element centroid), directed from
 * the lower to the higher node id; FP64, one thread per element, FP64 atomic
 * accumulation (so the summation order, and the last bits, vary from run to
 * run).  Equals em_edge_metrics' n_edge up to rounding.  Provided to measure
 * the paper's comparison on this GPU; n_edge [n_edges][dim] is overwritten.
 * Needs mesh->elems and mesh->elem2edge. */
int em_edge_areas_traditional(const em_mesh* mesh, const double* x, double* n_edge, void* stream);

/* em_edge_residual -- the edge-loop residual of the edge-based
 * discretization (Sec. 2) for a given nodal flux F [n_nodes][dim]:
 *   res_j = sum_{edges {j,k}} phi_jk - sum_{edges {i,j}} phi_ij + F_j . bnormal_j,
 *   phi_jk = sum_c 1/2 (F_j[c] + F_k[c]) n_jk[c]   (central flux),
 * the boundary term only at boundary nodes (bnormal [n_bnodes][dim] in
 * mesh->bnode order, as em_edge_metrics writes it).  For a linear F it equals
 * V_j div F at every interior node.  One thread per node sums its edges in
 * ascending edge id with explicitly rounded FP64 arithmetic (the same
 * expression as a serial edge loop).  res [n_nodes] is overwritten.  Needs
 * mesh->edges and mesh->bnode; lists are built in the workspace (size query
 * with ws == NULL). */
int em_edge_residual(const em_mesh* mesh, const double* F, const double* n_edge, const double* bnormal,
                     double* res, void* ws, size_t* ws_bytes, void* stream);

/* em_check_elements -- validation: counts elements with a node id outside
 * [0,n_nodes), a repeated node, or zero measure (det == 0 in FP64).
 *   ws       device workspace (size query with ws == NULL, as everywhere).
 *   counts   HOST int64[2] = {bad ids, degenerate}.
 * Returns EM_ERR_BAD_ID / EM_ERR_DEGENERATE when the respective count is
 * non-zero (degeneracy is only tested when every id is valid).
 * Synchronizes `stream`. */
int em_check_elements(int dim, int64_t n_nodes, int64_t n_elems, const int32_t* elems,
                      const double* x, void* ws, size_t* ws_bytes, int64_t* counts, void* stream);

/* em_edge_metrics_partial -- one rank's share of a grid split into
 * contiguous element ranges (multi-GPU partition of one grid).  Writes the
 * contributions of the elements [elem_begin, elem_end), and of the boundary
 * faces whose owner element (bface_owner / 4) lies in that range, to the
 * GLOBAL arrays: n_edge [n_edges][dim], vol [n_nodes], bnormal
 * [n_bnodes][dim] (forward) and grad_x [n_nodes][dim] (adjoint of L = sum
 * w.n + sum c V, c NULL: zero), each overwritten, zero where the range
 * contributes nothing.  The metrics are sums of per-element terms (Eq.
 * efficient_njk_formula_general_D, Sec. 4.2) and per-boundary-face terms
 * (the correction and closure of Sec. 3.2.3), so summing the partial arrays
 * of disjoint ranges that cover the grid (one all-reduce, or a reduce onto
 * the owner of each entry) gives the full result up to rounding order.
 * Element arithmetic as the ATOMIC path: precision EM_PREC_FP64 or
 * EM_PREC_MIXED, global FP64 atomics (the last bits vary from run to run),
 * no workspace.  Give the three forward outputs together or none of them;
 * grad_x NULL skips the adjoint (w is then unused).
 * Errors: EM_ERR_ARG (range outside [0, n_elems], bad precision, missing
 * arrays), EM_ERR_CUDA. */
int em_edge_metrics_partial(const em_mesh* mesh, int precision, int64_t elem_begin, int64_t elem_end,
                            const double* x, const double* w, const double* c,
                            double* n_edge, double* vol, double* bnormal, double* grad_x, void* stream);

/* ------------------------------------------------------------------------ */
/* Allocation-free forward                                                   */
/* ------------------------------------------------------------------------ */

/* Size of the fixed scratch array behind em_edge_metrics_noalloc: 64 MiB of
 * device memory that every GPU which loads this library's kernels keeps
 * reserved until the process exits.  With lazy module loading (the CUDA
 * default since 12.2) the array is committed when the module that holds it
 * is first loaded on a device: at the first em_edge_metrics_noalloc call
 * there (the address lookup), or at the first ATOMIC-path call of any entry
 * point.  Processes under a fixed memory cap should make one such call
 * during set-up; later calls commit nothing more. */
#define EM_NOALLOC_SCRATCH_BYTES (64ull * 1024ull * 1024ull)

/* em_edge_metrics_noalloc -- the forward outputs (n_edge, vol, bnormal, as
 * em_edge_metrics with EM_PATH_ATOMIC and EM_PREC_MIXED_COMP32) for callers
 * that cannot allocate device memory at call time: solver plug-ins and
 * callbacks whose host application owns every byte of device memory through
 * its own pool, processes running under a fixed device-memory cap, or code
 * paths where a cudaMalloc could fail or stall.  The paper has no counterpart:
 * this is a deployment variant of the compensated-FP32 atomic form.
 *
 * The two-float edge and node accumulators of that form live in a
 * library-owned array of EM_NOALLOC_SCRATCH_BYTES instead of a caller
 * workspace, so the call takes no workspace and never allocates (no
 * cudaMalloc, no cudaFree, no allocating library routine).  Requirement:
 * 4 * (2*dim*n_edges + 2*n_nodes) <= EM_NOALLOC_SCRATCH_BYTES, otherwise
 * EM_ERR_ARG and nothing is enqueued.
 *   - The first call on each device looks up the array's device address
 *     (once per device, with that device current), which loads the module
 *     and commits the 64 MiB if no ATOMIC-path call did so before; make that
 *     first call during set-up, before any stream capture begins.
 *   - The array is cleared on `stream` at the start of every call.  All calls
 *     share it, so calls whose work overlaps on the GPU (different streams or
 *     threads, same device) race and corrupt each other's results; serialize
 *     them.
 *   - n_edge, vol and bnormal must all be given.  Outputs match
 *     em_edge_metrics(ATOMIC, MIXED_COMP32) to its rounding (atomic order
 *     differs between runs). */
int em_edge_metrics_noalloc(const em_mesh* mesh, const double* x,
                            double* n_edge, double* vol, double* bnormal, void* stream);

/* ------------------------------------------------------------------------ */
/* Batched meshes                                                            */
/* ------------------------------------------------------------------------ */

/* One mesh of a batch: everything em_edge_metrics_fused needs (tile plan
 * required, mesh.plan_info filled) plus its inputs and outputs. */
typedef struct em_batch_item {
    em_mesh mesh;
    const double* x; const double* w; const double* c;
    double* n_edge; double* vol; double* bnormal; double* grad_x;
    void* rec;   /* DEVICE scratch of this grid's tile records: 32 *
                    (plan_info[EM_PLAN_INFO_REC_EDGES] + [REC_NODES] +
                    [REC_BNODES]) bytes, 8-byte aligned, owned by the caller;
                    no two items (and no concurrent call) may share one */
} em_batch_item;

/* Launch shapes of em_batched_fwd_adj (`blocks`). */
#define EM_BATCH_ITEM_GRID   0    /* one CTA per work item (the default, fastest) */
#define EM_BATCH_PERSISTENT (-1)  /* persistent: SMs x resident CTAs per SM */

/* em_batched_fwd_adj -- forward + adjoint (as em_edge_metrics_fused) for
 * n_meshes grids of uneven size in ONE launch.  The tiles of all grids form
 * one work list of (grid, tile) items; every item runs exactly as the
 * single-grid EM_PATH_TILED pass runs that tile (exact fixed-point
 * accumulation), so every output equals em_edge_metrics_fused(...,
 * EM_PATH_TILED) bit for bit, whatever the launch shape.  No block waits on
 * another block.  Grids with an edge valence above 340 or a node valence
 * above 170 are refused (EM_ERR_ARG), as in the tiled path.
 *   items        DEVICE array [n_meshes] of em_batch_item (pointers inside
 *                are device pointers); all grids must have the same dim.
 *   tile_prefix  DEVICE int64 [n_meshes+1]: exclusive prefix sum of the grids'
 *                tile counts (plan_info[EM_PLAN_INFO_TILES]).
 *   n_items      HOST: the number of work items, tile_prefix[n_meshes]
 *                (1 <= n_items < 2^31); it sizes the item grid.
 *   max_info     HOST int64 [EM_PLAN_INFO_LEN]: element-wise maximum of the
 *                grids' plan_info (sizes the shared memory of the launch).
 *   dim          dimension of every grid (2 or 3).
 *   blocks       EM_BATCH_ITEM_GRID (0): n_items CTAs, one per item, issued
 *                by the hardware in item order; > 0: that many persistent
 *                CTAs claiming items through an atomic counter;
 *                EM_BATCH_PERSISTENT (-1): persistent, SMs x resident CTAs.
 *   status       DEVICE int32[1], written: EM_OK, or EM_ERR_ARG if an item's
 *                dim differs from `dim`.
 * Workspace: a small counter (size query with ws == NULL).  The call reads
 * nothing back to the host and allocates nothing. */
int em_batched_fwd_adj(int n_meshes, const em_batch_item* items, const int64_t* tile_prefix, int64_t n_items,
                       const int64_t* max_info, int dim, int precision, int blocks, int32_t* status,
                       void* ws, size_t* ws_bytes, void* stream);

/* number of tiles in a plan (HOST read of the plan header; synchronizes) */
int em_plan_tiles(const void* plan, int64_t* n_tiles, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* EDGEMETRICS_H */

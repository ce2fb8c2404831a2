// Layout of the tiled gather plan (produced by em_plan_build, consumed by the
// tiled metric kernels).  All offsets are byte offsets from the plan start;
// the plan holds no pointers, so it can be copied freely.
//
// A tile owns the nodes [node0, node0 + n_own), the edges whose lower end it
// owns ([edge0, edge0 + n_eo): edges are sorted by their lower end) and the
// boundary nodes among its nodes ([bnode0, bnode0 + n_bo)).  Its elements are
// every element that touches an owned node, listed by ascending element id;
// their nodes are renumbered tile-locally (owned nodes first, then the sorted
// halo list) and each element's nodes are stored in ascending GLOBAL id, so
// that "lower end of an edge" is "lower local rank".  Tile edges are the owned
// edges followed by the sorted halo edges (edges of tile elements whose lower
// end is not owned).
//
// Gather lists (u16 entries, "slot" = (index << 2) | code):
//   eslot  per owned edge, ascending: element slots (tile element j, code p =
//          rank of the edge's lower end in the element, 0..2) followed by
//          boundary slots (tile boundary face j, code 3).
//   nslot  per node: (tile element j, rank r of the node in the element).
//   bslot  per boundary node: (tile boundary face j, position of the node in
//          the face's stored order).
//
// Scatter tiles (EM_PATH_TILED; the "s" sections): every element belongs to
// exactly one tile, the tile of its lowest node, and every boundary face to
// the tile of its owner element, so each element is computed once.  A
// scatter tile's local nodes are its owned nodes followed by the sorted
// nodes of its elements that it does not own ("halo" nodes: all of them lie
// in later tiles, because they are above the element's lowest node), its
// local edges the owned edges followed by the sorted non-owned edges of its
// elements, its local boundary nodes the owned ones followed by the sorted
// non-owned nodes of its boundary faces (as boundary-node indices).  Owned
// targets are written by the tile as outputs; every halo target's partial
// sum is written as a record at its position in the plan's halo list (so a
// tile's records are contiguous), and a merge pass adds the records of each
// target to the owner's output in ascending record order.
//   m*_id   targets that receive records (ascending global index),
//   m*_ptr  CSR offsets into m*_rec,
//   m*_rec  record indices (ascending tile order inside a target).
#pragma once
#include <stdint.h>

namespace em {

constexpr int64_t PLAN_MAGIC = 0x4e414c5054444745LL;  // "EGDTPLAN"
constexpr int64_t PLAN_VERSION = 2;

struct PlanHeader {
    int64_t magic, version, dim, tile_nodes, n_tiles;
    int64_t n_nodes, n_elems, n_edges, n_bfaces, n_bnodes;
    int64_t n_pairs, n_halo, n_hedge, n_tbf, n_eslot, n_nslot, n_bslot;
    int64_t max_el, max_nodes, max_edges, max_eo, max_bf, max_bo, max_own;
    int64_t off_tiles, off_conn, off_tedge, off_halo, off_hedge;
    int64_t off_eslot_ptr, off_eslot, off_nslot_ptr, off_nslot, off_tbf, off_bslot_ptr, off_bslot;
    // scatter tiles
    int64_t s_max_el, s_max_nodes, s_max_edges, s_max_bnodes, s_max_bf;
    int64_t n_shalo, n_shedge, n_shbo, n_me, n_mn, n_mb;
    int64_t off_stiles, off_sconn, off_stedge, off_shalo, off_shedge, off_shbo, off_sbf;
    int64_t off_me_id, off_me_ptr, off_me_rec, off_mn_id, off_mn_ptr, off_mn_rec, off_mb_id, off_mb_ptr, off_mb_rec;
};
static_assert(sizeof(PlanHeader) <= 512, "plan header too large");
constexpr int64_t PLAN_HEADER_BYTES = 512;

struct TileInfo {
    int32_t node0, n_own, edge0, n_eo;
    int32_t n_halo, n_hedge, bnode0, n_bo;
    int32_t elem_off, n_el, halo_off, hedge_off;
    int32_t bf_off, n_bf, pad0, pad1;
};
static_assert(sizeof(TileInfo) == 64, "TileInfo is 64 bytes");

// per tile element: 4 local node ids (ascending global id) and the local edge
// ids of the sorted-order edges (0,1),(0,2),(0,3),(1,2),(1,3),(2,3)
// (triangles: nodes 0..2, edges (0,1),(0,2),(1,2)).
struct ElemConn { uint16_t v[4]; };
struct ElemEdges { uint16_t e[8]; };
// tile boundary face: local nodes in stored (outward) order and local ids of
// its edges (f0,f1),(f1,f2),(f2,f0) (2D: the single edge in e[0])
struct TileBFace { uint16_t v[3]; uint16_t e[3]; uint16_t pad[2]; };

// scatter tile: owned ranges as in TileInfo; halo lists, elements and boundary
// faces of the scatter sections
struct STile {
    int32_t node0, n_own, edge0, n_eo;
    int32_t bnode0, n_bo, n_halo, n_hedge;
    int32_t n_hbo, elem_off, n_el, halo_off;
    int32_t hedge_off, hbo_off, bf_off, n_bf;
};
static_assert(sizeof(STile) == 64, "STile is 64 bytes");

// scatter boundary face: local nodes in stored (outward) order, local edges
// (f0,f1),(f1,f2),(f2,f0) (2D: the single edge in e[0]) and the local
// boundary-node ids of its nodes
struct SFace { uint16_t v[3]; uint16_t e[3]; uint16_t b[3]; uint16_t pad[3]; };
static_assert(sizeof(SFace) == 24, "SFace is 24 bytes");

// records: at most 4 doubles each (edges: n; nodes: V, grad; boundary nodes:
// bnormal), the bound that sizes a grid's record buffer
constexpr int REC_DOUBLES = 4;

template <typename T>
__host__ __device__ inline const T* plan_at(const void* plan, int64_t off) {
    return reinterpret_cast<const T*>(static_cast<const char*>(plan) + off);
}

}  // namespace em

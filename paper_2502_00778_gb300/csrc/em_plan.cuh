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
#pragma once
#include <stdint.h>

namespace em {

constexpr int64_t PLAN_MAGIC = 0x4e414c5054444745LL;  // "EGDTPLAN"
constexpr int64_t PLAN_VERSION = 1;

struct PlanHeader {
    int64_t magic, version, dim, tile_nodes, n_tiles;
    int64_t n_nodes, n_elems, n_edges, n_bfaces, n_bnodes;
    int64_t n_pairs, n_halo, n_hedge, n_tbf, n_eslot, n_nslot, n_bslot;
    int64_t max_el, max_nodes, max_edges, max_eo, max_bf, max_bo, max_own;
    int64_t off_tiles, off_conn, off_tedge, off_halo, off_hedge;
    int64_t off_eslot_ptr, off_eslot, off_nslot_ptr, off_nslot, off_tbf, off_bslot_ptr, off_bslot;
    int64_t reserved[20 - 0];
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

template <typename T>
__host__ __device__ inline const T* plan_at(const void* plan, int64_t off) {
    return reinterpret_cast<const T*>(static_cast<const char*>(plan) + off);
}

}  // namespace em

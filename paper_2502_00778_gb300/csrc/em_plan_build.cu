// em_plan_build: builds the tiled gather plan (layout in em_plan.cuh) on the
// GPU with the library's radix sort and scans.
//
// Call protocol (all sizes in bytes):
//   1. ws == NULL                 -> *ws_bytes = scratch needed by step 2.
//   2. ws, plan == NULL           -> counts everything; *plan_bytes = exact plan
//                                    size, *ws_bytes = scratch needed by step 3.
//   3. ws, plan                   -> builds the plan.
#include <algorithm>
#include <cstring>
#include <vector>

#include "em_common.cuh"
#include "em_kernels.cuh"
#include "em_plan.cuh"

namespace em {

namespace {

constexpr int NT = 256;

__device__ __forceinline__ int4 ld_el(const int32_t* e, int64_t i) { return reinterpret_cast<const int4*>(e)[i]; }
__device__ __forceinline__ int getc(const int4& v, int i) { return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w; }

// element nodes sorted by global id, with their stored positions
__device__ __forceinline__ void sorted_nodes(int dim, const int4& v4, int* v, int* pos) {
    const int k = dim + 1;
    for (int i = 0; i < k; i++) { v[i] = getc(v4, i); pos[i] = i; }
    for (int i = 1; i < k; i++) {
        int tv = v[i], tp = pos[i], j = i - 1;
        while (j >= 0 && v[j] > tv) { v[j + 1] = v[j]; pos[j + 1] = pos[j]; j--; }
        v[j + 1] = tv; pos[j + 1] = tp;
    }
}

// stored local edge index of the stored node pair {p, q}
__device__ __forceinline__ int stored_edge(int dim, int p, int q) {
    if (p > q) { int t = p; p = q; q = t; }
    if (dim == 3) return p == 0 ? q - 1 : (p == 1 ? q + 1 : 5);
    return p == 0 ? q - 1 : 2;
}

// sorted-order local edges and the rank of their lower end
__constant__ int c_se3[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
__constant__ int c_se2[3][2] = {{0, 1}, {0, 2}, {1, 2}};

__device__ __forceinline__ int distinct_tiles(int dim, const int* v, int T, int* t) {
    int n = 0;
    for (int i = 0; i < dim + 1; i++) {
        int ti = v[i] / T;
        bool seen = false;
        for (int j = 0; j < n; j++) seen |= (t[j] == ti);
        if (!seen) t[n++] = ti;
    }
    // ascending
    for (int i = 1; i < n; i++) {
        int x = t[i], j = i - 1;
        while (j >= 0 && t[j] > x) { t[j + 1] = t[j]; j--; }
        t[j + 1] = x;
    }
    return n;
}

template <typename T>
__device__ __forceinline__ int64_t lower_bound(const T* a, int64_t n, T key) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (a[mid] < key) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// first edge whose lower end is >= node
__device__ __forceinline__ int64_t edge_lower_bound(const int32_t* edges, int64_t ne, int32_t node) {
    int64_t lo = 0, hi = ne;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (edges[2 * mid] < node) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ int64_t find_edge(const int32_t* edges, int64_t ne, int32_t a, int32_t b) {
    int32_t j = a < b ? a : b, k = a < b ? b : a;
    int64_t lo = 0, hi = ne - 1;
    while (lo <= hi) {
        int64_t mid = (lo + hi) >> 1;
        int32_t p = edges[2 * mid], q = edges[2 * mid + 1];
        if (p == j && q == k) return mid;
        if (p < j || (p == j && q < k)) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

#define GRID_LOOP(i, n) for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < (n); i += int64_t(gridDim.x) * blockDim.x)

// ---- counting ---------------------------------------------------------------
// per element: number of distinct tiles, halo-node and halo-edge candidates
__global__ void k_count_elem(int dim, int64_t ne, const int32_t* elems, const int32_t* e2e, const int32_t* edges,
                             int T, int32_t* npair, int32_t* nhalo, int32_t* nhedge, int32_t* tile_cnt) {
    const int nle = dim == 3 ? 6 : 3;
    GRID_LOOP(E, ne) {
        int v[4], pos[4], t[4];
        sorted_nodes(dim, ld_el(elems, E), v, pos);
        int nt = distinct_tiles(dim, v, T, t);
        int h = 0, he = 0;
        for (int a = 0; a < nt; a++) {
            atomicAdd(&tile_cnt[t[a]], 1);
            for (int i = 0; i < dim + 1; i++) h += (v[i] / T != t[a]);
            for (int l = 0; l < nle; l++) {
                int32_t e = e2e[E * nle + l];
                he += (edges[2 * int64_t(e)] / T != t[a]);
            }
        }
        npair[E] = nt;
        nhalo[E] = h;
        nhedge[E] = he;
    }
}

// per boundary face: number of distinct tiles
__global__ void k_count_bface(int dim, int64_t nbf, const int32_t* bface, int T, int32_t* nbp) {
    GRID_LOOP(B, nbf) {
        int v[3], t[4];
        for (int i = 0; i < dim; i++) v[i] = bface[dim * B + i];
        int n = 0;
        for (int i = 0; i < dim; i++) {
            int ti = v[i] / T;
            bool seen = false;
            for (int j = 0; j < n; j++) seen |= (t[j] == ti);
            if (!seen) t[n++] = ti;
        }
        nbp[B] = n;
    }
}

// ---- pairs ------------------------------------------------------------------
// key = tile << 9 | owned mask << 5 | (element id mod 32) (mask bit r: the
// r-th smallest node of the element belongs to the tile).  Sorting by it
// groups a tile's elements by which of their nodes (and hence, by lower end,
// which of their edges) the tile owns, so the threads of a warp mostly share
// one mask and skip the same outputs; inside a group, elements whose ids
// differ by a multiple of 32 come together, so the 32 elements a warp takes
// lie far apart on the (spatially ordered) grid and rarely add into the same
// node or edge in one atomic instruction.
__global__ void k_fill_pairs(int dim, int64_t ne, const int32_t* elems, int T, const int64_t* off, uint64_t* keys,
                             uint32_t* vals) {
    GRID_LOOP(E, ne) {
        int v[4], pos[4], t[4];
        sorted_nodes(dim, ld_el(elems, E), v, pos);
        int nt = distinct_tiles(dim, v, T, t);
        int64_t o = off[E];
        for (int a = 0; a < nt; a++) {
            unsigned mask = 0;
            for (int r = 0; r <= dim; r++)
                if (v[r] / T == t[a]) mask |= 1u << r;
            keys[o + a] = ((uint64_t)t[a] << 9) | (mask << 5) | ((uint64_t)E & 31u);
            vals[o + a] = (uint32_t)E;
        }
    }
}
__global__ void k_key_drop_mask(int64_t n, uint64_t* keys) {
    GRID_LOOP(i, n) keys[i] >>= 9;
}

__global__ void k_fill_bpairs(int dim, int64_t nbf, const int32_t* bface, int T, const int64_t* off, uint64_t* keys,
                              uint32_t* vals, int32_t* tbf_cnt) {
    GRID_LOOP(B, nbf) {
        int t[3], n = 0;
        for (int i = 0; i < dim; i++) {
            int ti = bface[dim * B + i] / T;
            bool seen = false;
            for (int j = 0; j < n; j++) seen |= (t[j] == ti);
            if (!seen) t[n++] = ti;
        }
        for (int i = 1; i < n; i++) {
            int x = t[i], j = i - 1;
            while (j >= 0 && t[j] > x) { t[j + 1] = t[j]; j--; }
            t[j + 1] = x;
        }
        int64_t o = off[B];
        for (int a = 0; a < n; a++) {
            keys[o + a] = (uint64_t)t[a];
            vals[o + a] = (uint32_t)B;
            atomicAdd(&tbf_cnt[t[a]], 1);
        }
    }
}

// halo-node / halo-edge candidates of every (tile, element) pair, counted per pair
__global__ void k_pair_counts(int dim, int64_t P, const uint64_t* pkey, const uint32_t* pval, const int32_t* elems,
                              const int32_t* e2e, const int32_t* edges, int T, int32_t* hc, int32_t* hec) {
    const int nle = dim == 3 ? 6 : 3;
    GRID_LOOP(i, P) {
        int t = (int)pkey[i];
        int64_t E = pval[i];
        int4 v4 = ld_el(elems, E);
        int h = 0, he = 0;
        for (int a = 0; a < dim + 1; a++) h += (getc(v4, a) / T != t);
        for (int l = 0; l < nle; l++) he += (edges[2 * int64_t(e2e[E * nle + l])] / T != t);
        hc[i] = h;
        hec[i] = he;
    }
}

__global__ void k_fill_halo(int dim, int64_t P, const uint64_t* pkey, const uint32_t* pval, const int32_t* elems,
                            const int32_t* e2e, const int32_t* edges, int T, int bn, int be, const int64_t* hoff,
                            const int64_t* heoff, uint64_t* hk, uint32_t* hv, uint64_t* hek, uint32_t* hev) {
    const int nle = dim == 3 ? 6 : 3;
    GRID_LOOP(i, P) {
        uint64_t t = pkey[i];
        int64_t E = pval[i];
        int4 v4 = ld_el(elems, E);
        int64_t o = hoff[i];
        for (int a = 0; a < dim + 1; a++) {
            int v = getc(v4, a);
            if (v / T != (int)t) { hk[o] = (t << bn) | (uint64_t)v; hv[o] = 0; o++; }
        }
        o = heoff[i];
        for (int l = 0; l < nle; l++) {
            int32_t e = e2e[E * nle + l];
            if (edges[2 * int64_t(e)] / T != (int)t) { hek[o] = (t << be) | (uint64_t)e; hev[o] = 0; o++; }
        }
    }
}

__global__ void k_heads64(const uint64_t* k, int64_t n, int32_t* head) {
    GRID_LOOP(i, n) head[i] = (i == 0 || k[i] != k[i - 1]) ? 1 : 0;
}

__global__ void k_compact_unique(const uint64_t* k, int64_t n, int bits, const int32_t* head, const int64_t* pos,
                                 int32_t* out, int32_t* tile_cnt) {
    const uint64_t mask = (uint64_t(1) << bits) - 1;
    GRID_LOOP(i, n) {
        if (!head[i]) continue;
        out[pos[i]] = (int32_t)(k[i] & mask);
        atomicAdd(&tile_cnt[(int)(k[i] >> bits)], 1);
    }
}

// ---- tile info ----------------------------------------------------------------
__global__ void k_tile_info(int64_t n_tiles, int T, int64_t nv, const int32_t* edges, int64_t n_edges,
                            const int32_t* bnode, int64_t nbn, const int64_t* el_off, const int64_t* halo_off,
                            const int64_t* hedge_off, const int64_t* tbf_off, TileInfo* tiles, int64_t* maxv,
                            unsigned long long* status) {
    GRID_LOOP(t, n_tiles) {
        TileInfo ti;
        int64_t n0 = t * T, n1 = n0 + T < nv ? n0 + T : nv;
        int64_t e0 = edge_lower_bound(edges, n_edges, (int32_t)n0);
        int64_t e1 = edge_lower_bound(edges, n_edges, (int32_t)n1);
        int64_t b0 = nbn ? lower_bound<int32_t>(bnode, nbn, (int32_t)n0) : 0;
        int64_t b1 = nbn ? lower_bound<int32_t>(bnode, nbn, (int32_t)n1) : 0;
        ti.node0 = (int32_t)n0; ti.n_own = (int32_t)(n1 - n0);
        ti.edge0 = (int32_t)e0; ti.n_eo = (int32_t)(e1 - e0);
        ti.n_halo = (int32_t)(halo_off[t + 1] - halo_off[t]);
        ti.n_hedge = (int32_t)(hedge_off[t + 1] - hedge_off[t]);
        ti.bnode0 = (int32_t)b0; ti.n_bo = (int32_t)(b1 - b0);
        ti.elem_off = (int32_t)el_off[t]; ti.n_el = (int32_t)(el_off[t + 1] - el_off[t]);
        ti.halo_off = (int32_t)halo_off[t]; ti.hedge_off = (int32_t)hedge_off[t];
        ti.bf_off = (int32_t)tbf_off[t]; ti.n_bf = (int32_t)(tbf_off[t + 1] - tbf_off[t]);
        ti.pad0 = ti.pad1 = 0;
        tiles[t] = ti;
        if (ti.n_el > 16383 || ti.n_bf > 16383 || ti.n_own + ti.n_halo > 65535 || ti.n_eo + ti.n_hedge > 65534)
            atomicAdd(status, 1ull);
        atomicMax((unsigned long long*)&maxv[0], (unsigned long long)ti.n_el);
        atomicMax((unsigned long long*)&maxv[1], (unsigned long long)(ti.n_own + ti.n_halo));
        atomicMax((unsigned long long*)&maxv[2], (unsigned long long)(ti.n_eo + ti.n_hedge));
        atomicMax((unsigned long long*)&maxv[3], (unsigned long long)ti.n_eo);
        atomicMax((unsigned long long*)&maxv[4], (unsigned long long)ti.n_bf);
        atomicMax((unsigned long long*)&maxv[5], (unsigned long long)ti.n_bo);
        atomicMax((unsigned long long*)&maxv[6], (unsigned long long)ti.n_own);
    }
}

__device__ __forceinline__ int local_node(const TileInfo& ti, const int32_t* halo, int v) {
    if (v >= ti.node0 && v < ti.node0 + ti.n_own) return v - ti.node0;
    return ti.n_own + (int)lower_bound<int32_t>(halo + ti.halo_off, ti.n_halo, v);
}

__device__ __forceinline__ int local_edge(const TileInfo& ti, const int32_t* hedge, int32_t e) {
    if (e >= ti.edge0 && e < ti.edge0 + ti.n_eo) return e - ti.edge0;
    return ti.n_eo + (int)lower_bound<int32_t>(hedge + ti.hedge_off, ti.n_hedge, e);
}

// per pair: slot counts (edges with owned lower end, owned nodes)
__global__ void k_pair_slot_counts(int dim, int64_t P, const uint64_t* pkey, const uint32_t* pval,
                                   const int32_t* elems, int T, int32_t* ec, int32_t* nc) {
    GRID_LOOP(i, P) {
        int t = (int)pkey[i];
        int v[4], pos[4];
        sorted_nodes(dim, ld_el(elems, pval[i]), v, pos);
        int e = 0, n = 0;
        for (int r = 0; r < dim + 1; r++) {
            bool own = (v[r] / T == t);
            n += own;
            if (own) e += dim - r;   // edges (r, s), s > r
        }
        ec[i] = e;
        nc[i] = n;
    }
}

__global__ void k_elem_records(int dim, int64_t P, const uint64_t* pkey, const uint32_t* pval, const int32_t* elems,
                               const int32_t* e2e, const TileInfo* tiles, const int32_t* halo, const int32_t* hedge,
                               int T, const int64_t* ecoff, const int64_t* ncoff, ElemConn* conn, ElemEdges* tedge,
                               uint64_t* esk, uint32_t* esv, uint64_t* nsk, uint32_t* nsv) {
    const int nle = dim == 3 ? 6 : 3;
    GRID_LOOP(i, P) {
        int t = (int)pkey[i];
        int64_t E = pval[i];
        TileInfo ti = tiles[t];
        uint32_t j = (uint32_t)(i - ti.elem_off);
        int v[4], pos[4];
        sorted_nodes(dim, ld_el(elems, E), v, pos);
        ElemConn c;
        c.v[3] = 0xffff;
        for (int r = 0; r < dim + 1; r++) c.v[r] = (uint16_t)local_node(ti, halo, v[r]);
        conn[i] = c;
        ElemEdges ed;
        for (int q = 0; q < 8; q++) ed.e[q] = 0xffff;
        int64_t eo = ecoff[i], no = ncoff[i];
        for (int s = 0; s < nle; s++) {
            int p = dim == 3 ? c_se3[s][0] : c_se2[s][0];
            int q = dim == 3 ? c_se3[s][1] : c_se2[s][1];
            int32_t e = e2e[E * nle + stored_edge(dim, pos[p], pos[q])];
            ed.e[s] = (uint16_t)local_edge(ti, hedge, e);
            if (v[p] / T == t) { esk[eo] = (uint64_t)e; esv[eo] = (j << 2) | (uint32_t)p; eo++; }
        }
        tedge[i] = ed;
        for (int r = 0; r < dim + 1; r++)
            if (v[r] / T == t) { nsk[no] = (uint64_t)v[r]; nsv[no] = (j << 2) | (uint32_t)r; no++; }
    }
}

// boundary faces of a tile: records, boundary edge slots, boundary node slots
__global__ void k_bface_counts(int dim, int64_t BP, const uint64_t* bkey, const uint32_t* bval, const int32_t* bface,
                               const int32_t* edges, int T, int32_t* ec, int32_t* nc) {
    GRID_LOOP(i, BP) {
        int t = (int)bkey[i];
        int64_t B = bval[i];
        int e = 0, n = 0;
        for (int a = 0; a < dim; a++) {
            int v = bface[dim * B + a];
            n += (v / T == t);
            if (dim == 3 || a == 0) {
                int w = bface[dim * B + (a + 1) % dim];
                int lo = v < w ? v : w;
                e += (lo / T == t);
            }
        }
        ec[i] = e;
        nc[i] = n;
    }
}

__global__ void k_bface_records(int dim, int64_t BP, const uint64_t* bkey, const uint32_t* bval, const int32_t* bface,
                                const int32_t* edges, int64_t n_edges, const int32_t* bnode, int64_t nbn,
                                const TileInfo* tiles, const int32_t* halo, const int32_t* hedge, int T,
                                const int64_t* ecoff, const int64_t* ncoff, int64_t es_base, TileBFace* tbf,
                                uint64_t* esk, uint32_t* esv, uint64_t* bsk, uint32_t* bsv) {
    GRID_LOOP(i, BP) {
        int t = (int)bkey[i];
        int64_t B = bval[i];
        TileInfo ti = tiles[t];
        uint32_t j = (uint32_t)(i - ti.bf_off);
        TileBFace r;
        for (int q = 0; q < 3; q++) { r.v[q] = 0xffff; r.e[q] = 0xffff; }
        r.pad[0] = r.pad[1] = 0;
        int64_t eo = es_base + ecoff[i], no = ncoff[i];
        for (int a = 0; a < dim; a++) {
            int v = bface[dim * B + a];
            r.v[a] = (uint16_t)local_node(ti, halo, v);
            if (dim == 3 || a == 0) {
                int w = bface[dim * B + (a + 1) % dim];
                int64_t e = find_edge(edges, n_edges, v, w);
                r.e[a] = (uint16_t)local_edge(ti, hedge, (int32_t)e);
                int lo = v < w ? v : w;
                if (lo / T == t) { esk[eo] = (uint64_t)e; esv[eo] = (j << 2) | 3u; eo++; }
            }
            if (v / T == t) {
                bsk[no] = (uint64_t)lower_bound<int32_t>(bnode, nbn, v);
                bsv[no] = (j << 2) | (uint32_t)a;
                no++;
            }
        }
        tbf[i] = r;
    }
}

__global__ void k_tile_slot_max(int64_t n_tiles, const TileInfo* tiles, const int32_t* eptr, const int32_t* nptr,
                                const int32_t* bptr, int64_t* maxv) {
    GRID_LOOP(t, n_tiles) {
        TileInfo ti = tiles[t];
        atomicMax((unsigned long long*)&maxv[0], (unsigned long long)(eptr[ti.edge0 + ti.n_eo] - eptr[ti.edge0]));
        atomicMax((unsigned long long*)&maxv[1], (unsigned long long)(nptr[ti.node0 + ti.n_own] - nptr[ti.node0]));
        if (bptr)
            atomicMax((unsigned long long*)&maxv[2], (unsigned long long)(bptr[ti.bnode0 + ti.n_bo] - bptr[ti.bnode0]));
    }
}

// largest run length ptr[i+1] - ptr[i]: a warp reduction, then one atomic
// per warp (one atomic per element on a single address would serialise)
__global__ void k_max_run(const int32_t* ptr, int64_t n, int64_t* maxv) {
    unsigned m = 0u;
    GRID_LOOP(i, n) m = max(m, (unsigned)(ptr[i + 1] - ptr[i]));
    m = __reduce_max_sync(0xffffffffu, m);
    if ((threadIdx.x & 31) == 0 && m) atomicMax((unsigned long long*)maxv, (unsigned long long)m);
}

__global__ void k_key_counts(const uint64_t* k, int64_t n, int32_t* cnt) {
    GRID_LOOP(i, n) atomicAdd(&cnt[k[i]], 1);
}

__global__ void k_u32_to_u16(const uint32_t* a, int64_t n, uint16_t* b) {
    GRID_LOOP(i, n) b[i] = (uint16_t)a[i];
}

__global__ void k_i64_to_i32(const int64_t* a, int64_t n, int32_t* b) {
    GRID_LOOP(i, n) b[i] = (int32_t)a[i];
}

// ---- scatter tiles ------------------------------------------------------------
// element -> tile of its lowest node; key = tile << 5 | (element id mod 32):
// a stable sort by it lists a tile's elements residue class by residue class
// (ascending id inside a class), so the 32 elements a warp takes lie far
// apart on the spatially ordered grid and rarely add into the same target in
// one shared-memory atomic instruction.  Also counts, per element, the
// candidates of the tile's halo lists (nodes and edges the tile does not own).
__global__ void k_s_pairs(int dim, int64_t ne, const int32_t* elems, const int32_t* e2e, const int32_t* edges, int T,
                          uint64_t* key, uint32_t* val, int32_t* tile_cnt, int32_t* hn, int32_t* he) {
    const int nle = dim == 3 ? 6 : 3;
    GRID_LOOP(E, ne) {
        const int4 v4 = ld_el(elems, E);
        int lo = v4.x;
        for (int i = 1; i <= dim; i++) lo = min(lo, getc(v4, i));
        const int a = lo / T;
        key[E] = ((uint64_t)a << 5) | ((uint64_t)E & 31u);
        val[E] = (uint32_t)E;
        atomicAdd(&tile_cnt[a], 1);
        int h = 0, g = 0;
        for (int i = 0; i <= dim; i++) h += (getc(v4, i) / T != a);
        for (int l = 0; l < nle; l++) g += (edges[2 * int64_t(e2e[E * nle + l])] / T != a);
        hn[E] = h;
        he[E] = g;
    }
}

// candidates of the halo nodes (hk != NULL) or of the halo edges (hek != NULL)
__global__ void k_s_halo(int dim, int64_t ne, const int32_t* elems, const int32_t* e2e, const int32_t* edges, int T,
                         int bn, int be, const int64_t* hoff, const int64_t* heoff, uint64_t* hk, uint32_t* hv,
                         uint64_t* hek, uint32_t* hev) {
    const int nle = dim == 3 ? 6 : 3;
    GRID_LOOP(E, ne) {
        const int4 v4 = ld_el(elems, E);
        int lo = v4.x;
        for (int i = 1; i <= dim; i++) lo = min(lo, getc(v4, i));
        const uint64_t a = (uint64_t)(lo / T);
        if (hk) {
            int64_t o = hoff[E];
            for (int i = 0; i <= dim; i++) {
                const int v = getc(v4, i);
                if (v / T != (int)a) { hk[o] = (a << bn) | (uint64_t)v; hv[o] = 0; o++; }
            }
        }
        if (hek) {
            int64_t o = heoff[E];
            for (int l = 0; l < nle; l++) {
                const int32_t e = e2e[E * nle + l];
                if (edges[2 * int64_t(e)] / T != (int)a) { hek[o] = (a << be) | (uint64_t)e; hev[o] = 0; o++; }
            }
        }
    }
}

// tile of a boundary face's owner element (the owner's lowest node)
__device__ __forceinline__ int face_tile(int dim, const int32_t* elems, const int32_t* bowner, int64_t B, int T) {
    const int4 v4 = ld_el(elems, bowner[B] >> 2);
    int lo = v4.x;
    for (int i = 1; i <= dim; i++) lo = min(lo, getc(v4, i));
    return lo / T;
}

__global__ void k_s_faces(int dim, int64_t nbf, const int32_t* elems, const int32_t* bface, const int32_t* bowner,
                          int T, uint64_t* key, uint32_t* val, int32_t* tile_cnt, int32_t* hb) {
    GRID_LOOP(B, nbf) {
        const int a = face_tile(dim, elems, bowner, B, T);
        key[B] = (uint64_t)a;
        val[B] = (uint32_t)B;
        atomicAdd(&tile_cnt[a], 1);
        int h = 0;
        for (int i = 0; i < dim; i++) h += (bface[dim * B + i] / T != a);
        hb[B] = h;
    }
}

__global__ void k_s_face_halo(int dim, int64_t nbf, const int32_t* elems, const int32_t* bface, const int32_t* bowner,
                              const int32_t* bnode, int64_t nbn, int T, int bb, const int64_t* hoff, uint64_t* hk,
                              uint32_t* hv) {
    GRID_LOOP(B, nbf) {
        const uint64_t a = (uint64_t)face_tile(dim, elems, bowner, B, T);
        int64_t o = hoff[B];
        for (int i = 0; i < dim; i++) {
            const int v = bface[dim * B + i];
            if (v / T != (int)a) {
                hk[o] = (a << bb) | (uint64_t)lower_bound<int32_t>(bnode, nbn, v);
                hv[o] = 0;
                o++;
            }
        }
    }
}

// merge pairs: (target, record index) with the record index = position in the
// tile-major halo list
__global__ void k_s_merge_pairs(const int32_t* list, int64_t n, uint64_t* key, uint32_t* val) {
    GRID_LOOP(i, n) {
        key[i] = (uint64_t)(uint32_t)list[i];
        val[i] = (uint32_t)i;
    }
}

__global__ void k_s_u64_low32(const uint64_t* k, int64_t n, int32_t* out) {
    GRID_LOOP(i, n) out[i] = (int32_t)(uint32_t)k[i];
}

__global__ void k_s_tile_info(int64_t n_tiles, int T, int64_t nv, const int32_t* edges, int64_t n_edges,
                              const int32_t* bnode, int64_t nbn, const int64_t* el_off, const int64_t* halo_off,
                              const int64_t* hedge_off, const int64_t* hbo_off, const int64_t* bf_off, STile* tiles,
                              int64_t* maxv, unsigned long long* status) {
    GRID_LOOP(t, n_tiles) {
        STile ti;
        const int64_t n0 = t * T, n1 = n0 + T < nv ? n0 + T : nv;
        const int64_t e0 = edge_lower_bound(edges, n_edges, (int32_t)n0);
        const int64_t e1 = edge_lower_bound(edges, n_edges, (int32_t)n1);
        const int64_t b0 = nbn ? lower_bound<int32_t>(bnode, nbn, (int32_t)n0) : 0;
        const int64_t b1 = nbn ? lower_bound<int32_t>(bnode, nbn, (int32_t)n1) : 0;
        ti.node0 = (int32_t)n0; ti.n_own = (int32_t)(n1 - n0);
        ti.edge0 = (int32_t)e0; ti.n_eo = (int32_t)(e1 - e0);
        ti.bnode0 = (int32_t)b0; ti.n_bo = (int32_t)(b1 - b0);
        ti.n_halo = (int32_t)(halo_off[t + 1] - halo_off[t]);
        ti.n_hedge = (int32_t)(hedge_off[t + 1] - hedge_off[t]);
        ti.n_hbo = (int32_t)(hbo_off[t + 1] - hbo_off[t]);
        ti.elem_off = (int32_t)el_off[t]; ti.n_el = (int32_t)(el_off[t + 1] - el_off[t]);
        ti.halo_off = (int32_t)halo_off[t]; ti.hedge_off = (int32_t)hedge_off[t]; ti.hbo_off = (int32_t)hbo_off[t];
        ti.bf_off = (int32_t)bf_off[t]; ti.n_bf = (int32_t)(bf_off[t + 1] - bf_off[t]);
        tiles[t] = ti;
        const int64_t ln = int64_t(ti.n_own) + ti.n_halo, le = int64_t(ti.n_eo) + ti.n_hedge,
                      lb = int64_t(ti.n_bo) + ti.n_hbo;
        if (ln > 65535 || le > 65535 || lb > 65535) atomicAdd(status, 1ull);
        atomicMax((unsigned long long*)&maxv[0], (unsigned long long)ti.n_el);
        atomicMax((unsigned long long*)&maxv[1], (unsigned long long)ln);
        atomicMax((unsigned long long*)&maxv[2], (unsigned long long)le);
        atomicMax((unsigned long long*)&maxv[3], (unsigned long long)lb);
        atomicMax((unsigned long long*)&maxv[4], (unsigned long long)ti.n_bf);
    }
}

__device__ __forceinline__ int s_local_node(const STile& ti, const int32_t* halo, int v) {
    if (v >= ti.node0 && v < ti.node0 + ti.n_own) return v - ti.node0;
    return ti.n_own + (int)lower_bound<int32_t>(halo + ti.halo_off, ti.n_halo, v);
}

__device__ __forceinline__ int s_local_edge(const STile& ti, const int32_t* hedge, int32_t e) {
    if (e >= ti.edge0 && e < ti.edge0 + ti.n_eo) return e - ti.edge0;
    return ti.n_eo + (int)lower_bound<int32_t>(hedge + ti.hedge_off, ti.n_hedge, e);
}

__device__ __forceinline__ int s_local_bnode(const STile& ti, const int32_t* hbo, int32_t b) {
    if (b >= ti.bnode0 && b < ti.bnode0 + ti.n_bo) return b - ti.bnode0;
    return ti.n_bo + (int)lower_bound<int32_t>(hbo + ti.hbo_off, ti.n_hbo, b);
}

// element records of the scatter tiles, at their sorted positions
__global__ void k_s_elem_records(int dim, int64_t ne, const uint64_t* key, const uint32_t* val, const int32_t* elems,
                                 const int32_t* e2e, const STile* tiles, const int32_t* halo, const int32_t* hedge,
                                 ElemConn* conn, ElemEdges* tedge) {
    const int nle = dim == 3 ? 6 : 3;
    GRID_LOOP(i, ne) {
        const STile ti = tiles[key[i] >> 5];
        const int64_t E = val[i];
        int v[4], pos[4];
        sorted_nodes(dim, ld_el(elems, E), v, pos);
        ElemConn c;
        c.v[3] = 0xffff;
        for (int r = 0; r <= dim; r++) c.v[r] = (uint16_t)s_local_node(ti, halo, v[r]);
        conn[i] = c;
        ElemEdges ed;
        for (int q = 0; q < 8; q++) ed.e[q] = 0xffff;
        for (int s2 = 0; s2 < nle; s2++) {
            const int p = dim == 3 ? c_se3[s2][0] : c_se2[s2][0];
            const int q = dim == 3 ? c_se3[s2][1] : c_se2[s2][1];
            const int32_t e = e2e[E * nle + stored_edge(dim, pos[p], pos[q])];
            ed.e[s2] = (uint16_t)s_local_edge(ti, hedge, e);
        }
        tedge[i] = ed;
    }
}

__global__ void k_s_face_records(int dim, int64_t nbf, const uint64_t* key, const uint32_t* val, const int32_t* bface,
                                 const int32_t* edges, int64_t n_edges, const int32_t* bnode, int64_t nbn,
                                 const STile* tiles, const int32_t* halo, const int32_t* hedge, const int32_t* hbo,
                                 SFace* sbf) {
    GRID_LOOP(i, nbf) {
        const STile ti = tiles[key[i]];
        const int64_t B = val[i];
        SFace r;
        for (int q = 0; q < 3; q++) { r.v[q] = 0xffff; r.e[q] = 0xffff; r.b[q] = 0xffff; r.pad[q] = 0; }
        for (int a = 0; a < dim; a++) {
            const int v = bface[dim * B + a];
            r.v[a] = (uint16_t)s_local_node(ti, halo, v);
            r.b[a] = (uint16_t)s_local_bnode(ti, hbo, (int32_t)lower_bound<int32_t>(bnode, nbn, v));
            if (dim == 3 || a == 0) {
                const int w = bface[dim * B + (a + 1) % dim];
                r.e[a] = (uint16_t)s_local_edge(ti, hedge, (int32_t)find_edge(edges, n_edges, v, w));
            }
        }
        sbf[i] = r;
    }
}

// merge CSR of sorted (target, record) pairs: heads -> unique targets and
// their first pair
__global__ void k_s_merge_csr(const uint64_t* k, const uint32_t* v, int64_t n, const int32_t* head, const int64_t* pos,
                              int32_t* m_id, int32_t* m_ptr, int32_t* m_rec) {
    GRID_LOOP(i, n) {
        if (head[i]) {
            m_id[pos[i]] = (int32_t)(uint32_t)k[i];
            m_ptr[pos[i]] = (int32_t)i;
        }
        m_rec[i] = (int32_t)v[i];
    }
}

#undef GRID_LOOP

inline unsigned G(int64_t n) { return grid_for(n, NT); }

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

struct PlanOffsets {
    int64_t tiles, conn, tedge, halo, hedge, eslot_ptr, eslot, nslot_ptr, nslot, tbf, bslot_ptr, bslot, total;
};

PlanOffsets plan_offsets(int64_t n_tiles, int64_t nv, int64_t n_edges, int64_t nbn, int64_t P, int64_t n_halo,
                         int64_t n_hedge, int64_t ES, int64_t NS, int64_t BP, int64_t BS) {
    PlanOffsets o;
    size_t p = PLAN_HEADER_BYTES;
    auto take = [&](size_t bytes) { p = align256(p); int64_t r = (int64_t)p; p += bytes; return r; };
    o.tiles = take(sizeof(TileInfo) * n_tiles);
    o.conn = take(sizeof(ElemConn) * P);
    o.tedge = take(sizeof(ElemEdges) * P);
    o.halo = take(4 * n_halo);
    o.hedge = take(4 * n_hedge);
    o.eslot_ptr = take(4 * (n_edges + 1));
    o.eslot = take(2 * ES);
    o.nslot_ptr = take(4 * (nv + 1));
    o.nslot = take(2 * NS);
    o.tbf = take(sizeof(TileBFace) * BP);
    o.bslot_ptr = take(4 * (nbn + 1));
    o.bslot = take(2 * BS);
    o.total = (int64_t)align256(p);
    return o;
}

// counts -> int32 CSR offsets (n+1 entries)
int csr_from_keys(uint64_t* keys, int64_t n, int64_t nkeys, int32_t* cnt, int64_t* off64, int32_t* ptr, void* scan_ws,
                  cudaStream_t s) {
    EM_CUDA_TRY(cudaMemsetAsync(cnt, 0, 4 * (nkeys + 1), s));
    if (n) k_key_counts<<<G(n), NT, 0, s>>>(keys, n, cnt);
    EM_TRY(exclusive_scan_i32_to_i64(cnt, off64, nkeys, scan_ws, s));
    k_i64_to_i32<<<G(nkeys + 1), NT, 0, s>>>(off64, nkeys + 1, ptr);
    EM_CUDA_TRY(cudaGetLastError());
    return EM_OK;
}

// ---- scatter tiles: host side ---------------------------------------------------
struct SCounts {
    int64_t n_halo = 0, n_hedge = 0, n_hbo = 0, n_me = 0, n_mn = 0, n_mb = 0;
};

struct SOffsets {
    int64_t tiles, conn, tedge, halo, hedge, hbo, sbf, me_id, me_ptr, me_rec, mn_id, mn_ptr, mn_rec, mb_id, mb_ptr,
        mb_rec, total;
};

SOffsets s_offsets(int64_t base, int64_t n_tiles, int64_t ne, int64_t nbf, const SCounts& c) {
    SOffsets o;
    size_t p = (size_t)base;
    auto take = [&](size_t bytes) { p = align256(p); int64_t r = (int64_t)p; p += bytes; return r; };
    o.tiles = take(sizeof(STile) * n_tiles);
    o.conn = take(sizeof(ElemConn) * ne);
    o.tedge = take(sizeof(ElemEdges) * ne);
    o.halo = take(4 * c.n_halo);
    o.hedge = take(4 * c.n_hedge);
    o.hbo = take(4 * c.n_hbo);
    o.sbf = take(sizeof(SFace) * nbf);
    o.me_id = take(4 * c.n_me);
    o.me_ptr = take(4 * (c.n_me + 1));
    o.me_rec = take(4 * c.n_hedge);
    o.mn_id = take(4 * c.n_mn);
    o.mn_ptr = take(4 * (c.n_mn + 1));
    o.mn_rec = take(4 * c.n_halo);
    o.mb_id = take(4 * c.n_mb);
    o.mb_ptr = take(4 * (c.n_mb + 1));
    o.mb_rec = take(4 * c.n_hbo);
    o.total = (int64_t)align256(p);
    return o;
}

// dedicated scratch of the scatter-tile build (candidate lists are bounded by
// D halo nodes and 3 halo edges per element, D halo boundary nodes per face)
struct SScratch {
    uint64_t* pk; uint32_t* pv;          // element pairs [ne]
    int32_t *hn, *he;                    // candidate counts [ne]
    int64_t *hoff, *heoff;               // [ne + 1]
    uint64_t* ck; uint32_t* cv;          // candidates / merge pairs [cmax]
    int32_t* head; int64_t* pos;         // [cmax], [cmax + 1]
    int32_t* list;                       // unique list (count mode) [cmax]
    uint64_t* fk; uint32_t* fv;          // face pairs [nbf]
    int32_t* fh; int64_t* fhoff;         // [nbf], [nbf + 1]
    int32_t *ecnt, *hcnt, *hecnt, *hbcnt, *fcnt;   // [n_tiles + 1]
    int64_t *el_off, *halo_off, *hedge_off, *hbo_off, *bf_off;
    int64_t* maxv;                        // [8]
    unsigned long long* status;           // [2]
};

int64_t s_cmax(int dim, int64_t ne, int64_t nbf) {
    return std::max<int64_t>({int64_t(dim) * ne, 3 * ne, int64_t(dim) * nbf, 1});
}

void s_take(WsLayout& L, SScratch& S, int dim, int64_t ne, int64_t nbf, int64_t n_tiles) {
    const int64_t cm = s_cmax(dim, ne, nbf);
    S.pk = L.take<uint64_t>(ne); S.pv = L.take<uint32_t>(ne);
    S.hn = L.take<int32_t>(ne); S.he = L.take<int32_t>(ne);
    S.hoff = L.take<int64_t>(ne + 1); S.heoff = L.take<int64_t>(ne + 1);
    S.ck = L.take<uint64_t>(cm); S.cv = L.take<uint32_t>(cm);
    S.head = L.take<int32_t>(cm); S.pos = L.take<int64_t>(cm + 1);
    S.list = L.take<int32_t>(cm);
    S.fk = L.take<uint64_t>(nbf + 1); S.fv = L.take<uint32_t>(nbf + 1);
    S.fh = L.take<int32_t>(nbf + 1); S.fhoff = L.take<int64_t>(nbf + 1);
    S.ecnt = L.take<int32_t>(n_tiles + 1); S.hcnt = L.take<int32_t>(n_tiles + 1);
    S.hecnt = L.take<int32_t>(n_tiles + 1); S.hbcnt = L.take<int32_t>(n_tiles + 1);
    S.fcnt = L.take<int32_t>(n_tiles + 1);
    S.el_off = L.take<int64_t>(n_tiles + 1); S.halo_off = L.take<int64_t>(n_tiles + 1);
    S.hedge_off = L.take<int64_t>(n_tiles + 1); S.hbo_off = L.take<int64_t>(n_tiles + 1);
    S.bf_off = L.take<int64_t>(n_tiles + 1);
    S.maxv = L.take<int64_t>(8);
    S.status = L.take<unsigned long long>(2);
}

// sorted candidates -> unique list (out) and per-tile counts; returns the
// number of unique entries through *n_out (synchronizes)
int s_unique(uint64_t* k, int64_t n, int bits, SScratch& S, int32_t* out, int32_t* tile_cnt, int64_t n_tiles,
             void* scan_ws, int64_t* n_out, cudaStream_t s) {
    EM_CUDA_TRY(cudaMemsetAsync(tile_cnt, 0, 4 * (n_tiles + 1), s));
    *n_out = 0;
    if (n) {
        k_heads64<<<G(n), NT, 0, s>>>(k, n, S.head);
        EM_TRY(exclusive_scan_i32_to_i64(S.head, S.pos, n, scan_ws, s));
        k_compact_unique<<<G(n), NT, 0, s>>>(k, n, bits, S.head, S.pos, out, tile_cnt);
        EM_CUDA_TRY(cudaMemcpyAsync(n_out, S.pos + n, 8, cudaMemcpyDeviceToHost, s));
    }
    EM_CUDA_TRY(cudaStreamSynchronize(s));
    EM_CUDA_TRY(cudaGetLastError());
    return EM_OK;
}

// merge CSR of one halo list: (target, position) pairs sorted by target;
// count mode (m_id == NULL) only counts the targets
int s_merge(const int32_t* list, int64_t n, int bits, SScratch& S, uint64_t* kt, uint32_t* vt, void* sort_ws,
            void* scan_ws, int32_t* m_id, int32_t* m_ptr, int32_t* m_rec, int64_t* n_targets, cudaStream_t s) {
    *n_targets = 0;
    if (n == 0) {
        if (m_ptr) EM_CUDA_TRY(cudaMemsetAsync(m_ptr, 0, 4, s));
        return EM_OK;
    }
    k_s_merge_pairs<<<G(n), NT, 0, s>>>(list, n, S.ck, S.cv);
    EM_TRY(radix_sort_pairs(S.ck, S.cv, kt, vt, n, bits, sort_ws, s));
    k_heads64<<<G(n), NT, 0, s>>>(S.ck, n, S.head);
    EM_TRY(exclusive_scan_i32_to_i64(S.head, S.pos, n, scan_ws, s));
    EM_CUDA_TRY(cudaMemcpyAsync(n_targets, S.pos + n, 8, cudaMemcpyDeviceToHost, s));
    EM_CUDA_TRY(cudaStreamSynchronize(s));
    if (m_id) {
        k_s_merge_csr<<<G(n), NT, 0, s>>>(S.ck, S.cv, n, S.head, S.pos, m_id, m_ptr, m_rec);
        const int32_t tail = (int32_t)n;
        EM_CUDA_TRY(cudaMemcpyAsync(m_ptr + *n_targets, &tail, 4, cudaMemcpyHostToDevice, s));
        EM_CUDA_TRY(cudaStreamSynchronize(s));
    }
    EM_CUDA_TRY(cudaGetLastError());
    return EM_OK;
}

struct SInput {
    int dim, T;
    int64_t nv, ne, n_edges, nbf, nbn, n_tiles;
    const int32_t *elems, *e2e, *edges, *bface, *bowner, *bnode;
};

// Scatter tiles.  plan == NULL: counts only (*c written).  Otherwise builds
// every scatter section at the offsets *o (from the counts of a first call,
// which this call reproduces) and fills the scatter fields of *h.
int s_build(const SInput& in, SScratch& S, uint64_t* kt, uint32_t* vt, void* sort_ws, void* scan_ws, char* plan,
            const SOffsets* o, SCounts* c, PlanHeader* h, cudaStream_t s) {
    const int dim = in.dim, T = in.T;
    const int64_t ne = in.ne, nbf = in.nbf, n_tiles = in.n_tiles;
    const int bt = bits_for(std::max<int64_t>(n_tiles - 1, 1));
    const int bn = bits_for(in.nv - 1), be = bits_for(in.n_edges - 1), bb = bits_for(std::max<int64_t>(in.nbn - 1, 1));
    if (bt + 5 > 63 || bt + bn > 63 || bt + be > 63 || bt + bb > 63)
        return fail(EM_ERR_ARG, "grid too large for the tile keys");
    const bool build = plan != nullptr;
    auto at = [&](int64_t off) { return reinterpret_cast<int32_t*>(plan + off); };
    SCounts cc;

    // elements: pairs sorted by (tile, residue) and halo candidate counts
    EM_CUDA_TRY(cudaMemsetAsync(S.ecnt, 0, 4 * (n_tiles + 1), s));
    k_s_pairs<<<G(ne), NT, 0, s>>>(dim, ne, in.elems, in.e2e, in.edges, T, S.pk, S.pv, S.ecnt, S.hn, S.he);
    EM_TRY(radix_sort_pairs(S.pk, S.pv, kt, vt, ne, bt + 5, sort_ws, s));
    EM_TRY(exclusive_scan_i32_to_i64(S.ecnt, S.el_off, n_tiles, scan_ws, s));
    EM_TRY(exclusive_scan_i32_to_i64(S.hn, S.hoff, ne, scan_ws, s));
    EM_TRY(exclusive_scan_i32_to_i64(S.he, S.heoff, ne, scan_ws, s));
    int64_t HC = 0, HEC = 0;
    EM_CUDA_TRY(cudaMemcpyAsync(&HC, S.hoff + ne, 8, cudaMemcpyDeviceToHost, s));
    EM_CUDA_TRY(cudaMemcpyAsync(&HEC, S.heoff + ne, 8, cudaMemcpyDeviceToHost, s));
    EM_CUDA_TRY(cudaStreamSynchronize(s));

    // halo nodes: candidates (tile, node) -> sorted unique list per tile, then
    // their merge lists; the same for halo edges and halo boundary nodes (one
    // candidate buffer, used in turn)
    int32_t* halo = build ? at(o->halo) : S.list;
    if (HC) {
        k_s_halo<<<G(ne), NT, 0, s>>>(dim, ne, in.elems, in.e2e, in.edges, T, bn, be, S.hoff, S.heoff, S.ck, S.cv,
                                       nullptr, nullptr);
        EM_TRY(radix_sort_pairs(S.ck, S.cv, kt, vt, HC, bt + bn, sort_ws, s));
    }
    EM_TRY(s_unique(S.ck, HC, bn, S, halo, S.hcnt, n_tiles, scan_ws, &cc.n_halo, s));
    EM_TRY(exclusive_scan_i32_to_i64(S.hcnt, S.halo_off, n_tiles, scan_ws, s));
    EM_TRY(s_merge(halo, cc.n_halo, bn, S, kt, vt, sort_ws, scan_ws, build ? at(o->mn_id) : nullptr,
                   build ? at(o->mn_ptr) : nullptr, build ? at(o->mn_rec) : nullptr, &cc.n_mn, s));

    int32_t* hedge = build ? at(o->hedge) : S.list;
    if (HEC) {
        k_s_halo<<<G(ne), NT, 0, s>>>(dim, ne, in.elems, in.e2e, in.edges, T, bn, be, S.hoff, S.heoff, nullptr, nullptr,
                                       S.ck, S.cv);
        EM_TRY(radix_sort_pairs(S.ck, S.cv, kt, vt, HEC, bt + be, sort_ws, s));
    }
    EM_TRY(s_unique(S.ck, HEC, be, S, hedge, S.hecnt, n_tiles, scan_ws, &cc.n_hedge, s));
    EM_TRY(exclusive_scan_i32_to_i64(S.hecnt, S.hedge_off, n_tiles, scan_ws, s));
    EM_TRY(s_merge(hedge, cc.n_hedge, be, S, kt, vt, sort_ws, scan_ws, build ? at(o->me_id) : nullptr,
                   build ? at(o->me_ptr) : nullptr, build ? at(o->me_rec) : nullptr, &cc.n_me, s));

    // boundary faces: tile of the owner element, stable by face id
    EM_CUDA_TRY(cudaMemsetAsync(S.fcnt, 0, 4 * (n_tiles + 1), s));
    int64_t HBC = 0;
    if (nbf) {
        k_s_faces<<<G(nbf), NT, 0, s>>>(dim, nbf, in.elems, in.bface, in.bowner, T, S.fk, S.fv, S.fcnt, S.fh);
        EM_TRY(radix_sort_pairs(S.fk, S.fv, kt, vt, nbf, bt, sort_ws, s));
        EM_TRY(exclusive_scan_i32_to_i64(S.fh, S.fhoff, nbf, scan_ws, s));
        EM_CUDA_TRY(cudaMemcpyAsync(&HBC, S.fhoff + nbf, 8, cudaMemcpyDeviceToHost, s));
        EM_CUDA_TRY(cudaStreamSynchronize(s));
    }
    EM_TRY(exclusive_scan_i32_to_i64(S.fcnt, S.bf_off, n_tiles, scan_ws, s));
    int32_t* hbo = build ? at(o->hbo) : S.list;
    if (HBC) {
        k_s_face_halo<<<G(nbf), NT, 0, s>>>(dim, nbf, in.elems, in.bface, in.bowner, in.bnode, in.nbn, T, bb, S.fhoff,
                                             S.ck, S.cv);
        EM_TRY(radix_sort_pairs(S.ck, S.cv, kt, vt, HBC, bt + bb, sort_ws, s));
    }
    EM_TRY(s_unique(S.ck, HBC, bb, S, hbo, S.hbcnt, n_tiles, scan_ws, &cc.n_hbo, s));
    EM_TRY(exclusive_scan_i32_to_i64(S.hbcnt, S.hbo_off, n_tiles, scan_ws, s));
    EM_TRY(s_merge(hbo, cc.n_hbo, bb, S, kt, vt, sort_ws, scan_ws, build ? at(o->mb_id) : nullptr,
                   build ? at(o->mb_ptr) : nullptr, build ? at(o->mb_rec) : nullptr, &cc.n_mb, s));
    if (!build) {
        *c = cc;
        return EM_OK;
    }
    if (cc.n_halo != c->n_halo || cc.n_hedge != c->n_hedge || cc.n_hbo != c->n_hbo || cc.n_me != c->n_me ||
        cc.n_mn != c->n_mn || cc.n_mb != c->n_mb)
        return fail(EM_ERR_CUDA, "scatter plan: counts differ between the sizing and the build pass");

    // tile table, element records, face records
    STile* tiles = reinterpret_cast<STile*>(plan + o->tiles);
    EM_CUDA_TRY(cudaMemsetAsync(S.maxv, 0, 64, s));
    EM_CUDA_TRY(cudaMemsetAsync(S.status, 0, 16, s));
    k_s_tile_info<<<G(n_tiles), NT, 0, s>>>(n_tiles, T, in.nv, in.edges, in.n_edges, in.bnode, in.nbn, S.el_off,
                                             S.halo_off, S.hedge_off, S.hbo_off, S.bf_off, tiles, S.maxv, S.status);
    k_s_elem_records<<<G(ne), NT, 0, s>>>(dim, ne, S.pk, S.pv, in.elems, in.e2e, tiles, halo, hedge,
                                           reinterpret_cast<ElemConn*>(plan + o->conn),
                                           reinterpret_cast<ElemEdges*>(plan + o->tedge));
    if (nbf)
        k_s_face_records<<<G(nbf), NT, 0, s>>>(dim, nbf, S.fk, S.fv, in.bface, in.edges, in.n_edges, in.bnode, in.nbn,
                                                tiles, halo, hedge, hbo, reinterpret_cast<SFace*>(plan + o->sbf));
    EM_CUDA_TRY(cudaGetLastError());
    int64_t mx[8];
    unsigned long long st[2];
    EM_CUDA_TRY(cudaMemcpyAsync(mx, S.maxv, sizeof(mx), cudaMemcpyDeviceToHost, s));
    EM_CUDA_TRY(cudaMemcpyAsync(st, S.status, sizeof(st), cudaMemcpyDeviceToHost, s));
    EM_CUDA_TRY(cudaStreamSynchronize(s));
    if (st[0])
        return fail(EM_ERR_ARG, std::to_string(st[0]) + " scatter tile(s) exceed the 16-bit local index limits: use a "
                                                         "smaller tile_nodes");
    h->s_max_el = mx[0]; h->s_max_nodes = mx[1]; h->s_max_edges = mx[2]; h->s_max_bnodes = mx[3]; h->s_max_bf = mx[4];
    h->n_shalo = cc.n_halo; h->n_shedge = cc.n_hedge; h->n_shbo = cc.n_hbo;
    h->n_me = cc.n_me; h->n_mn = cc.n_mn; h->n_mb = cc.n_mb;
    h->off_stiles = o->tiles; h->off_sconn = o->conn; h->off_stedge = o->tedge; h->off_shalo = o->halo;
    h->off_shedge = o->hedge; h->off_shbo = o->hbo; h->off_sbf = o->sbf;
    h->off_me_id = o->me_id; h->off_me_ptr = o->me_ptr; h->off_me_rec = o->me_rec;
    h->off_mn_id = o->mn_id; h->off_mn_ptr = o->mn_ptr; h->off_mn_rec = o->mn_rec;
    h->off_mb_id = o->mb_id; h->off_mb_ptr = o->mb_ptr; h->off_mb_rec = o->mb_rec;
    return EM_OK;
}

}  // namespace

int plan_build_impl(int dim, int64_t nv, int64_t ne, const int32_t* elems, const int32_t* e2e, int64_t n_edges,
                    const int32_t* edges, int64_t nbf, const int32_t* bface, const int32_t* bowner, int64_t nbn,
                    const int32_t* bnode, int tile_nodes, void* ws, size_t* ws_bytes, void* plan, size_t* plan_bytes,
                    int64_t* plan_info, cudaStream_t s) {
    if (dim != 2 && dim != 3) return fail(EM_ERR_ARG, "dim must be 2 or 3");
    if (nv <= 0 || ne <= 0 || n_edges <= 0 || nbf < 0 || nbn < 0) return fail(EM_ERR_ARG, "bad sizes");
    if (!ws_bytes || !plan_bytes) return fail(EM_ERR_ARG, "ws_bytes and plan_bytes must not be NULL");
    const int T = tile_nodes ? tile_nodes : 256;
    if (T < 32 || T > 2048 || (T % 32)) return fail(EM_ERR_ARG, "tile_nodes must be a multiple of 32 in [32, 2048]");
    const int64_t n_tiles = (nv + T - 1) / T;
    const int nle = dim == 3 ? 6 : 3;
    const int nfe = dim == 3 ? 3 : 1;

    // ---- count pass scratch ----------------------------------------------
    WsLayout A(ws);
    int32_t* npair = A.take<int32_t>(ne);
    int32_t* nhalo = A.take<int32_t>(ne);
    int32_t* nhedge = A.take<int32_t>(ne);
    int32_t* tile_cnt = A.take<int32_t>(n_tiles + 1);
    int64_t* poff = A.take<int64_t>(ne + 1);
    int32_t* nbp = A.take<int32_t>(nbf + 1);
    int64_t* bpoff = A.take<int64_t>(nbf + 1);
    int64_t* tmp = A.take<int64_t>(ne + 1);
    void* scan_a = A.take<char>(scan_ws_bytes(std::max<int64_t>({ne, nbf, n_tiles + 1, 1})));
    const size_t count_bytes = A.bytes();
    if (!ws) {
        *ws_bytes = count_bytes;
        *plan_bytes = 0;
        return EM_OK;
    }
    if (*ws_bytes < count_bytes) return fail(EM_ERR_WORKSPACE, "plan workspace too small for the count pass");
    if (!elems || !e2e || !edges || (nbf && (!bface || !bowner)) || (nbn && !bnode))
        return fail(EM_ERR_ARG, "null topology array");

    int64_t P = 0, HC = 0, HEC = 0, BP = 0;
    EM_CUDA_TRY(cudaMemsetAsync(tile_cnt, 0, 4 * (n_tiles + 1), s));
    k_count_elem<<<G(ne), NT, 0, s>>>(dim, ne, elems, e2e, edges, T, npair, nhalo, nhedge, tile_cnt);
    EM_TRY(exclusive_scan_i32_to_i64(nhalo, tmp, ne, scan_a, s));
    EM_CUDA_TRY(cudaMemcpyAsync(&HC, tmp + ne, 8, cudaMemcpyDeviceToHost, s));
    EM_CUDA_TRY(cudaStreamSynchronize(s));
    EM_TRY(exclusive_scan_i32_to_i64(nhedge, tmp, ne, scan_a, s));
    EM_CUDA_TRY(cudaMemcpyAsync(&HEC, tmp + ne, 8, cudaMemcpyDeviceToHost, s));
    EM_CUDA_TRY(cudaStreamSynchronize(s));
    EM_TRY(exclusive_scan_i32_to_i64(npair, poff, ne, scan_a, s));
    EM_CUDA_TRY(cudaMemcpyAsync(&P, poff + ne, 8, cudaMemcpyDeviceToHost, s));
    if (nbf) {
        k_count_bface<<<G(nbf), NT, 0, s>>>(dim, nbf, bface, T, nbp);
        EM_TRY(exclusive_scan_i32_to_i64(nbp, bpoff, nbf, scan_a, s));
        EM_CUDA_TRY(cudaMemcpyAsync(&BP, bpoff + nbf, 8, cudaMemcpyDeviceToHost, s));
    }
    EM_CUDA_TRY(cudaStreamSynchronize(s));
    EM_CUDA_TRY(cudaGetLastError());

    // ---- build scratch (exact) ------------------------------------------
    const int64_t ES = nle * ne + nfe * nbf;
    const int64_t NS = (dim + 1) * ne;
    const int64_t BS = dim * nbf;
    const int64_t SMAX = std::max<int64_t>({P, HC, HEC, ES, NS, BP, BS, 1});
    const int64_t CMAX = std::max<int64_t>({P, BP, HC, HEC, 1});
    WsLayout L(ws);
    L.take<char>(count_bytes);
    uint64_t* kt = L.take<uint64_t>(SMAX);
    uint32_t* vt = L.take<uint32_t>(SMAX);
    void* sort_ws = L.take<char>(radix_sort_ws_bytes(SMAX));
    void* scan_b = L.take<char>(scan_ws_bytes(std::max<int64_t>({SMAX, n_edges + 1, nv + 1, nbn + 1})));
    uint64_t* pk = L.take<uint64_t>(P);
    uint32_t* pv = L.take<uint32_t>(P);
    uint64_t* hk = L.take<uint64_t>(HC);
    uint32_t* hv = L.take<uint32_t>(HC);
    uint64_t* hek = L.take<uint64_t>(HEC);
    uint32_t* hev = L.take<uint32_t>(HEC);
    uint64_t* bk = L.take<uint64_t>(BP);
    uint32_t* bv = L.take<uint32_t>(BP);
    uint64_t* esk = L.take<uint64_t>(ES);
    uint32_t* esv = L.take<uint32_t>(ES);
    uint64_t* nsk = L.take<uint64_t>(NS);
    uint32_t* nsv = L.take<uint32_t>(NS);
    uint64_t* bsk = L.take<uint64_t>(BS);
    uint32_t* bsv = L.take<uint32_t>(BS);
    int32_t* c32a = L.take<int32_t>(CMAX);
    int32_t* c32b = L.take<int32_t>(CMAX);
    int64_t* o64a = L.take<int64_t>(CMAX + 1);
    int64_t* o64b = L.take<int64_t>(CMAX + 1);
    int32_t* halo_l = L.take<int32_t>(HC + 1);
    int32_t* hedge_l = L.take<int32_t>(HEC + 1);
    int32_t* hcnt = L.take<int32_t>(n_tiles + 1);
    int32_t* hecnt = L.take<int32_t>(n_tiles + 1);
    int32_t* tbfcnt = L.take<int32_t>(n_tiles + 1);
    int64_t* el_off = L.take<int64_t>(n_tiles + 1);
    int64_t* halo_off = L.take<int64_t>(n_tiles + 1);
    int64_t* hedge_off = L.take<int64_t>(n_tiles + 1);
    int64_t* tbf_off = L.take<int64_t>(n_tiles + 1);
    int32_t* kcnt = L.take<int32_t>(std::max<int64_t>({n_edges, nv, nbn}) + 1);
    int64_t* koff = L.take<int64_t>(std::max<int64_t>({n_edges, nv, nbn}) + 1);
    int64_t* maxv = L.take<int64_t>(8);
    int64_t* smax = L.take<int64_t>(4);
    unsigned long long* status = L.take<unsigned long long>(2);
    SScratch S;
    s_take(L, S, dim, ne, nbf, n_tiles);
    const size_t full_bytes = L.bytes();
    const SInput sin{dim, T, nv, ne, n_edges, nbf, nbn, n_tiles, elems, e2e, edges, bface, bowner, bnode};

    const int bt = bits_for(std::max<int64_t>(n_tiles - 1, 1));
    const int bn = bits_for(nv - 1);
    const int be = bits_for(n_edges - 1);
    if (bt + bn > 63 || bt + be > 63 || bt + 9 > 63) return fail(EM_ERR_ARG, "grid too large for the tile keys");

    if (*ws_bytes < full_bytes) {
        if (plan) return fail(EM_ERR_WORKSPACE, "plan workspace too small: need " + std::to_string(full_bytes));
        // size report with halo counts bounded by their candidates
        PlanOffsets po = plan_offsets(n_tiles, nv, n_edges, nbn, P, HC, HEC, ES, NS, BP, BS);
        SCounts sb;
        sb.n_halo = dim * ne; sb.n_hedge = 3 * ne; sb.n_hbo = dim * nbf;
        sb.n_me = n_edges; sb.n_mn = nv; sb.n_mb = nbn;
        *plan_bytes = (size_t)s_offsets(po.total, n_tiles, ne, nbf, sb).total;
        *ws_bytes = full_bytes;
        return EM_OK;
    }

    // 1. pairs (tile, element), elements ascending inside a tile (stable sort)
    k_fill_pairs<<<G(ne), NT, 0, s>>>(dim, ne, elems, T, poff, pk, pv);
    EM_TRY(radix_sort_pairs(pk, pv, kt, vt, P, bt + 9, sort_ws, s));
    k_key_drop_mask<<<G(P), NT, 0, s>>>(P, pk);
    EM_TRY(exclusive_scan_i32_to_i64(tile_cnt, el_off, n_tiles, scan_b, s));

    // 2. halo nodes and halo edges of every tile (sorted, unique)
    k_pair_counts<<<G(P), NT, 0, s>>>(dim, P, pk, pv, elems, e2e, edges, T, c32a, c32b);
    EM_TRY(exclusive_scan_i32_to_i64(c32a, o64a, P, scan_b, s));
    EM_TRY(exclusive_scan_i32_to_i64(c32b, o64b, P, scan_b, s));
    k_fill_halo<<<G(P), NT, 0, s>>>(dim, P, pk, pv, elems, e2e, edges, T, bn, be, o64a, o64b, hk, hv, hek, hev);
    EM_TRY(radix_sort_pairs(hk, hv, kt, vt, HC, bt + bn, sort_ws, s));
    EM_TRY(radix_sort_pairs(hek, hev, kt, vt, HEC, bt + be, sort_ws, s));
    int64_t n_halo = 0, n_hedge = 0;
    EM_CUDA_TRY(cudaMemsetAsync(hcnt, 0, 4 * (n_tiles + 1), s));
    EM_CUDA_TRY(cudaMemsetAsync(hecnt, 0, 4 * (n_tiles + 1), s));
    if (HC) {
        k_heads64<<<G(HC), NT, 0, s>>>(hk, HC, c32a);
        EM_TRY(exclusive_scan_i32_to_i64(c32a, o64a, HC, scan_b, s));
        k_compact_unique<<<G(HC), NT, 0, s>>>(hk, HC, bn, c32a, o64a, halo_l, hcnt);
        EM_CUDA_TRY(cudaMemcpyAsync(&n_halo, o64a + HC, 8, cudaMemcpyDeviceToHost, s));
    }
    if (HEC) {
        k_heads64<<<G(HEC), NT, 0, s>>>(hek, HEC, c32b);
        EM_TRY(exclusive_scan_i32_to_i64(c32b, o64b, HEC, scan_b, s));
        k_compact_unique<<<G(HEC), NT, 0, s>>>(hek, HEC, be, c32b, o64b, hedge_l, hecnt);
        EM_CUDA_TRY(cudaMemcpyAsync(&n_hedge, o64b + HEC, 8, cudaMemcpyDeviceToHost, s));
    }
    EM_TRY(exclusive_scan_i32_to_i64(hcnt, halo_off, n_tiles, scan_b, s));
    EM_TRY(exclusive_scan_i32_to_i64(hecnt, hedge_off, n_tiles, scan_b, s));
    EM_CUDA_TRY(cudaStreamSynchronize(s));
    EM_CUDA_TRY(cudaGetLastError());

    PlanOffsets po = plan_offsets(n_tiles, nv, n_edges, nbn, P, n_halo, n_hedge, ES, NS, BP, BS);
    // scatter tiles: exact counts, then the sections behind the gather plan
    SCounts sc;
    EM_TRY(s_build(sin, S, kt, vt, sort_ws, scan_b, nullptr, nullptr, &sc, nullptr, s));
    const SOffsets so = s_offsets(po.total, n_tiles, ne, nbf, sc);
    if (!plan) {
        *plan_bytes = (size_t)so.total;
        *ws_bytes = full_bytes;
        return EM_OK;
    }
    if (*plan_bytes < (size_t)so.total)
        return fail(EM_ERR_WORKSPACE, "plan buffer too small: need " + std::to_string(so.total));
    char* pb = static_cast<char*>(plan);
    TileInfo* tiles = reinterpret_cast<TileInfo*>(pb + po.tiles);
    ElemConn* conn = reinterpret_cast<ElemConn*>(pb + po.conn);
    ElemEdges* tedge = reinterpret_cast<ElemEdges*>(pb + po.tedge);
    int32_t* halo = reinterpret_cast<int32_t*>(pb + po.halo);
    int32_t* hedge = reinterpret_cast<int32_t*>(pb + po.hedge);
    int32_t* eslot_ptr = reinterpret_cast<int32_t*>(pb + po.eslot_ptr);
    uint16_t* eslot = reinterpret_cast<uint16_t*>(pb + po.eslot);
    int32_t* nslot_ptr = reinterpret_cast<int32_t*>(pb + po.nslot_ptr);
    uint16_t* nslot = reinterpret_cast<uint16_t*>(pb + po.nslot);
    TileBFace* tbf = reinterpret_cast<TileBFace*>(pb + po.tbf);
    int32_t* bslot_ptr = reinterpret_cast<int32_t*>(pb + po.bslot_ptr);
    uint16_t* bslot = reinterpret_cast<uint16_t*>(pb + po.bslot);
    if (n_halo) EM_CUDA_TRY(cudaMemcpyAsync(halo, halo_l, 4 * n_halo, cudaMemcpyDeviceToDevice, s));
    if (n_hedge) EM_CUDA_TRY(cudaMemcpyAsync(hedge, hedge_l, 4 * n_hedge, cudaMemcpyDeviceToDevice, s));

    // 3. boundary pairs (tile, face)
    EM_CUDA_TRY(cudaMemsetAsync(tbfcnt, 0, 4 * (n_tiles + 1), s));
    if (BP) {
        k_fill_bpairs<<<G(nbf), NT, 0, s>>>(dim, nbf, bface, T, bpoff, bk, bv, tbfcnt);
        EM_TRY(radix_sort_pairs(bk, bv, kt, vt, BP, bt, sort_ws, s));
    }
    EM_TRY(exclusive_scan_i32_to_i64(tbfcnt, tbf_off, n_tiles, scan_b, s));

    // 4. tile table
    EM_CUDA_TRY(cudaMemsetAsync(maxv, 0, 64, s));
    EM_CUDA_TRY(cudaMemsetAsync(status, 0, 16, s));
    k_tile_info<<<G(n_tiles), NT, 0, s>>>(n_tiles, T, nv, edges, n_edges, bnode, nbn, el_off, halo_off, hedge_off,
                                          tbf_off, tiles, maxv, status);

    // 5. element records, element edge slots and node slots
    k_pair_slot_counts<<<G(P), NT, 0, s>>>(dim, P, pk, pv, elems, T, c32a, c32b);
    EM_TRY(exclusive_scan_i32_to_i64(c32a, o64a, P, scan_b, s));
    EM_TRY(exclusive_scan_i32_to_i64(c32b, o64b, P, scan_b, s));
    k_elem_records<<<G(P), NT, 0, s>>>(dim, P, pk, pv, elems, e2e, tiles, halo, hedge, T, o64a, o64b, conn, tedge,
                                       esk, esv, nsk, nsv);
    EM_CUDA_TRY(cudaGetLastError());

    // 6. boundary face records, boundary edge slots (after all element slots) and boundary node slots
    if (BP) {
        k_bface_counts<<<G(BP), NT, 0, s>>>(dim, BP, bk, bv, bface, edges, T, c32a, c32b);
        EM_TRY(exclusive_scan_i32_to_i64(c32a, o64a, BP, scan_b, s));
        EM_TRY(exclusive_scan_i32_to_i64(c32b, o64b, BP, scan_b, s));
        k_bface_records<<<G(BP), NT, 0, s>>>(dim, BP, bk, bv, bface, edges, n_edges, bnode, nbn, tiles, halo, hedge,
                                             T, o64a, o64b, nle * ne, tbf, esk, esv, bsk, bsv);
        EM_CUDA_TRY(cudaGetLastError());
    }

    // 7. gather lists: stable sorts by target, CSR offsets, 16-bit slots
    EM_TRY(radix_sort_pairs(esk, esv, kt, vt, ES, be, sort_ws, s));
    EM_TRY(csr_from_keys(esk, ES, n_edges, kcnt, koff, eslot_ptr, scan_b, s));
    k_u32_to_u16<<<G(ES), NT, 0, s>>>(esv, ES, eslot);
    EM_TRY(radix_sort_pairs(nsk, nsv, kt, vt, NS, bn, sort_ws, s));
    EM_TRY(csr_from_keys(nsk, NS, nv, kcnt, koff, nslot_ptr, scan_b, s));
    k_u32_to_u16<<<G(NS), NT, 0, s>>>(nsv, NS, nslot);
    if (nbn) {
        EM_TRY(radix_sort_pairs(bsk, bsv, kt, vt, BS, bits_for(std::max<int64_t>(nbn - 1, 1)), sort_ws, s));
        EM_TRY(csr_from_keys(bsk, BS, nbn, kcnt, koff, bslot_ptr, scan_b, s));
        if (BS) k_u32_to_u16<<<G(BS), NT, 0, s>>>(bsv, BS, bslot);
    }
    EM_CUDA_TRY(cudaGetLastError());

    EM_CUDA_TRY(cudaMemsetAsync(smax, 0, 32, s));
    k_tile_slot_max<<<G(n_tiles), NT, 0, s>>>(n_tiles, tiles, eslot_ptr, nslot_ptr, nbn ? bslot_ptr : nullptr, smax);
    k_max_run<<<G(n_edges), NT, 0, s>>>(eslot_ptr, n_edges, smax + 3);
    int64_t* vmax = maxv + 7;
    EM_CUDA_TRY(cudaMemsetAsync(vmax, 0, 8, s));
    k_max_run<<<G(nv), NT, 0, s>>>(nslot_ptr, nv, vmax);
    // 8. header
    int64_t mx[8], sm[4];
    int64_t node_val = 0;
    EM_CUDA_TRY(cudaMemcpyAsync(sm, smax, sizeof(sm), cudaMemcpyDeviceToHost, s));
    EM_CUDA_TRY(cudaMemcpyAsync(&node_val, vmax, 8, cudaMemcpyDeviceToHost, s));
    unsigned long long st[2];
    EM_CUDA_TRY(cudaMemcpyAsync(mx, maxv, sizeof(mx), cudaMemcpyDeviceToHost, s));
    EM_CUDA_TRY(cudaMemcpyAsync(st, status, sizeof(st), cudaMemcpyDeviceToHost, s));
    EM_CUDA_TRY(cudaStreamSynchronize(s));
    if (st[0]) return fail(EM_ERR_ARG, std::to_string(st[0]) + " tile(s) exceed the 16-bit local index limits: use a "
                                                             "smaller tile_nodes");
    PlanHeader h;
    memset(&h, 0, sizeof(h));
    h.magic = PLAN_MAGIC; h.version = PLAN_VERSION; h.dim = dim; h.tile_nodes = T; h.n_tiles = n_tiles;
    h.n_nodes = nv; h.n_elems = ne; h.n_edges = n_edges; h.n_bfaces = nbf; h.n_bnodes = nbn;
    h.n_pairs = P; h.n_halo = n_halo; h.n_hedge = n_hedge; h.n_tbf = BP; h.n_eslot = ES; h.n_nslot = NS;
    h.n_bslot = BS;
    h.max_el = mx[0]; h.max_nodes = mx[1]; h.max_edges = mx[2]; h.max_eo = mx[3]; h.max_bf = mx[4];
    h.max_bo = mx[5]; h.max_own = mx[6];
    h.off_tiles = po.tiles; h.off_conn = po.conn; h.off_tedge = po.tedge; h.off_halo = po.halo; h.off_hedge = po.hedge;
    h.off_eslot_ptr = po.eslot_ptr; h.off_eslot = po.eslot; h.off_nslot_ptr = po.nslot_ptr; h.off_nslot = po.nslot;
    h.off_tbf = po.tbf; h.off_bslot_ptr = po.bslot_ptr; h.off_bslot = po.bslot;
    EM_TRY(s_build(sin, S, kt, vt, sort_ws, scan_b, pb, &so, &sc, &h, s));
    EM_CUDA_TRY(cudaMemcpyAsync(plan, &h, sizeof(h), cudaMemcpyHostToDevice, s));
    EM_CUDA_TRY(cudaStreamSynchronize(s));
    *plan_bytes = (size_t)so.total;
    if (plan_info) {
        for (int i = 0; i < EM_PLAN_INFO_LEN; i++) plan_info[i] = 0;
        plan_info[EM_PLAN_INFO_TILE_NODES] = T;
        plan_info[EM_PLAN_INFO_TILES] = n_tiles;
        plan_info[EM_PLAN_INFO_MAX_ELEMS] = h.max_el;
        plan_info[EM_PLAN_INFO_MAX_NODES] = h.max_nodes;
        plan_info[EM_PLAN_INFO_MAX_EDGES] = h.max_edges;
        plan_info[EM_PLAN_INFO_MAX_OWNED_EDGES] = h.max_eo;
        plan_info[EM_PLAN_INFO_MAX_BFACES] = h.max_bf;
        plan_info[EM_PLAN_INFO_MAX_OWNED_BNODES] = h.max_bo;
        plan_info[EM_PLAN_INFO_MAX_OWNED_NODES] = h.max_own;
        plan_info[EM_PLAN_INFO_CHECK] = so.total;
        plan_info[EM_PLAN_INFO_S_MAX_ELEMS] = h.s_max_el;
        plan_info[EM_PLAN_INFO_S_MAX_NODES] = h.s_max_nodes;
        plan_info[EM_PLAN_INFO_S_MAX_EDGES] = h.s_max_edges;
        plan_info[EM_PLAN_INFO_S_MAX_BNODES] = h.s_max_bnodes;
        plan_info[EM_PLAN_INFO_S_MAX_BFACES] = h.s_max_bf;
        plan_info[EM_PLAN_INFO_REC_NODES] = h.n_shalo;
        plan_info[EM_PLAN_INFO_REC_EDGES] = h.n_shedge;
        plan_info[EM_PLAN_INFO_REC_BNODES] = h.n_shbo;
        plan_info[EM_PLAN_INFO_MAX_ESLOTS] = sm[0];
        plan_info[EM_PLAN_INFO_MAX_NSLOTS] = sm[1];
        plan_info[EM_PLAN_INFO_MAX_BSLOTS] = sm[2];
        plan_info[EM_PLAN_INFO_MAX_EDGE_VALENCE] = sm[3];
        plan_info[EM_PLAN_INFO_MAX_NODE_VALENCE] = node_val;
    }
    return EM_OK;
}

int plan_tiles_impl(const void* plan, int64_t* n_tiles, cudaStream_t s) {
    if (!plan || !n_tiles) return fail(EM_ERR_ARG, "null argument");
    PlanHeader h;
    EM_CUDA_TRY(cudaMemcpyAsync(&h, plan, sizeof(h), cudaMemcpyDeviceToHost, s));
    EM_CUDA_TRY(cudaStreamSynchronize(s));
    if (h.magic != PLAN_MAGIC) return fail(EM_ERR_ARG, "not a plan");
    *n_tiles = h.n_tiles;
    return EM_OK;
}

}  // namespace em

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
    const size_t full_bytes = L.bytes();

    const int bt = bits_for(std::max<int64_t>(n_tiles - 1, 1));
    const int bn = bits_for(nv - 1);
    const int be = bits_for(n_edges - 1);
    if (bt + bn > 63 || bt + be > 63 || bt + 9 > 63) return fail(EM_ERR_ARG, "grid too large for the tile keys");

    if (*ws_bytes < full_bytes) {
        if (plan) return fail(EM_ERR_WORKSPACE, "plan workspace too small: need " + std::to_string(full_bytes));
        // size report with halo counts bounded by their candidates
        PlanOffsets po = plan_offsets(n_tiles, nv, n_edges, nbn, P, HC, HEC, ES, NS, BP, BS);
        *plan_bytes = (size_t)po.total;
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
    if (!plan) {
        *plan_bytes = (size_t)po.total;
        *ws_bytes = full_bytes;
        return EM_OK;
    }
    if (*plan_bytes < (size_t)po.total)
        return fail(EM_ERR_WORKSPACE, "plan buffer too small: need " + std::to_string(po.total));
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
    EM_CUDA_TRY(cudaMemcpyAsync(plan, &h, sizeof(h), cudaMemcpyHostToDevice, s));
    EM_CUDA_TRY(cudaStreamSynchronize(s));
    *plan_bytes = (size_t)po.total;
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
        plan_info[EM_PLAN_INFO_CHECK] = po.total;
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

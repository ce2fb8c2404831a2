// EM_PATH_CSR: edge-centric CSR gather in FP64 (deterministic reference form).
//
// n_jk: one thread per edge walks the edge's element slots (edge_slot, in
//       ascending slot id = ascending element id) and recomputes for each the
//       area vector of the face opposite the lower end j (one cross product,
//       oriented away from j), then adds n_B for each boundary face of the
//       edge in ascending face id, and scales: 3D accumulates 2 n_j and n_B and
//       applies 1/12 at the end (Eqs. add_contribution_to_njk_tetra,
//       njk_boundary_correction_3d, apply_1over12_at_the_end_njk_tetra);
//       2D adds n_j/3 and n_B/6 (Eqs. njk_eff_algorithm_tria_01,
//       njk_eff_algorithm_tria_02p5_nB).
// V_i:  one thread per node over its elements in ascending id, V_E/(D+1)
//       (Sec. 4.2).
// b_i:  one thread per boundary node over its boundary faces, n_B/D (Sec. 3.2.3).
// Every product and sum is rounded explicitly (no fused multiply-add) in the
// order of the serial element and boundary loops, so each output is the same
// floating-point expression as in a plain serial implementation of those
// loops.  The node and boundary lists are built per call in the workspace
// (counting sort + per-list insertion sort).
#include "em_common.cuh"
#include "em_kernels.cuh"

namespace em {

namespace {

constexpr int NTC = 256;
#define GLOOP(i, n) for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < (n); i += int64_t(gridDim.x) * blockDim.x)

__constant__ int c_le3c[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
__constant__ int c_le2c[3][2] = {{0, 1}, {0, 2}, {1, 2}};

__device__ __forceinline__ double M(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double S(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double P(double a, double b) { return __dadd_rn(a, b); }

__device__ __forceinline__ int comp4(const int4& v, int i) { return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w; }

// outward area vector of the face of the element opposite stored node o
// (3D: 1/2 (x_l - x_k) x (x_r - x_k); 2D: (y_r - y_k, x_k - x_r)), sign chosen
// so that it points away from node o
template <int DIM>
__device__ __forceinline__ void face_opposite(const double* x, const int4& v, int o, double* n) {
    int oth[3], c = 0;
    for (int i = 0; i < DIM + 1; i++)
        if (i != o) oth[c++] = comp4(v, i);
    const int64_t vo = comp4(v, o), k = oth[0];
    double d[3] = {0, 0, 0};
    for (int i = 0; i < DIM; i++) d[i] = S(x[DIM * k + i], x[DIM * vo + i]);
    double dotv;
    if (DIM == 3) {
        const int64_t l = oth[1], r = oth[2];
        double u0 = S(x[3 * l], x[3 * k]), u1 = S(x[3 * l + 1], x[3 * k + 1]), u2 = S(x[3 * l + 2], x[3 * k + 2]);
        double t0 = S(x[3 * r], x[3 * k]), t1 = S(x[3 * r + 1], x[3 * k + 1]), t2 = S(x[3 * r + 2], x[3 * k + 2]);
        n[0] = M(S(M(u1, t2), M(u2, t1)), 0.5);
        n[1] = M(S(M(u2, t0), M(u0, t2)), 0.5);
        n[2] = M(S(M(u0, t1), M(u1, t0)), 0.5);
        dotv = P(P(P(0.0, M(n[0], d[0])), M(n[1], d[1])), M(n[2], d[2]));
    } else {
        const int64_t r = oth[1];
        n[0] = S(x[2 * r + 1], x[2 * k + 1]);
        n[1] = S(x[2 * k], x[2 * r]);
        dotv = P(P(0.0, M(n[0], d[0])), M(n[1], d[1]));
    }
    if (dotv < 0)
        for (int i = 0; i < DIM; i++) n[i] = -n[i];
}

template <int DIM>
__device__ __forceinline__ void bface_vector(const double* x, const int32_t* f, double* nB) {
    if (DIM == 3) {
        const int64_t p = f[0], q = f[1], r = f[2];
        double u0 = S(x[3 * q], x[3 * p]), u1 = S(x[3 * q + 1], x[3 * p + 1]), u2 = S(x[3 * q + 2], x[3 * p + 2]);
        double t0 = S(x[3 * r], x[3 * p]), t1 = S(x[3 * r + 1], x[3 * p + 1]), t2 = S(x[3 * r + 2], x[3 * p + 2]);
        nB[0] = M(S(M(u1, t2), M(u2, t1)), 0.5);
        nB[1] = M(S(M(u2, t0), M(u0, t2)), 0.5);
        nB[2] = M(S(M(u0, t1), M(u1, t0)), 0.5);
    } else {
        const int64_t a = f[0], b = f[1];
        nB[0] = S(x[2 * a + 1], x[2 * b + 1]);
        nB[1] = S(x[2 * b], x[2 * a]);
    }
}

template <int DIM>
__global__ void k_csr_edges(int64_t n_edges, const int32_t* __restrict__ eptr, const int32_t* __restrict__ eslot,
                            const int32_t* __restrict__ elems, const double* __restrict__ x,
                            const int64_t* __restrict__ boff, const int32_t* __restrict__ bent,
                            const int32_t* __restrict__ bface, double* __restrict__ n) {
    constexpr int NLE = DIM == 3 ? 6 : 3;
    GLOOP(e, n_edges) {
        double acc[3] = {0, 0, 0};
        for (int32_t q = eptr[e]; q < eptr[e + 1]; q++) {
            const int32_t sl = eslot[q];
            const int64_t E = sl / NLE;
            const int l = sl % NLE;
            const int4 v = reinterpret_cast<const int4*>(elems)[E];
            const int p0 = DIM == 3 ? c_le3c[l][0] : c_le2c[l][0];
            const int p1 = DIM == 3 ? c_le3c[l][1] : c_le2c[l][1];
            const int low = comp4(v, p0) < comp4(v, p1) ? p0 : p1;
            double nj[3];
            face_opposite<DIM>(x, v, low, nj);
            for (int i = 0; i < DIM; i++) {
                if (DIM == 3) acc[i] = P(acc[i], M(2.0, nj[i]));
                else acc[i] = P(acc[i], __ddiv_rn(nj[i], 3.0));
            }
        }
        for (int64_t q = boff[e]; q < boff[e + 1]; q++) {
            double nB[3];
            bface_vector<DIM>(x, bface + DIM * int64_t(bent[q]), nB);
            for (int i = 0; i < DIM; i++) acc[i] = DIM == 3 ? P(acc[i], nB[i]) : P(acc[i], __ddiv_rn(nB[i], 6.0));
        }
        for (int i = 0; i < DIM; i++) n[DIM * e + i] = DIM == 3 ? M(acc[i], 1.0 / 12.0) : acc[i];
    }
}

template <int DIM>
__global__ void k_csr_vol(int64_t nv, const int64_t* __restrict__ noff, const int32_t* __restrict__ nent,
                          const int32_t* __restrict__ elems, const double* __restrict__ x, double* __restrict__ vol) {
    GLOOP(i, nv) {
        double acc = 0.0;
        for (int64_t q = noff[i]; q < noff[i + 1]; q++) {
            const int64_t E = nent[q];
            const int4 v = reinterpret_cast<const int4*>(elems)[E];
            double vE;
            if (DIM == 3) {
                const int64_t a0 = v.x, a1 = v.y, a2 = v.z, a3 = v.w;
                double a[3], b[3], c[3];
                for (int k = 0; k < 3; k++) {
                    a[k] = S(x[3 * a1 + k], x[3 * a0 + k]);
                    b[k] = S(x[3 * a2 + k], x[3 * a0 + k]);
                    c[k] = S(x[3 * a3 + k], x[3 * a0 + k]);
                }
                double bc0 = S(M(b[1], c[2]), M(b[2], c[1]));
                double bc1 = S(M(b[2], c[0]), M(b[0], c[2]));
                double bc2 = S(M(b[0], c[1]), M(b[1], c[0]));
                double det = P(P(P(0.0, M(a[0], bc0)), M(a[1], bc1)), M(a[2], bc2));
                vE = __ddiv_rn(fabs(det), 6.0);
            } else {
                const int64_t a0 = v.x, a1 = v.y, a2 = v.z;
                double ax = S(x[2 * a1], x[2 * a0]), ay = S(x[2 * a1 + 1], x[2 * a0 + 1]);
                double bx = S(x[2 * a2], x[2 * a0]), by = S(x[2 * a2 + 1], x[2 * a0 + 1]);
                vE = __ddiv_rn(fabs(S(M(ax, by), M(ay, bx))), 2.0);
            }
            acc = P(acc, __ddiv_rn(vE, (double)(DIM + 1)));
        }
        vol[i] = acc;
    }
}

template <int DIM>
__global__ void k_csr_bnormal(int64_t nbn, const int64_t* __restrict__ off, const int32_t* __restrict__ ent,
                              const int32_t* __restrict__ bface, const double* __restrict__ x,
                              double* __restrict__ bnormal) {
    GLOOP(k, nbn) {
        double acc[3] = {0, 0, 0};
        for (int64_t q = off[k]; q < off[k + 1]; q++) {
            double nB[3];
            bface_vector<DIM>(x, bface + DIM * int64_t(ent[q]), nB);
            for (int i = 0; i < DIM; i++) acc[i] = P(acc[i], __ddiv_rn(nB[i], (double)DIM));
        }
        for (int i = 0; i < DIM; i++) bnormal[DIM * k + i] = acc[i];
    }
}

// ---- list building: counting sort by key, then each list sorted ascending --
__global__ void k_node_keys(int dim, int64_t ne, const int32_t* __restrict__ elems, int32_t* __restrict__ cnt) {
    GLOOP(E, ne) {
        const int4 v = reinterpret_cast<const int4*>(elems)[E];
        for (int r = 0; r < dim + 1; r++) atomicAdd(&cnt[comp4(v, r)], 1);
    }
}
__global__ void k_node_fill(int dim, int64_t ne, const int32_t* __restrict__ elems, const int64_t* __restrict__ off,
                            int32_t* __restrict__ fill, int32_t* __restrict__ ent) {
    GLOOP(E, ne) {
        const int4 v = reinterpret_cast<const int4*>(elems)[E];
        for (int r = 0; r < dim + 1; r++) {
            const int key = comp4(v, r);
            ent[off[key] + atomicAdd(&fill[key], 1)] = (int32_t)E;
        }
    }
}

__device__ __forceinline__ int64_t bnode_index(const int32_t* bnode, int64_t nbn, int32_t v) {
    int64_t lo = 0, hi = nbn - 1;
    while (lo <= hi) {
        int64_t mid = (lo + hi) >> 1;
        if (bnode[mid] == v) return mid;
        if (bnode[mid] < v) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

// boundary face -> its edges (from the owner's element-to-edge map) and nodes
template <int DIM>
__global__ void k_bface_keys(int64_t nbf, const int32_t* __restrict__ bowner, const int32_t* __restrict__ e2e,
                             const int32_t* __restrict__ bface, const int32_t* __restrict__ bnode, int64_t nbn,
                             int32_t* __restrict__ ecnt, int32_t* __restrict__ bcnt, int pass,
                             const int64_t* __restrict__ eoff, int32_t* __restrict__ efill, int32_t* __restrict__ eent,
                             const int64_t* __restrict__ boff, int32_t* __restrict__ bfill, int32_t* __restrict__ bent) {
    constexpr int NLE = DIM == 3 ? 6 : 3;
    GLOOP(B, nbf) {
        const int32_t f = bowner[B];
        const int64_t E = f >> 2;
        const int o = f & 3;
        for (int l = 0; l < NLE; l++) {
            const int p0 = DIM == 3 ? c_le3c[l][0] : c_le2c[l][0];
            const int p1 = DIM == 3 ? c_le3c[l][1] : c_le2c[l][1];
            if (p0 == o || p1 == o) continue;
            const int32_t e = e2e[E * NLE + l];
            if (pass == 0) atomicAdd(&ecnt[e], 1);
            else eent[eoff[e] + atomicAdd(&efill[e], 1)] = (int32_t)B;
        }
        for (int a = 0; a < DIM; a++) {
            const int64_t k = bnode_index(bnode, nbn, bface[DIM * B + a]);
            if (k < 0) continue;
            if (pass == 0) atomicAdd(&bcnt[k], 1);
            else bent[boff[k] + atomicAdd(&bfill[k], 1)] = (int32_t)B;
        }
    }
}

__global__ void k_sort_lists(int64_t nkeys, const int64_t* __restrict__ off, int32_t* __restrict__ ent) {
    GLOOP(k, nkeys) {
        const int64_t a = off[k], b = off[k + 1];
        for (int64_t i = a + 1; i < b; i++) {
            const int32_t t = ent[i];
            int64_t j = i - 1;
            while (j >= a && ent[j] > t) { ent[j + 1] = ent[j]; j--; }
            ent[j + 1] = t;
        }
    }
}

// edge-based volume (Sec. 4.1): node -> incident edges, ascending
__global__ void k_edge_node_count(int64_t n_edges, const int32_t* __restrict__ edges, int32_t* __restrict__ cnt) {
    GLOOP(e, n_edges) {
        atomicAdd(&cnt[edges[2 * e]], 1);
        atomicAdd(&cnt[edges[2 * e + 1]], 1);
    }
}
__global__ void k_edge_node_fill(int64_t n_edges, const int32_t* __restrict__ edges, const int64_t* __restrict__ off,
                                 int32_t* __restrict__ fill, int32_t* __restrict__ ent) {
    GLOOP(e, n_edges) {
        for (int a = 0; a < 2; a++) {
            const int32_t v = edges[2 * e + a];
            ent[off[v] + atomicAdd(&fill[v], 1)] = (int32_t)e;
        }
    }
}
template <int DIM>
__global__ void k_edge_volume(int64_t nv, const int64_t* __restrict__ off, const int32_t* __restrict__ ent,
                              const int32_t* __restrict__ edges, const double* __restrict__ x,
                              const double* __restrict__ n, double* __restrict__ vol) {
    GLOOP(i, nv) {
        double acc = 0.0;
        for (int64_t q = off[i]; q < off[i + 1]; q++) {
            const int64_t e = ent[q];
            const int64_t j = edges[2 * e], k = edges[2 * e + 1];
            double sd = 0.0;
            for (int c = 0; c < DIM; c++) sd = P(sd, M(S(x[DIM * k + c], x[DIM * j + c]), n[DIM * e + c]));
            acc = P(acc, sd);
        }
        vol[i] = M(acc, 1.0 / (2.0 * DIM));
    }
}

// edge-loop residual (Sec. 2): central flux out of the lower end, into the
// upper end, plus F . bnormal at boundary nodes; per node in ascending edge id
__global__ void k_bnode_map(int64_t nbn, const int32_t* __restrict__ bnode, int32_t* __restrict__ bmap) {
    GLOOP(b, nbn) bmap[bnode[b]] = (int32_t)b;
}
template <int DIM>
__global__ void k_edge_residual(int64_t nv, const int64_t* __restrict__ off, const int32_t* __restrict__ ent,
                                const int32_t* __restrict__ edges, const double* __restrict__ F,
                                const double* __restrict__ n, const int32_t* __restrict__ bmap,
                                const double* __restrict__ bnormal, double* __restrict__ res) {
    GLOOP(i, nv) {
        double acc = 0.0;
        for (int64_t q = off[i]; q < off[i + 1]; q++) {
            const int64_t e = ent[q];
            const int64_t j = edges[2 * e], k = edges[2 * e + 1];
            double phi = 0.0;
            for (int c = 0; c < DIM; c++)
                phi = P(phi, M(M(0.5, P(F[DIM * j + c], F[DIM * k + c])), n[DIM * e + c]));
            acc = (j == i) ? P(acc, phi) : S(acc, phi);
        }
        const int32_t b = bmap[i];
        if (b >= 0) {
            double t = 0.0;
            for (int c = 0; c < DIM; c++) t = P(t, M(F[DIM * i + c], bnormal[DIM * int64_t(b) + c]));
            acc = P(acc, t);
        }
        res[i] = acc;
    }
}

#undef GLOOP

inline unsigned Gc(int64_t n) { return grid_for(n, NTC); }

struct CsrWs {
    int32_t *ncnt, *nfill, *nent, *ecnt, *efill, *eent, *bcnt, *bfill, *bent;
    int64_t *noff, *eoff, *boff;
    void* scan;
};

CsrWs csr_layout(const em_mesh* m, void* ws, size_t* bytes) {
    WsLayout L(ws);
    const int nfe = m->dim == 3 ? 3 : 1;
    CsrWs w;
    w.ncnt = L.take<int32_t>(m->n_nodes + 1);
    w.nfill = L.take<int32_t>(m->n_nodes + 1);
    w.noff = L.take<int64_t>(m->n_nodes + 1);
    w.nent = L.take<int32_t>((m->dim + 1) * m->n_elems);
    w.ecnt = L.take<int32_t>(m->n_edges + 1);
    w.efill = L.take<int32_t>(m->n_edges + 1);
    w.eoff = L.take<int64_t>(m->n_edges + 1);
    w.eent = L.take<int32_t>(nfe * m->n_bfaces + 1);
    w.bcnt = L.take<int32_t>(m->n_bnodes + 1);
    w.bfill = L.take<int32_t>(m->n_bnodes + 1);
    w.boff = L.take<int64_t>(m->n_bnodes + 1);
    w.bent = L.take<int32_t>(m->dim * m->n_bfaces + 1);
    int64_t big = m->n_nodes > m->n_edges ? m->n_nodes : m->n_edges;
    w.scan = L.take<char>(scan_ws_bytes(big + 1));
    if (bytes) *bytes = L.bytes();
    return w;
}

struct EvWs {
    int32_t *cnt, *fill, *ent, *bmap;
    int64_t* off;
    void* scan;
};
EvWs ev_layout(const em_mesh* m, void* ws, size_t* bytes) {
    WsLayout L(ws);
    EvWs w;
    w.cnt = L.take<int32_t>(m->n_nodes + 1);
    w.fill = L.take<int32_t>(m->n_nodes + 1);
    w.off = L.take<int64_t>(m->n_nodes + 1);
    w.ent = L.take<int32_t>(2 * m->n_edges);
    w.bmap = L.take<int32_t>(m->n_nodes);
    w.scan = L.take<char>(scan_ws_bytes(m->n_nodes + 1));
    if (bytes) *bytes = L.bytes();
    return w;
}

// node -> incident edges, each list ascending (shared by the edge-based
// volume and the edge-loop residual)
int node_edge_lists(const em_mesh* m, const EvWs& w, cudaStream_t s) {
    EM_CUDA_TRY(cudaMemsetAsync(w.cnt, 0, 4 * (m->n_nodes + 1), s));
    EM_CUDA_TRY(cudaMemsetAsync(w.fill, 0, 4 * (m->n_nodes + 1), s));
    k_edge_node_count<<<Gc(m->n_edges), NTC, 0, s>>>(m->n_edges, m->edges, w.cnt);
    EM_TRY(exclusive_scan_i32_to_i64(w.cnt, w.off, m->n_nodes, w.scan, s));
    k_edge_node_fill<<<Gc(m->n_edges), NTC, 0, s>>>(m->n_edges, m->edges, w.off, w.fill, w.ent);
    k_sort_lists<<<Gc(m->n_nodes), NTC, 0, s>>>(m->n_nodes, w.off, w.ent);
    note_launches(3 + 3);
    return EM_OK;
}

}  // namespace

size_t edge_volume_ws_bytes(const em_mesh* m) {
    size_t b = 0;
    ev_layout(m, nullptr, &b);
    return b;
}

int edge_volume(const em_mesh* m, const double* x, const double* n, double* vol, void* ws, cudaStream_t s) {
    EvWs w = ev_layout(m, ws, nullptr);
    EM_TRY(node_edge_lists(m, w, s));
    if (m->dim == 3) k_edge_volume<3><<<Gc(m->n_nodes), NTC, 0, s>>>(m->n_nodes, w.off, w.ent, m->edges, x, n, vol);
    else k_edge_volume<2><<<Gc(m->n_nodes), NTC, 0, s>>>(m->n_nodes, w.off, w.ent, m->edges, x, n, vol);
    note_launches(1);
    EM_CUDA_TRY(cudaGetLastError());
    return EM_OK;
}

int edge_residual(const em_mesh* m, const double* F, const double* n, const double* bnormal, double* res, void* ws,
                  cudaStream_t s) {
    EvWs w = ev_layout(m, ws, nullptr);
    EM_TRY(node_edge_lists(m, w, s));
    EM_CUDA_TRY(cudaMemsetAsync(w.bmap, 0xff, 4 * m->n_nodes, s));
    if (m->n_bnodes) k_bnode_map<<<Gc(m->n_bnodes), NTC, 0, s>>>(m->n_bnodes, m->bnode, w.bmap);
    if (m->dim == 3)
        k_edge_residual<3><<<Gc(m->n_nodes), NTC, 0, s>>>(m->n_nodes, w.off, w.ent, m->edges, F, n, w.bmap, bnormal, res);
    else
        k_edge_residual<2><<<Gc(m->n_nodes), NTC, 0, s>>>(m->n_nodes, w.off, w.ent, m->edges, F, n, w.bmap, bnormal, res);
    note_launches(m->n_bnodes ? 2 : 1);
    EM_CUDA_TRY(cudaGetLastError());
    return EM_OK;
}

size_t csr_fwd_ws_bytes(const em_mesh* m) {
    size_t b = 0;
    csr_layout(m, nullptr, &b);
    return b;
}

int csr_fwd(const em_mesh* m, const double* x, double* n, double* vol, double* bnormal, void* ws, cudaStream_t s) {
    CsrWs w = csr_layout(m, ws, nullptr);
    const int dim = m->dim;
    // node -> elements
    EM_CUDA_TRY(cudaMemsetAsync(w.ncnt, 0, 4 * (m->n_nodes + 1), s));
    EM_CUDA_TRY(cudaMemsetAsync(w.nfill, 0, 4 * (m->n_nodes + 1), s));
    k_node_keys<<<Gc(m->n_elems), NTC, 0, s>>>(dim, m->n_elems, m->elems, w.ncnt);
    EM_TRY(exclusive_scan_i32_to_i64(w.ncnt, w.noff, m->n_nodes, w.scan, s));
    k_node_fill<<<Gc(m->n_elems), NTC, 0, s>>>(dim, m->n_elems, m->elems, w.noff, w.nfill, w.nent);
    k_sort_lists<<<Gc(m->n_nodes), NTC, 0, s>>>(m->n_nodes, w.noff, w.nent);
    // edge -> boundary faces, boundary node -> boundary faces
    EM_CUDA_TRY(cudaMemsetAsync(w.ecnt, 0, 4 * (m->n_edges + 1), s));
    EM_CUDA_TRY(cudaMemsetAsync(w.efill, 0, 4 * (m->n_edges + 1), s));
    EM_CUDA_TRY(cudaMemsetAsync(w.bcnt, 0, 4 * (m->n_bnodes + 1), s));
    EM_CUDA_TRY(cudaMemsetAsync(w.bfill, 0, 4 * (m->n_bnodes + 1), s));
    int launches = 3;
    for (int pass = 0; pass < 2; pass++) {
        if (pass == 1) {
            EM_TRY(exclusive_scan_i32_to_i64(w.ecnt, w.eoff, m->n_edges, w.scan, s));
            EM_TRY(exclusive_scan_i32_to_i64(w.bcnt, w.boff, m->n_bnodes, w.scan, s));
        }
        if (m->n_bfaces) {
            if (dim == 3)
                k_bface_keys<3><<<Gc(m->n_bfaces), NTC, 0, s>>>(m->n_bfaces, m->bface_owner, m->elem2edge, m->bface,
                                                              m->bnode, m->n_bnodes, w.ecnt, w.bcnt, pass, w.eoff,
                                                              w.efill, w.eent, w.boff, w.bfill, w.bent);
            else
                k_bface_keys<2><<<Gc(m->n_bfaces), NTC, 0, s>>>(m->n_bfaces, m->bface_owner, m->elem2edge, m->bface,
                                                              m->bnode, m->n_bnodes, w.ecnt, w.bcnt, pass, w.eoff,
                                                              w.efill, w.eent, w.boff, w.bfill, w.bent);
            launches++;
        }
    }
    k_sort_lists<<<Gc(m->n_edges), NTC, 0, s>>>(m->n_edges, w.eoff, w.eent);
    k_sort_lists<<<Gc(m->n_bnodes ? m->n_bnodes : 1), NTC, 0, s>>>(m->n_bnodes, w.boff, w.bent);
    if (dim == 3) {
        k_csr_edges<3><<<Gc(m->n_edges), NTC, 0, s>>>(m->n_edges, m->edge_ptr, m->edge_slot, m->elems, x, w.eoff,
                                                     w.eent, m->bface, n);
        k_csr_vol<3><<<Gc(m->n_nodes), NTC, 0, s>>>(m->n_nodes, w.noff, w.nent, m->elems, x, vol);
        k_csr_bnormal<3><<<Gc(m->n_bnodes ? m->n_bnodes : 1), NTC, 0, s>>>(m->n_bnodes, w.boff, w.bent, m->bface, x,
                                                                          bnormal);
    } else {
        k_csr_edges<2><<<Gc(m->n_edges), NTC, 0, s>>>(m->n_edges, m->edge_ptr, m->edge_slot, m->elems, x, w.eoff,
                                                     w.eent, m->bface, n);
        k_csr_vol<2><<<Gc(m->n_nodes), NTC, 0, s>>>(m->n_nodes, w.noff, w.nent, m->elems, x, vol);
        k_csr_bnormal<2><<<Gc(m->n_bnodes ? m->n_bnodes : 1), NTC, 0, s>>>(m->n_bnodes, w.boff, w.bent, m->bface, x,
                                                                          bnormal);
    }
    note_launches(launches + 5);
    EM_CUDA_TRY(cudaGetLastError());
    return EM_OK;
}

}  // namespace em

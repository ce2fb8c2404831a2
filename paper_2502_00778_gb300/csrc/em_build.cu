// edge_build: bit-exact integer topology on the GPU.
//
//   edges      all element edges {j,k}, j < k (Sec. 2), in lexicographic order,
//              from a stable LSD radix sort of packed (min,max) keys + unique;
//   elem2edge  edge id of every local edge (stored node order);
//   CSR        edge -> element slots (the sorted slot ids themselves);
//   bface      faces seen by exactly one element (boundary elements of
//              Sec. 3.2), outward node order, owner element and local face;
//   bnode      ascending ids of the nodes on boundary faces.
#include "em_common.cuh"
#include "em_kernels.cuh"

namespace em {

namespace {

__constant__ int c_le3[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
__constant__ int c_le2[3][2] = {{0, 1}, {0, 2}, {1, 2}};

__device__ __forceinline__ int4 load_elem(const int32_t* elems, int64_t e) {
    return reinterpret_cast<const int4*>(elems)[e];
}
__device__ __forceinline__ int comp(const int4& v, int i) { return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w; }

// status[0]: bad ids, status[1]: degenerate, status[2]: non-manifold faces
__global__ void k_check_ids(int dim, int64_t nv, int64_t ne, const int32_t* __restrict__ elems,
                            unsigned long long* status) {
    unsigned long long bad = 0;
    for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < ne; e += int64_t(gridDim.x) * blockDim.x) {
        int4 v = load_elem(elems, e);
        int k = dim + 1;
        bool ok = true;
        for (int i = 0; i < k; i++) {
            int a = comp(v, i);
            if (a < 0 || a >= nv) ok = false;
            for (int j = 0; j < i; j++)
                if (comp(v, j) == a) ok = false;
        }
        if (dim == 2 && v.w != -1) ok = false;
        bad += ok ? 0 : 1;
    }
    if (bad) atomicAdd(&status[0], bad);
}

__global__ void k_check_degenerate(int dim, int64_t ne, const int32_t* __restrict__ elems, const double* __restrict__ x,
                                   unsigned long long* status) {
    unsigned long long deg = 0;
    for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < ne; e += int64_t(gridDim.x) * blockDim.x) {
        int4 v = load_elem(elems, e);
        double det;
        if (dim == 3) {
            const double* p0 = x + 3 * int64_t(v.x);
            double a[3], b[3], c[3];
            for (int i = 0; i < 3; i++) {
                a[i] = x[3 * int64_t(v.y) + i] - p0[i];
                b[i] = x[3 * int64_t(v.z) + i] - p0[i];
                c[i] = x[3 * int64_t(v.w) + i] - p0[i];
            }
            det = a[0] * (b[1] * c[2] - b[2] * c[1]) - a[1] * (b[0] * c[2] - b[2] * c[0]) + a[2] * (b[0] * c[1] - b[1] * c[0]);
        } else {
            const double* p0 = x + 2 * int64_t(v.x);
            double ax = x[2 * int64_t(v.y)] - p0[0], ay = x[2 * int64_t(v.y) + 1] - p0[1];
            double bx = x[2 * int64_t(v.z)] - p0[0], by = x[2 * int64_t(v.z) + 1] - p0[1];
            det = ax * by - ay * bx;
        }
        deg += (det == 0.0) ? 1 : 0;
    }
    if (deg) atomicAdd(&status[1], deg);
}

// packed edge key (min << b) | max, value = slot e*nle + l
__global__ void k_edge_keys(int dim, int64_t ne, const int32_t* __restrict__ elems, int b, uint64_t* __restrict__ keys,
                            uint32_t* __restrict__ vals) {
    const int nle = dim == 3 ? 6 : 3;
    for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < ne; e += int64_t(gridDim.x) * blockDim.x) {
        int4 v = load_elem(elems, e);
        for (int l = 0; l < nle; l++) {
            int p = comp(v, dim == 3 ? c_le3[l][0] : c_le2[l][0]);
            int q = comp(v, dim == 3 ? c_le3[l][1] : c_le2[l][1]);
            uint64_t j = (uint64_t)(p < q ? p : q), k = (uint64_t)(p < q ? q : p);
            keys[e * nle + l] = (j << b) | k;
            vals[e * nle + l] = (uint32_t)(e * nle + l);
        }
    }
}

__global__ void k_heads(const uint64_t* __restrict__ keys, int64_t n, int32_t* __restrict__ head) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        head[i] = (i == 0 || keys[i] != keys[i - 1]) ? 1 : 0;
}

__global__ void k_edge_emit(const uint64_t* __restrict__ keys, const uint32_t* __restrict__ vals, int64_t n, int b,
                            const int32_t* __restrict__ head, const int64_t* __restrict__ excl,
                            int32_t* __restrict__ edges, int32_t* __restrict__ elem2edge, int32_t* __restrict__ edge_ptr,
                            int32_t* __restrict__ edge_slot) {
    const uint64_t mask = (uint64_t(1) << b) - 1;
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        int64_t e = excl[i] + head[i] - 1;
        uint32_t s = vals[i];
        if (head[i]) {
            uint64_t k = keys[i];
            edges[2 * e] = (int32_t)(k >> b);
            edges[2 * e + 1] = (int32_t)(k & mask);
            if (edge_ptr) edge_ptr[e] = (int32_t)i;
        }
        elem2edge[s] = (int32_t)e;
        if (edge_slot) edge_slot[i] = (int32_t)s;
    }
}

__global__ void k_set_i32(int32_t* p, int64_t i, int32_t v) { p[i] = v; }

// ---- 3D boundary faces ----------------------------------------------------
__device__ __forceinline__ void face_nodes(const int32_t* elems, uint32_t f, int& p, int& q, int& r) {
    int4 v = load_elem(elems, f >> 2);
    int o = f & 3;
    int a[3], c = 0;
    for (int i = 0; i < 4; i++)
        if (i != o) a[c++] = comp(v, i);
    // sort 3
    if (a[0] > a[1]) { int t = a[0]; a[0] = a[1]; a[1] = t; }
    if (a[1] > a[2]) { int t = a[1]; a[1] = a[2]; a[2] = t; }
    if (a[0] > a[1]) { int t = a[0]; a[0] = a[1]; a[1] = t; }
    p = a[0]; q = a[1]; r = a[2];
}

__global__ void k_face_keys_r(int64_t ne, const int32_t* __restrict__ elems, uint64_t* __restrict__ keys,
                              uint32_t* __restrict__ vals) {
    for (int64_t f = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; f < 4 * ne; f += int64_t(gridDim.x) * blockDim.x) {
        int p, q, r;
        face_nodes(elems, (uint32_t)f, p, q, r);
        keys[f] = (uint64_t)r;
        vals[f] = (uint32_t)f;
    }
}

__global__ void k_face_keys_pq(int64_t n, const int32_t* __restrict__ elems, int b, const uint32_t* __restrict__ vin,
                               uint64_t* __restrict__ keys, uint32_t* __restrict__ vals) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        uint32_t f = vin[i];
        int p, q, r;
        face_nodes(elems, f, p, q, r);
        keys[i] = ((uint64_t)p << b) | (uint64_t)q;
        vals[i] = f;
    }
}

__device__ __forceinline__ bool same_face(const int32_t* elems, uint32_t f, uint32_t g) {
    int p, q, r, p2, q2, r2;
    face_nodes(elems, f, p, q, r);
    face_nodes(elems, g, p2, q2, r2);
    return p == p2 && q == q2 && r == r2;
}

__global__ void k_face_flags(int64_t n, const int32_t* __restrict__ elems, const uint32_t* __restrict__ vals,
                             int32_t* __restrict__ bflag, unsigned long long* status) {
    unsigned long long bad = 0;
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        bool head = (i == 0) || !same_face(elems, vals[i], vals[i - 1]);
        bool tail = (i == n - 1) || !same_face(elems, vals[i], vals[i + 1]);
        bflag[i] = (head && tail) ? 1 : 0;
        if (head && !tail && i + 2 < n && same_face(elems, vals[i], vals[i + 2])) bad++;
    }
    if (bad) atomicAdd(&status[2], bad);
}

// orientation test in FP64 with explicit rounding (no FMA contraction), the
// same operation sequence as the CPU definition
__device__ __forceinline__ void orient_face3(const double* x, int& p, int& q, int& r, int o) {
    const double* xp = x + 3 * int64_t(p);
    const double* xq = x + 3 * int64_t(q);
    const double* xr = x + 3 * int64_t(r);
    const double* xo = x + 3 * int64_t(o);
    double u0 = __dsub_rn(xq[0], xp[0]), u1 = __dsub_rn(xq[1], xp[1]), u2 = __dsub_rn(xq[2], xp[2]);
    double t0 = __dsub_rn(xr[0], xp[0]), t1 = __dsub_rn(xr[1], xp[1]), t2 = __dsub_rn(xr[2], xp[2]);
    double n0 = __dmul_rn(__dsub_rn(__dmul_rn(u1, t2), __dmul_rn(u2, t1)), 0.5);
    double n1 = __dmul_rn(__dsub_rn(__dmul_rn(u2, t0), __dmul_rn(u0, t2)), 0.5);
    double n2 = __dmul_rn(__dsub_rn(__dmul_rn(u0, t1), __dmul_rn(u1, t0)), 0.5);
    double d0 = __dsub_rn(xo[0], xp[0]), d1 = __dsub_rn(xo[1], xp[1]), d2 = __dsub_rn(xo[2], xp[2]);
    double s = __dadd_rn(__dadd_rn(__dmul_rn(n0, d0), __dmul_rn(n1, d1)), __dmul_rn(n2, d2));
    if (s > 0) { int t = q; q = r; r = t; }
}

__global__ void k_face_emit3(int64_t n, const int32_t* __restrict__ elems, const double* __restrict__ x,
                             const uint32_t* __restrict__ vals, const int32_t* __restrict__ bflag,
                             const int64_t* __restrict__ pos, int32_t* __restrict__ bface, int32_t* __restrict__ bowner) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        if (!bflag[i]) continue;
        uint32_t f = vals[i];
        int p, q, r;
        face_nodes(elems, f, p, q, r);
        int4 v = load_elem(elems, f >> 2);
        int o = comp(v, f & 3);
        orient_face3(x, p, q, r, o);
        int64_t B = pos[i];
        bface[3 * B] = p; bface[3 * B + 1] = q; bface[3 * B + 2] = r;
        bowner[B] = (int32_t)f;
    }
}

// ---- 2D boundary edges: edges with a single slot ------------------------
__global__ void k_bedge_flags(const int32_t* __restrict__ head, int64_t n, int32_t* __restrict__ bflag) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        bool tail = (i == n - 1) || head[i + 1];
        bflag[i] = (head[i] && tail) ? 1 : 0;
    }
}

__global__ void k_bedge_emit2(int64_t n, const int32_t* __restrict__ elems, const double* __restrict__ x,
                              const uint32_t* __restrict__ vals, const int32_t* __restrict__ bflag,
                              const int64_t* __restrict__ pos, int32_t* __restrict__ bface, int32_t* __restrict__ bowner) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        if (!bflag[i]) continue;
        uint32_t s = vals[i];
        int64_t E = s / 3;
        int l = s % 3;
        int4 v = load_elem(elems, E);
        int lp = c_le2[l][0], lq = c_le2[l][1];
        int lo = 3 - lp - lq;
        int p = comp(v, lp), q = comp(v, lq), o = comp(v, lo);
        int a = p < q ? p : q, c = p < q ? q : p;
        const double* xa = x + 2 * int64_t(a);
        const double* xc = x + 2 * int64_t(c);
        const double* xo = x + 2 * int64_t(o);
        double n0 = __dsub_rn(xa[1], xc[1]), n1 = __dsub_rn(xc[0], xa[0]);
        double d0 = __dsub_rn(xo[0], xa[0]), d1 = __dsub_rn(xo[1], xa[1]);
        double sdot = __dadd_rn(__dmul_rn(n0, d0), __dmul_rn(n1, d1));
        if (sdot > 0) { int t = a; a = c; c = t; }
        int64_t B = pos[i];
        bface[2 * B] = a; bface[2 * B + 1] = c;
        bowner[B] = (int32_t)(E * 4 + lo);
    }
}

// ---- boundary nodes -----------------------------------------------------
__global__ void k_mark_bnodes(int dim, int64_t nb, const int32_t* __restrict__ bface, int32_t* __restrict__ mark) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < nb * dim; i += int64_t(gridDim.x) * blockDim.x)
        mark[bface[i]] = 1;
}

__global__ void k_emit_bnodes(int64_t nv, const int32_t* __restrict__ mark, const int64_t* __restrict__ pos,
                              int32_t* __restrict__ bnode) {
    for (int64_t v = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; v < nv; v += int64_t(gridDim.x) * blockDim.x)
        if (mark[v]) bnode[pos[v]] = (int32_t)v;
}

}  // namespace

// ---------------------------------------------------------------------------
int edge_build_impl(int dim, int64_t nv, int64_t ne, const int32_t* elems, const double* x, void* ws, size_t* ws_bytes,
                    int32_t* edges, int64_t edges_cap, int32_t* elem2edge, int32_t* edge_ptr, int32_t* edge_slot,
                    int32_t* bface, int32_t* bowner, int64_t bface_cap, int32_t* bnode, int64_t bnode_cap,
                    int64_t* counts, cudaStream_t s) {
    if (dim != 2 && dim != 3) return fail(EM_ERR_ARG, "dim must be 2 or 3");
    if (nv <= 0 || ne <= 0 || nv >= INT32_MAX || ne >= INT32_MAX) return fail(EM_ERR_ARG, "bad n_nodes / n_elems");
    const int nle = dim == 3 ? 6 : 3;
    const int64_t nslots = ne * nle;
    if (nslots >= INT32_MAX) return fail(EM_ERR_ARG, "n_elems * edges per element must be < 2^31");
    const int64_t nf = dim == 3 ? 4 * ne : nslots;
    const int64_t nsort = nslots > nf ? nslots : nf;
    const int b = bits_for(nv - 1);

    WsLayout L(ws);
    uint64_t* keys = L.take<uint64_t>(nsort);
    uint32_t* vals = L.take<uint32_t>(nsort);
    uint64_t* kt = L.take<uint64_t>(nsort);
    uint32_t* vt = L.take<uint32_t>(nsort);
    void* sort_ws = L.take<char>(radix_sort_ws_bytes(nsort));
    int32_t* head = L.take<int32_t>(nsort);
    int64_t* excl = L.take<int64_t>(nsort + 1);
    int32_t* bflag = L.take<int32_t>(nsort);
    int64_t* bpos = L.take<int64_t>(nsort + 1);
    int32_t* mark = L.take<int32_t>(nv);
    int64_t* mpos = L.take<int64_t>(nv + 1);
    void* scan_ws = L.take<char>(scan_ws_bytes(nsort > nv ? nsort : nv));
    unsigned long long* status = L.take<unsigned long long>(4);
    bool query;
    EM_TRY(check_ws(ws, ws_bytes, L.bytes(), &query));
    if (query) return EM_OK;
    if (!elems || !x || !edges || !elem2edge || !bface || !bowner || !bnode || !counts)
        return fail(EM_ERR_ARG, "null pointer argument");

    const int T = 256;
    EM_CUDA_TRY(cudaMemsetAsync(status, 0, 4 * sizeof(unsigned long long), s));
    k_check_ids<<<grid_for(ne, T), T, 0, s>>>(dim, nv, ne, elems, status);
    unsigned long long st[4];
    EM_CUDA_TRY(cudaMemcpyAsync(st, status, sizeof(st), cudaMemcpyDeviceToHost, s));
    EM_CUDA_TRY(cudaStreamSynchronize(s));
    if (st[0]) return fail(EM_ERR_BAD_ID, std::to_string(st[0]) + " element(s) with node ids out of range or repeated");

    // edges
    k_edge_keys<<<grid_for(ne, T), T, 0, s>>>(dim, ne, elems, b, keys, vals);
    EM_TRY(radix_sort_pairs(keys, vals, kt, vt, nslots, 2 * b, sort_ws, s));
    k_heads<<<grid_for(nslots, T), T, 0, s>>>(keys, nslots, head);
    EM_TRY(exclusive_scan_i32_to_i64(head, excl, nslots, scan_ws, s));
    int64_t n_edges = 0;
    EM_CUDA_TRY(cudaMemcpyAsync(&n_edges, excl + nslots, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    EM_CUDA_TRY(cudaStreamSynchronize(s));
    counts[0] = n_edges;
    counts[1] = counts[2] = 0;
    if (n_edges > edges_cap) return fail(EM_ERR_CAPACITY, "edges_cap too small: need " + std::to_string(n_edges));
    k_edge_emit<<<grid_for(nslots, T), T, 0, s>>>(keys, vals, nslots, b, head, excl, edges, elem2edge, edge_ptr, edge_slot);
    if (edge_ptr) k_set_i32<<<1, 1, 0, s>>>(edge_ptr, n_edges, (int32_t)nslots);
    EM_CUDA_TRY(cudaGetLastError());

    // boundary faces
    int64_t n_bf = 0;
    if (dim == 3) {
        k_face_keys_r<<<grid_for(nf, T), T, 0, s>>>(ne, elems, keys, vals);
        EM_TRY(radix_sort_pairs(keys, vals, kt, vt, nf, b, sort_ws, s));
        k_face_keys_pq<<<grid_for(nf, T), T, 0, s>>>(nf, elems, b, vals, kt, vt);
        EM_TRY(radix_sort_pairs(kt, vt, keys, vals, nf, 2 * b, sort_ws, s));
        k_face_flags<<<grid_for(nf, T), T, 0, s>>>(nf, elems, vt, bflag, status);
        EM_TRY(exclusive_scan_i32_to_i64(bflag, bpos, nf, scan_ws, s));
        EM_CUDA_TRY(cudaMemcpyAsync(&n_bf, bpos + nf, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        EM_CUDA_TRY(cudaMemcpyAsync(st, status, sizeof(st), cudaMemcpyDeviceToHost, s));
        EM_CUDA_TRY(cudaStreamSynchronize(s));
        if (st[2]) return fail(EM_ERR_TOPOLOGY, std::to_string(st[2]) + " face(s) shared by more than two elements");
        counts[1] = n_bf;
        if (n_bf > bface_cap) return fail(EM_ERR_CAPACITY, "bface_cap too small: need " + std::to_string(n_bf));
        k_face_emit3<<<grid_for(nf, T), T, 0, s>>>(nf, elems, x, vt, bflag, bpos, bface, bowner);
    } else {
        k_bedge_flags<<<grid_for(nslots, T), T, 0, s>>>(head, nslots, bflag);
        EM_TRY(exclusive_scan_i32_to_i64(bflag, bpos, nslots, scan_ws, s));
        EM_CUDA_TRY(cudaMemcpyAsync(&n_bf, bpos + nslots, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        EM_CUDA_TRY(cudaStreamSynchronize(s));
        counts[1] = n_bf;
        if (n_bf > bface_cap) return fail(EM_ERR_CAPACITY, "bface_cap too small: need " + std::to_string(n_bf));
        k_bedge_emit2<<<grid_for(nslots, T), T, 0, s>>>(nslots, elems, x, vals, bflag, bpos, bface, bowner);
    }
    EM_CUDA_TRY(cudaGetLastError());

    // boundary nodes
    EM_CUDA_TRY(cudaMemsetAsync(mark, 0, sizeof(int32_t) * nv, s));
    if (n_bf) k_mark_bnodes<<<grid_for(n_bf * dim, T), T, 0, s>>>(dim, n_bf, bface, mark);
    EM_TRY(exclusive_scan_i32_to_i64(mark, mpos, nv, scan_ws, s));
    int64_t n_bn = 0;
    EM_CUDA_TRY(cudaMemcpyAsync(&n_bn, mpos + nv, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    EM_CUDA_TRY(cudaStreamSynchronize(s));
    counts[2] = n_bn;
    if (n_bn > bnode_cap) return fail(EM_ERR_CAPACITY, "bnode_cap too small: need " + std::to_string(n_bn));
    k_emit_bnodes<<<grid_for(nv, T), T, 0, s>>>(nv, mark, mpos, bnode);
    EM_CUDA_TRY(cudaGetLastError());
    EM_CUDA_TRY(cudaStreamSynchronize(s));
    return EM_OK;
}

size_t check_elements_ws_bytes() { return 256; }

int check_elements_impl(int dim, int64_t nv, int64_t ne, const int32_t* elems, const double* x, void* ws,
                        int64_t* counts, cudaStream_t s) {
    if (dim != 2 && dim != 3) return fail(EM_ERR_ARG, "dim must be 2 or 3");
    if (!elems || !x || !counts || ne < 0 || nv <= 0) return fail(EM_ERR_ARG, "bad arguments");
    unsigned long long* status = static_cast<unsigned long long*>(ws);
    EM_CUDA_TRY(cudaMemsetAsync(status, 0, 4 * sizeof(unsigned long long), s));
    const int T = 256;
    unsigned long long st[4] = {0, 0, 0, 0};
    if (ne) k_check_ids<<<grid_for(ne, T), T, 0, s>>>(dim, nv, ne, elems, status);
    EM_CUDA_TRY(cudaMemcpyAsync(st, status, sizeof(st), cudaMemcpyDeviceToHost, s));
    EM_CUDA_TRY(cudaStreamSynchronize(s));
    if (st[0] == 0 && ne) {
        k_check_degenerate<<<grid_for(ne, T), T, 0, s>>>(dim, ne, elems, x, status);
        EM_CUDA_TRY(cudaMemcpyAsync(st, status, sizeof(st), cudaMemcpyDeviceToHost, s));
        EM_CUDA_TRY(cudaStreamSynchronize(s));
    }
    counts[0] = (int64_t)st[0];
    counts[1] = (int64_t)st[1];
    if (st[0]) return fail(EM_ERR_BAD_ID, std::to_string(st[0]) + " element(s) with bad node ids");
    if (st[1]) return fail(EM_ERR_DEGENERATE, std::to_string(st[1]) + " degenerate element(s)");
    return EM_OK;
}

}  // namespace em

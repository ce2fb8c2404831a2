// EM_PATH_ATOMIC: element-centric scatter with global atomics.
//
// One thread per element.  With a, b, c the edge vectors from the element's
// first stored node and N1 = b x c, N2 = c x a, N3 = a x b, det = a . N1,
// s = sign(det), the outward area vector of the face opposite stored node i
// is n_i = -s N_i / 2 (i = 1..3) and n_0 = -(n_1 + n_2 + n_3).  The proposed
// algorithm (Eq. efficient_njk_formula_general_D) adds 2/(D(D+1)) n_j to edge
// {j,k}, j the lower global id; the element-based volume (Sec. 4.2) adds
// |det|/D! /(D+1) to every node.  The boundary correction n_B/(D(D+1)) and
// the boundary dual-face normal n_B/D (Sec. 3.2.3) come from a second kernel
// over boundary faces.
//
// Adjoint of L = sum_e w_e.n_e + sum_i c_i V_i: with W_i the sum of w over the
// element's edges whose lower end is node i, A_i = W_i - W_0 and C = sum c_i,
//   L_E = -(s/12) (A1.N1 + A2.N2 + A3.N3) + C s det / 24          (3D)
// so, using w.(p x q) = p.(q x w):
//   dL/da = -(s/12)(A2 x c - A3 x b) + (C s/24) N1
//   dL/db = -(s/12)(A3 x a - A1 x c) + (C s/24) N2
//   dL/dc = -(s/12)(A1 x b - A2 x a) + (C s/24) N3,  dL/dx_0 = -(sum).
// In 2D n_1 = -s (b_y,-b_x), n_2 = -s (-a_y,a_x), factor 1/3, V_E/3 = |det|/6.
#include <mutex>

#include "em_common.cuh"
#include "em_kernels.cuh"

namespace em {

namespace {

__constant__ int c_le3a[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
__constant__ int c_le2a[3][2] = {{0, 1}, {0, 2}, {1, 2}};


struct d3 { double x, y, z; };
__device__ __forceinline__ d3 mk(double a, double b, double c) { return {a, b, c}; }
__device__ __forceinline__ d3 operator-(d3 a, d3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ d3 operator+(d3 a, d3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ d3 operator*(double s, d3 a) { return {s * a.x, s * a.y, s * a.z}; }
__device__ __forceinline__ d3 cross(d3 a, d3 b) { return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x}; }
__device__ __forceinline__ double dot(d3 a, d3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ d3 ld3(const double* x, int64_t i) { return {x[3 * i], x[3 * i + 1], x[3 * i + 2]}; }

struct f3 { float x, y, z; };
__device__ __forceinline__ f3 operator-(f3 a, f3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ f3 operator+(f3 a, f3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ f3 operator*(float s, f3 a) { return {s * a.x, s * a.y, s * a.z}; }
__device__ __forceinline__ f3 cross(f3 a, f3 b) { return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x}; }
__device__ __forceinline__ float dot(f3 a, f3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ f3 tof(d3 a) { return {(float)a.x, (float)a.y, (float)a.z}; }

// compensated FP32 atomic accumulation into (hi, lo)
__device__ __forceinline__ void comp_add(float* hi, float* lo, float v) {
    float old = atomicAdd(hi, v);
    float s = __fadd_rn(old, v);
    float bb = __fsub_rn(s, old);
    float err = __fadd_rn(__fsub_rn(old, __fsub_rn(s, bb)), __fsub_rn(v, bb));
    atomicAdd(lo, err);
}

// ---- the traditional dual-face construction (Sec. 3.1), for comparison ------
// Per element and per element edge {j,k} (j the lower global id): the part of
// the edge's dual face inside the element, built from the edge midpoint, the
// centroids of the element's two faces that contain the edge and the element
// centroid (3D: two triangles; 2D: the segment from the edge midpoint to the
// element centroid), each directed from j to k, added with FP64 atomics.  In
// element-local coordinates (the first stored node subtracted).
__global__ void k_trad_atomic3(int64_t ne, const int32_t* __restrict__ elems, const int32_t* __restrict__ e2e,
                               const double* __restrict__ x, double* __restrict__ n) {
    for (int64_t E = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; E < ne; E += int64_t(gridDim.x) * blockDim.x) {
        const int4 v = reinterpret_cast<const int4*>(elems)[E];
        const d3 x0 = ld3(x, v.x);
        d3 p[4] = {mk(0.0, 0.0, 0.0), ld3(x, v.y) - x0, ld3(x, v.z) - x0, ld3(x, v.w) - x0};
        const int gid[4] = {v.x, v.y, v.z, v.w};
        const d3 xE = 0.25 * (p[0] + p[1] + p[2] + p[3]);
#pragma unroll
        for (int l = 0; l < 6; l++) {
            const int a = c_le3a[l][0], b = c_le3a[l][1];
            const int jl = gid[a] < gid[b] ? a : b, kl = jl == a ? b : a;
            const int ll = (a == 0 || b == 0) ? (a == 1 || b == 1 ? 2 : 1) : 0;
            const int rl = 6 - a - b - ll;
            const d3 djk = p[kl] - p[jl];
            const d3 xm = 0.5 * (p[jl] + p[kl]);
            const d3 xL = (1.0 / 3.0) * (p[jl] + p[ll] + p[kl]);
            const d3 xR = (1.0 / 3.0) * (p[jl] + p[rl] + p[kl]);
            const d3 Em = xE - xm;
            d3 nEL = 0.5 * cross(Em, xL - xm), nER = 0.5 * cross(xR - xm, Em);
            if (dot(nEL, djk) < 0) nEL = -1.0 * nEL;
            if (dot(nER, djk) < 0) nER = -1.0 * nER;
            const int64_t e = e2e[E * 6 + l];
            atomicAdd(n + 3 * e, nEL.x + nER.x);
            atomicAdd(n + 3 * e + 1, nEL.y + nER.y);
            atomicAdd(n + 3 * e + 2, nEL.z + nER.z);
        }
    }
}

__global__ void k_trad_atomic2(int64_t ne, const int32_t* __restrict__ elems, const int32_t* __restrict__ e2e,
                               const double* __restrict__ x, double* __restrict__ n) {
    for (int64_t E = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; E < ne; E += int64_t(gridDim.x) * blockDim.x) {
        const int4 v = reinterpret_cast<const int4*>(elems)[E];
        const int gid[3] = {v.x, v.y, v.z};
        const double x0 = x[2 * int64_t(v.x)], y0 = x[2 * int64_t(v.x) + 1];
        double px[3] = {0.0, x[2 * int64_t(v.y)] - x0, x[2 * int64_t(v.z)] - x0};
        double py[3] = {0.0, x[2 * int64_t(v.y) + 1] - y0, x[2 * int64_t(v.z) + 1] - y0};
        const double xE = (px[0] + px[1] + px[2]) * (1.0 / 3.0), yE = (py[0] + py[1] + py[2]) * (1.0 / 3.0);
#pragma unroll
        for (int l = 0; l < 3; l++) {
            const int a = c_le2a[l][0], b = c_le2a[l][1];
            const int jl = gid[a] < gid[b] ? a : b, kl = jl == a ? b : a;
            const double xm = 0.5 * (px[jl] + px[kl]), ym = 0.5 * (py[jl] + py[kl]);
            double nx = ym - yE, ny = xE - xm;
            if (nx * (px[kl] - px[jl]) + ny * (py[kl] - py[jl]) < 0) {
                nx = -nx;
                ny = -ny;
            }
            const int64_t e = e2e[E * 3 + l];
            atomicAdd(n + 2 * e, nx);
            atomicAdd(n + 2 * e + 1, ny);
        }
    }
}

// ---- forward, 3D ----------------------------------------------------------
template <int PREC>
__global__ void k_fwd_atomic3(int64_t ne, const int32_t* __restrict__ elems, const int32_t* __restrict__ e2e,
                              const double* __restrict__ x, double* __restrict__ n, double* __restrict__ vol,
                              float* __restrict__ nhi, float* __restrict__ nlo, float* __restrict__ vhi,
                              float* __restrict__ vlo) {
    for (int64_t E = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; E < ne; E += int64_t(gridDim.x) * blockDim.x) {
        int4 v = reinterpret_cast<const int4*>(elems)[E];
        d3 p0 = ld3(x, v.x), p1 = ld3(x, v.y), p2 = ld3(x, v.z), p3 = ld3(x, v.w);
        d3 m[4];
        double vq;
        if (PREC == EM_PREC_FP64) {
            d3 a = p1 - p0, b = p2 - p0, c = p3 - p0;
            d3 N1 = cross(b, c), N2 = cross(c, a), N3 = cross(a, b);
            double det = dot(a, N1);
            double f = det > 0 ? -1.0 / 12.0 : 1.0 / 12.0;
            m[1] = f * N1; m[2] = f * N2; m[3] = f * N3;
            m[0] = -1.0 * (m[1] + m[2] + m[3]);
            vq = fabs(det) * (1.0 / 24.0);
        } else {
            // FP32 element arithmetic on coordinates relative to the first node
            f3 a = tof(p1 - p0), b = tof(p2 - p0), c = tof(p3 - p0);
            f3 N1 = cross(b, c), N2 = cross(c, a), N3 = cross(a, b);
            float det = dot(a, N1);
            float f = det > 0 ? -1.0f / 12.0f : 1.0f / 12.0f;
            f3 q1 = f * N1, q2 = f * N2, q3 = f * N3;
            f3 q0 = -1.0f * (q1 + q2 + q3);
            m[0] = mk(q0.x, q0.y, q0.z); m[1] = mk(q1.x, q1.y, q1.z);
            m[2] = mk(q2.x, q2.y, q2.z); m[3] = mk(q3.x, q3.y, q3.z);
            vq = fabsf(det) * (1.0f / 24.0f);
        }
        int gid[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int l = 0; l < 6; l++) {
            int p = c_le3a[l][0], q = c_le3a[l][1];
            int lo = gid[p] < gid[q] ? p : q;
            int64_t e = e2e[E * 6 + l];
            if (PREC == EM_PREC_MIXED_COMP32) {
                comp_add(nhi + 3 * e, nlo + 3 * e, (float)m[lo].x);
                comp_add(nhi + 3 * e + 1, nlo + 3 * e + 1, (float)m[lo].y);
                comp_add(nhi + 3 * e + 2, nlo + 3 * e + 2, (float)m[lo].z);
            } else {
                atomicAdd(n + 3 * e, m[lo].x);
                atomicAdd(n + 3 * e + 1, m[lo].y);
                atomicAdd(n + 3 * e + 2, m[lo].z);
            }
        }
        if (vol || vhi) {
#pragma unroll
            for (int i = 0; i < 4; i++) {
                if (PREC == EM_PREC_MIXED_COMP32) comp_add(vhi + gid[i], vlo + gid[i], (float)vq);
                else atomicAdd(vol + gid[i], vq);
            }
        }
    }
}

// ---- forward, 2D ----------------------------------------------------------
template <int PREC>
__global__ void k_fwd_atomic2(int64_t ne, const int32_t* __restrict__ elems, const int32_t* __restrict__ e2e,
                              const double* __restrict__ x, double* __restrict__ n, double* __restrict__ vol,
                              float* __restrict__ nhi, float* __restrict__ nlo, float* __restrict__ vhi,
                              float* __restrict__ vlo) {
    for (int64_t E = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; E < ne; E += int64_t(gridDim.x) * blockDim.x) {
        int4 v = reinterpret_cast<const int4*>(elems)[E];
        double m[3][2];
        double vq;
        double ax = x[2 * int64_t(v.y)] - x[2 * int64_t(v.x)], ay = x[2 * int64_t(v.y) + 1] - x[2 * int64_t(v.x) + 1];
        double bx = x[2 * int64_t(v.z)] - x[2 * int64_t(v.x)], by = x[2 * int64_t(v.z) + 1] - x[2 * int64_t(v.x) + 1];
        if (PREC == EM_PREC_FP64) {
            double det = ax * by - ay * bx;
            double f = det > 0 ? -1.0 / 3.0 : 1.0 / 3.0;   // n_i/3 with n_1 = -s (b_y,-b_x), n_2 = -s (-a_y,a_x)
            m[1][0] = f * by; m[1][1] = -f * bx;
            m[2][0] = -f * ay; m[2][1] = f * ax;
            m[0][0] = -(m[1][0] + m[2][0]); m[0][1] = -(m[1][1] + m[2][1]);
            vq = fabs(det) * (1.0 / 6.0);
        } else {
            float fax = (float)ax, fay = (float)ay, fbx = (float)bx, fby = (float)by;
            float det = fax * fby - fay * fbx;
            float f = det > 0 ? -1.0f / 3.0f : 1.0f / 3.0f;
            float q1x = f * fby, q1y = -f * fbx, q2x = -f * fay, q2y = f * fax;
            m[1][0] = q1x; m[1][1] = q1y; m[2][0] = q2x; m[2][1] = q2y;
            m[0][0] = -(q1x + q2x); m[0][1] = -(q1y + q2y);
            vq = fabsf(det) * (1.0f / 6.0f);
        }
        int gid[3] = {v.x, v.y, v.z};
#pragma unroll
        for (int l = 0; l < 3; l++) {
            int p = c_le2a[l][0], q = c_le2a[l][1];
            int lo = gid[p] < gid[q] ? p : q;
            int64_t e = e2e[E * 3 + l];
            if (PREC == EM_PREC_MIXED_COMP32) {
                comp_add(nhi + 2 * e, nlo + 2 * e, (float)m[lo][0]);
                comp_add(nhi + 2 * e + 1, nlo + 2 * e + 1, (float)m[lo][1]);
            } else {
                atomicAdd(n + 2 * e, m[lo][0]);
                atomicAdd(n + 2 * e + 1, m[lo][1]);
            }
        }
        if (vol || vhi) {
#pragma unroll
            for (int i = 0; i < 3; i++) {
                if (PREC == EM_PREC_MIXED_COMP32) comp_add(vhi + gid[i], vlo + gid[i], (float)vq);
                else atomicAdd(vol + gid[i], vq);
            }
        }
    }
}

__global__ void k_comp_finalize(int64_t m, const float* __restrict__ hi, const float* __restrict__ lo,
                                double* __restrict__ out) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < m; i += int64_t(gridDim.x) * blockDim.x)
        out[i] = (double)hi[i] + (double)lo[i];
}

__device__ __forceinline__ int64_t find_bnode(const int32_t* bnode, int64_t nb, int32_t v) {
    int64_t lo = 0, hi = nb - 1;
    while (lo <= hi) {
        int64_t mid = (lo + hi) >> 1;
        int32_t t = bnode[mid];
        if (t == v) return mid;
        if (t < v) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

// boundary faces: correction n_B/(D(D+1)) on the face's edges, n_B/D on its
// nodes; only faces whose owner element lies in [e0, e1)
template <int DIM>
__global__ void k_bnd_atomic(int64_t nbf, const int32_t* __restrict__ bface, const int32_t* __restrict__ bowner,
                             const int32_t* __restrict__ elems, const int32_t* __restrict__ e2e,
                             const double* __restrict__ x, int64_t nbn, const int32_t* __restrict__ bnode,
                             double* __restrict__ n, double* __restrict__ bnormal, int64_t e0, int64_t e1) {
    for (int64_t B = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; B < nbf; B += int64_t(gridDim.x) * blockDim.x) {
        int32_t f = bowner[B];
        int64_t E = f >> 2;
        int o = f & 3;
        if (E < e0 || E >= e1) continue;
        if (DIM == 3) {
            int p = bface[3 * B], q = bface[3 * B + 1], r = bface[3 * B + 2];
            d3 xp = ld3(x, p);
            d3 nB = 0.5 * cross(ld3(x, q) - xp, ld3(x, r) - xp);
            if (n) {
                d3 cB = (1.0 / 12.0) * nB;
                for (int l = 0; l < 6; l++) {
                    if (c_le3a[l][0] == o || c_le3a[l][1] == o) continue;
                    int64_t e = e2e[E * 6 + l];
                    atomicAdd(n + 3 * e, cB.x); atomicAdd(n + 3 * e + 1, cB.y); atomicAdd(n + 3 * e + 2, cB.z);
                }
            }
            if (bnormal) {
                d3 bB = (1.0 / 3.0) * nB;
                int vv[3] = {p, q, r};
                for (int i = 0; i < 3; i++) {
                    int64_t k = find_bnode(bnode, nbn, vv[i]);
                    if (k < 0) continue;
                    atomicAdd(bnormal + 3 * k, bB.x); atomicAdd(bnormal + 3 * k + 1, bB.y); atomicAdd(bnormal + 3 * k + 2, bB.z);
                }
            }
        } else {
            int a = bface[2 * B], b2 = bface[2 * B + 1];
            double nx = x[2 * int64_t(a) + 1] - x[2 * int64_t(b2) + 1], ny = x[2 * int64_t(b2)] - x[2 * int64_t(a)];
            if (n) {
                int l = (o == 0) ? 2 : (o == 1 ? 1 : 0);
                int64_t e = e2e[E * 3 + l];
                atomicAdd(n + 2 * e, nx / 6.0); atomicAdd(n + 2 * e + 1, ny / 6.0);
            }
            if (bnormal) {
                int vv[2] = {a, b2};
                for (int i = 0; i < 2; i++) {
                    int64_t k = find_bnode(bnode, nbn, vv[i]);
                    if (k < 0) continue;
                    atomicAdd(bnormal + 2 * k, 0.5 * nx); atomicAdd(bnormal + 2 * k + 1, 0.5 * ny);
                }
            }
        }
    }
}

// ---- adjoint --------------------------------------------------------------
template <int PREC>
__global__ void k_adj_atomic3(int64_t ne, const int32_t* __restrict__ elems, const int32_t* __restrict__ e2e,
                              const double* __restrict__ x, const double* __restrict__ w, const double* __restrict__ c,
                              double* __restrict__ g) {
    for (int64_t E = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; E < ne; E += int64_t(gridDim.x) * blockDim.x) {
        int4 v = reinterpret_cast<const int4*>(elems)[E];
        int gid[4] = {v.x, v.y, v.z, v.w};
        d3 W[4] = {mk(0, 0, 0), mk(0, 0, 0), mk(0, 0, 0), mk(0, 0, 0)};
#pragma unroll
        for (int l = 0; l < 6; l++) {
            int p = c_le3a[l][0], q = c_le3a[l][1];
            int lo = gid[p] < gid[q] ? p : q;
            W[lo] = W[lo] + ld3(w, e2e[E * 6 + l]);
        }
        double C = c ? (c[gid[0]] + c[gid[1]] + c[gid[2]] + c[gid[3]]) : 0.0;
        d3 p0 = ld3(x, gid[0]);
        d3 a = ld3(x, gid[1]) - p0, b = ld3(x, gid[2]) - p0, cc = ld3(x, gid[3]) - p0;
        d3 ga, gb, gc;
        if (PREC == EM_PREC_FP64) {
            d3 A1 = W[1] - W[0], A2 = W[2] - W[0], A3 = W[3] - W[0];
            d3 N1 = cross(b, cc), N2 = cross(cc, a), N3 = cross(a, b);
            double det = dot(a, N1);
            double s = det > 0 ? 1.0 : -1.0;
            double f = -s / 12.0, h = C * s / 24.0;
            ga = f * (cross(A2, cc) - cross(A3, b)) + h * N1;
            gb = f * (cross(A3, a) - cross(A1, cc)) + h * N2;
            gc = f * (cross(A1, b) - cross(A2, a)) + h * N3;
        } else {
            f3 fa = tof(a), fb = tof(b), fc = tof(cc);
            f3 A1 = tof(W[1] - W[0]), A2 = tof(W[2] - W[0]), A3 = tof(W[3] - W[0]);
            f3 N1 = cross(fb, fc), N2 = cross(fc, fa), N3 = cross(fa, fb);
            float det = dot(fa, N1);
            float s = det > 0 ? 1.0f : -1.0f;
            float f = -s / 12.0f, h = (float)C * s / 24.0f;
            f3 qa = f * (cross(A2, fc) - cross(A3, fb)) + h * N1;
            f3 qb = f * (cross(A3, fa) - cross(A1, fc)) + h * N2;
            f3 qc = f * (cross(A1, fb) - cross(A2, fa)) + h * N3;
            ga = mk(qa.x, qa.y, qa.z); gb = mk(qb.x, qb.y, qb.z); gc = mk(qc.x, qc.y, qc.z);
        }
        d3 g0 = -1.0 * (ga + gb + gc);
        d3 gg[4] = {g0, ga, gb, gc};
#pragma unroll
        for (int i = 0; i < 4; i++) {
            atomicAdd(g + 3 * int64_t(gid[i]), gg[i].x);
            atomicAdd(g + 3 * int64_t(gid[i]) + 1, gg[i].y);
            atomicAdd(g + 3 * int64_t(gid[i]) + 2, gg[i].z);
        }
    }
}

template <int PREC>
__global__ void k_adj_atomic2(int64_t ne, const int32_t* __restrict__ elems, const int32_t* __restrict__ e2e,
                              const double* __restrict__ x, const double* __restrict__ w, const double* __restrict__ c,
                              double* __restrict__ g) {
    for (int64_t E = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; E < ne; E += int64_t(gridDim.x) * blockDim.x) {
        int4 v = reinterpret_cast<const int4*>(elems)[E];
        int gid[3] = {v.x, v.y, v.z};
        double W[3][2] = {{0, 0}, {0, 0}, {0, 0}};
#pragma unroll
        for (int l = 0; l < 3; l++) {
            int p = c_le2a[l][0], q = c_le2a[l][1];
            int lo = gid[p] < gid[q] ? p : q;
            int64_t e = e2e[E * 3 + l];
            W[lo][0] += w[2 * e]; W[lo][1] += w[2 * e + 1];
        }
        double C = c ? (c[gid[0]] + c[gid[1]] + c[gid[2]]) : 0.0;
        double ax = x[2 * int64_t(gid[1])] - x[2 * int64_t(gid[0])], ay = x[2 * int64_t(gid[1]) + 1] - x[2 * int64_t(gid[0]) + 1];
        double bx = x[2 * int64_t(gid[2])] - x[2 * int64_t(gid[0])], by = x[2 * int64_t(gid[2]) + 1] - x[2 * int64_t(gid[0]) + 1];
        double A1x = W[1][0] - W[0][0], A1y = W[1][1] - W[0][1], A2x = W[2][0] - W[0][0], A2y = W[2][1] - W[0][1];
        double gax, gay, gbx, gby;
        double det = ax * by - ay * bx;
        double s = det > 0 ? 1.0 : -1.0;
        double f = s / 3.0, h = C * s / 6.0;
        gax = f * (-A2y) + h * by;  gay = f * A2x - h * bx;
        gbx = f * A1y - h * ay;     gby = -f * A1x + h * ax;
        if (PREC != EM_PREC_FP64) {
            gax = (float)gax; gay = (float)gay; gbx = (float)gbx; gby = (float)gby;
        }
        double gg[3][2] = {{-(gax + gbx), -(gay + gby)}, {gax, gay}, {gbx, gby}};
#pragma unroll
        for (int i = 0; i < 3; i++) {
            atomicAdd(g + 2 * int64_t(gid[i]), gg[i][0]);
            atomicAdd(g + 2 * int64_t(gid[i]) + 1, gg[i][1]);
        }
    }
}

// the boundary faces' part of the adjoint; only faces whose owner element
// lies in [e0, e1)
template <int DIM>
__global__ void k_bnd_adj_atomic(int64_t nbf, const int32_t* __restrict__ bface, const int32_t* __restrict__ bowner,
                                 const int32_t* __restrict__ e2e, const double* __restrict__ x,
                                 const double* __restrict__ w, double* __restrict__ g, int64_t e0, int64_t e1) {
    for (int64_t B = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; B < nbf; B += int64_t(gridDim.x) * blockDim.x) {
        int32_t f = bowner[B];
        int64_t E = f >> 2;
        int o = f & 3;
        if (E < e0 || E >= e1) continue;
        if (DIM == 3) {
            d3 WB = mk(0, 0, 0);
            for (int l = 0; l < 6; l++) {
                if (c_le3a[l][0] == o || c_le3a[l][1] == o) continue;
                WB = WB + ld3(w, e2e[E * 6 + l]);
            }
            int p = bface[3 * B], q = bface[3 * B + 1], r = bface[3 * B + 2];
            d3 xp = ld3(x, p);
            d3 u = ld3(x, q) - xp, t = ld3(x, r) - xp;
            d3 gu = (1.0 / 24.0) * cross(t, WB), gt = (1.0 / 24.0) * cross(WB, u);
            atomicAdd(g + 3 * int64_t(q), gu.x); atomicAdd(g + 3 * int64_t(q) + 1, gu.y); atomicAdd(g + 3 * int64_t(q) + 2, gu.z);
            atomicAdd(g + 3 * int64_t(r), gt.x); atomicAdd(g + 3 * int64_t(r) + 1, gt.y); atomicAdd(g + 3 * int64_t(r) + 2, gt.z);
            atomicAdd(g + 3 * int64_t(p), -(gu.x + gt.x));
            atomicAdd(g + 3 * int64_t(p) + 1, -(gu.y + gt.y));
            atomicAdd(g + 3 * int64_t(p) + 2, -(gu.z + gt.z));
        } else {
            int l = (o == 0) ? 2 : (o == 1 ? 1 : 0);
            int64_t e = e2e[E * 3 + l];
            int a = bface[2 * B], b2 = bface[2 * B + 1];
            double gx = w[2 * e + 1] / 6.0, gy = -w[2 * e] / 6.0;   // d/d(x_b - x_a) of w.(-d_y, d_x)/6
            atomicAdd(g + 2 * int64_t(b2), gx); atomicAdd(g + 2 * int64_t(b2) + 1, gy);
            atomicAdd(g + 2 * int64_t(a), -gx); atomicAdd(g + 2 * int64_t(a) + 1, -gy);
        }
    }
}

// ---- boundary-normal weights: L += sum_b bw_b . bnormal_b ------------------
// bnormal_b = (1/D) sum_{faces B at b} n_B, so each face adds the gradient of
// K.n_B with K = (1/D) sum_{b in B} bw_b (3D n_B = 1/2 (x_q - x_p) x (x_r - x_p),
// 2D n_B = (y_a - y_b, x_b - x_a)).  map[node] = boundary-node index or -1.
__global__ void k_bw_map(int64_t nbn, const int32_t* __restrict__ bnode, int32_t* __restrict__ map) {
    for (int64_t b = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; b < nbn; b += int64_t(gridDim.x) * blockDim.x)
        map[bnode[b]] = (int32_t)b;
}
// order-preserving key (upper word of |v|) of the largest |bw| component
__global__ void k_bw_maxkey(int64_t m, const double* __restrict__ bw, unsigned* __restrict__ key) {
    unsigned k = 0u;
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < m; i += int64_t(gridDim.x) * blockDim.x) {
        // non-finite weights stay out of the bound (their targets become NaN)
        const unsigned ki = (unsigned)((unsigned long long)__double_as_longlong(bw[i]) >> 32) & 0x7fffffffu;
        k = max(k, ki < 0x7ff00000u ? ki : 0u);
    }
    k = __reduce_max_sync(0xffffffffu, k);
    if ((threadIdx.x & 31) == 0) atomicMax(key, k);
}

template <int DIM>
__global__ void k_bnd_bw_adj(int64_t nbf, const int32_t* __restrict__ bface, const double* __restrict__ x,
                             const double* __restrict__ bw, const int32_t* __restrict__ map, double* __restrict__ g) {
    for (int64_t B = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; B < nbf; B += int64_t(gridDim.x) * blockDim.x) {
        if (DIM == 3) {
            const int p = bface[3 * B], q = bface[3 * B + 1], r = bface[3 * B + 2];
            const d3 K = (1.0 / 3.0) * (ld3(bw, map[p]) + ld3(bw, map[q]) + ld3(bw, map[r]));
            const d3 xp = ld3(x, p);
            const d3 u = ld3(x, q) - xp, t = ld3(x, r) - xp;
            const d3 gu = 0.5 * cross(t, K), gt = 0.5 * cross(K, u);
            atomicAdd(g + 3 * int64_t(q), gu.x); atomicAdd(g + 3 * int64_t(q) + 1, gu.y); atomicAdd(g + 3 * int64_t(q) + 2, gu.z);
            atomicAdd(g + 3 * int64_t(r), gt.x); atomicAdd(g + 3 * int64_t(r) + 1, gt.y); atomicAdd(g + 3 * int64_t(r) + 2, gt.z);
            atomicAdd(g + 3 * int64_t(p), -(gu.x + gt.x));
            atomicAdd(g + 3 * int64_t(p) + 1, -(gu.y + gt.y));
            atomicAdd(g + 3 * int64_t(p) + 2, -(gu.z + gt.z));
        } else {
            const int a = bface[2 * B], b2 = bface[2 * B + 1];
            const int64_t ia = map[a], ib = map[b2];
            const double Kx = 0.5 * (bw[2 * ia] + bw[2 * ib]), Ky = 0.5 * (bw[2 * ia + 1] + bw[2 * ib + 1]);
            atomicAdd(g + 2 * int64_t(b2), Ky); atomicAdd(g + 2 * int64_t(b2) + 1, -Kx);
            atomicAdd(g + 2 * int64_t(a), -Ky); atomicAdd(g + 2 * int64_t(a) + 1, Kx);
        }
    }
}

}  // namespace

size_t bw_ws_bytes(const em_mesh* m) { return 256 + sizeof(int32_t) * (size_t)m->n_nodes; }

int bw_prepare(const em_mesh* m, const double* bw, void* ws, BwAux* aux, cudaStream_t s) {
    unsigned* key = static_cast<unsigned*>(ws);
    int32_t* map = reinterpret_cast<int32_t*>(static_cast<char*>(ws) + 256);
    aux->key = key;
    aux->map = map;
    aux->bw = bw;
    if (!bw) return EM_OK;
    if (m->n_bnodes && !m->bnode) return fail(EM_ERR_ARG, "boundary-normal weights need mesh->bnode");
    const int T = 256;
    EM_CUDA_TRY(cudaMemsetAsync(ws, 0, 256, s));
    EM_CUDA_TRY(cudaMemsetAsync(map, 0xff, sizeof(int32_t) * m->n_nodes, s));
    if (m->n_bnodes) {
        k_bw_map<<<grid_for(m->n_bnodes, T), T, 0, s>>>(m->n_bnodes, m->bnode, map);
        k_bw_maxkey<<<grid_for(m->n_bnodes * m->dim, T), T, 0, s>>>(m->n_bnodes * m->dim, bw, key);
        note_launches(2);
    }
    EM_CUDA_TRY(cudaGetLastError());
    return EM_OK;
}

int atomic_bw_adj(const em_mesh* m, const double* x, const BwAux& aux, double* g, cudaStream_t s) {
    if (!aux.bw || !m->n_bfaces) return EM_OK;
    const int T = 256;
    if (m->dim == 3)
        k_bnd_bw_adj<3><<<grid_for(m->n_bfaces, T), T, 0, s>>>(m->n_bfaces, m->bface, x, aux.bw, aux.map, g);
    else
        k_bnd_bw_adj<2><<<grid_for(m->n_bfaces, T), T, 0, s>>>(m->n_bfaces, m->bface, x, aux.bw, aux.map, g);
    note_launches(1);
    EM_CUDA_TRY(cudaGetLastError());
    return EM_OK;
}

int traditional_areas(const em_mesh* m, const double* x, double* n, cudaStream_t s) {
    const int T = 256;
    EM_CUDA_TRY(cudaMemsetAsync(n, 0, sizeof(double) * m->n_edges * m->dim, s));
    const unsigned G = grid_for(m->n_elems, T, int64_t(num_sms()) * 16);
    if (m->dim == 3) k_trad_atomic3<<<G, T, 0, s>>>(m->n_elems, m->elems, m->elem2edge, x, n);
    else k_trad_atomic2<<<G, T, 0, s>>>(m->n_elems, m->elems, m->elem2edge, x, n);
    note_launches(1);
    EM_CUDA_TRY(cudaGetLastError());
    return EM_OK;
}

size_t atomic_fwd_ws_bytes(const em_mesh* m, int prec) {
    WsLayout L(nullptr);
    if (prec == EM_PREC_MIXED_COMP32) {
        L.take<float>(size_t(m->n_edges) * m->dim);
        L.take<float>(size_t(m->n_edges) * m->dim);
        L.take<float>(size_t(m->n_nodes));
        L.take<float>(size_t(m->n_nodes));
    }
    return L.bytes();
}

int atomic_fwd(const em_mesh* m, int prec, const double* x, double* n, double* vol, double* bnormal, void* ws,
               cudaStream_t s) {
    const int T = 256;
    const int dim = m->dim;
    const unsigned G = grid_for(m->n_elems, T, int64_t(num_sms()) * 16);
    float *nhi = nullptr, *nlo = nullptr, *vhi = nullptr, *vlo = nullptr;
    if (prec == EM_PREC_MIXED_COMP32) {
        WsLayout L(ws);
        nhi = L.take<float>(size_t(m->n_edges) * dim);
        nlo = L.take<float>(size_t(m->n_edges) * dim);
        vhi = L.take<float>(size_t(m->n_nodes));
        vlo = L.take<float>(size_t(m->n_nodes));
        EM_CUDA_TRY(cudaMemsetAsync(nhi, 0, sizeof(float) * m->n_edges * dim, s));
        EM_CUDA_TRY(cudaMemsetAsync(nlo, 0, sizeof(float) * m->n_edges * dim, s));
        EM_CUDA_TRY(cudaMemsetAsync(vhi, 0, sizeof(float) * m->n_nodes, s));
        EM_CUDA_TRY(cudaMemsetAsync(vlo, 0, sizeof(float) * m->n_nodes, s));
    } else {
        if (n) EM_CUDA_TRY(cudaMemsetAsync(n, 0, sizeof(double) * m->n_edges * dim, s));
        if (vol) EM_CUDA_TRY(cudaMemsetAsync(vol, 0, sizeof(double) * m->n_nodes, s));
    }
    if (bnormal) EM_CUDA_TRY(cudaMemsetAsync(bnormal, 0, sizeof(double) * m->n_bnodes * dim, s));
    double* vol_arg = (prec == EM_PREC_MIXED_COMP32) ? nullptr : vol;
#define LAUNCH_FWD(K, P) K<P><<<G, T, 0, s>>>(m->n_elems, m->elems, m->elem2edge, x, n, vol_arg, nhi, nlo, vhi, vlo)
    if (dim == 3) {
        if (prec == EM_PREC_FP64) LAUNCH_FWD(k_fwd_atomic3, EM_PREC_FP64);
        else if (prec == EM_PREC_MIXED) LAUNCH_FWD(k_fwd_atomic3, EM_PREC_MIXED);
        else LAUNCH_FWD(k_fwd_atomic3, EM_PREC_MIXED_COMP32);
    } else {
        if (prec == EM_PREC_FP64) LAUNCH_FWD(k_fwd_atomic2, EM_PREC_FP64);
        else if (prec == EM_PREC_MIXED) LAUNCH_FWD(k_fwd_atomic2, EM_PREC_MIXED);
        else LAUNCH_FWD(k_fwd_atomic2, EM_PREC_MIXED_COMP32);
    }
#undef LAUNCH_FWD
    note_launches(1);
    EM_CUDA_TRY(cudaGetLastError());
    if (prec == EM_PREC_MIXED_COMP32) {
        k_comp_finalize<<<grid_for(m->n_edges * dim, T), T, 0, s>>>(m->n_edges * dim, nhi, nlo, n);
        if (vol) k_comp_finalize<<<grid_for(m->n_nodes, T), T, 0, s>>>(m->n_nodes, vhi, vlo, vol);
        note_launches(vol ? 2 : 1);
    }
    if (m->n_bfaces && (n || bnormal)) {
        if (dim == 3)
            k_bnd_atomic<3><<<grid_for(m->n_bfaces, T), T, 0, s>>>(m->n_bfaces, m->bface, m->bface_owner, m->elems,
                                                                  m->elem2edge, x, m->n_bnodes, m->bnode, n, bnormal, 0,
                                                                  INT64_MAX);
        else
            k_bnd_atomic<2><<<grid_for(m->n_bfaces, T), T, 0, s>>>(m->n_bfaces, m->bface, m->bface_owner, m->elems,
                                                                  m->elem2edge, x, m->n_bnodes, m->bnode, n, bnormal, 0,
                                                                  INT64_MAX);
        note_launches(1);
    }
    EM_CUDA_TRY(cudaGetLastError());
    return EM_OK;
}

int atomic_adj(const em_mesh* m, int prec, const double* x, const double* w, const double* c, double* g,
               cudaStream_t s) {
    const int T = 256;
    const int dim = m->dim;
    const unsigned G = grid_for(m->n_elems, T, int64_t(num_sms()) * 16);
    EM_CUDA_TRY(cudaMemsetAsync(g, 0, sizeof(double) * m->n_nodes * dim, s));
    if (dim == 3) {
        if (prec == EM_PREC_FP64) k_adj_atomic3<EM_PREC_FP64><<<G, T, 0, s>>>(m->n_elems, m->elems, m->elem2edge, x, w, c, g);
        else k_adj_atomic3<EM_PREC_MIXED><<<G, T, 0, s>>>(m->n_elems, m->elems, m->elem2edge, x, w, c, g);
    } else {
        if (prec == EM_PREC_FP64) k_adj_atomic2<EM_PREC_FP64><<<G, T, 0, s>>>(m->n_elems, m->elems, m->elem2edge, x, w, c, g);
        else k_adj_atomic2<EM_PREC_MIXED><<<G, T, 0, s>>>(m->n_elems, m->elems, m->elem2edge, x, w, c, g);
    }
    note_launches(1);
    if (m->n_bfaces) {
        if (dim == 3)
            k_bnd_adj_atomic<3><<<grid_for(m->n_bfaces, T), T, 0, s>>>(m->n_bfaces, m->bface, m->bface_owner,
                                                                      m->elem2edge, x, w, g, 0, INT64_MAX);
        else
            k_bnd_adj_atomic<2><<<grid_for(m->n_bfaces, T), T, 0, s>>>(m->n_bfaces, m->bface, m->bface_owner,
                                                                      m->elem2edge, x, w, g, 0, INT64_MAX);
        note_launches(1);
    }
    EM_CUDA_TRY(cudaGetLastError());
    return EM_OK;
}

// ---------------------------------------------------------------------------
// One contiguous range of elements [e0, e1) (a rank's part of a partitioned
// grid): the contributions of its elements, and of the boundary faces whose
// owner element lies in it, to the GLOBAL edge / node / boundary-node arrays.
// Every metric is a sum of such per-element and per-face terms, so the sum of
// the partial arrays of disjoint ranges covering the grid is the full result
// up to rounding order.  FP64 or MIXED, global atomics, no workspace.
// ---------------------------------------------------------------------------
int atomic_partial(const em_mesh* m, int prec, int64_t e0, int64_t e1, const double* x, const double* w,
                   const double* c, double* n, double* vol, double* bnormal, double* g, cudaStream_t s) {
    const int T = 256;
    const int dim = m->dim;
    const int nle = dim == 3 ? 6 : 3;
    const int64_t ne = e1 - e0;
    const int32_t* el = m->elems + 4 * e0;        // 16-byte rows: stays 16-byte aligned
    const int32_t* e2e = m->elem2edge + nle * e0;
    const unsigned G = grid_for(ne > 0 ? ne : 1, T, int64_t(num_sms()) * 16);
    const bool fp64 = prec == EM_PREC_FP64;
    if (n || vol || bnormal) {
        if (n) EM_CUDA_TRY(cudaMemsetAsync(n, 0, sizeof(double) * m->n_edges * dim, s));
        if (vol) EM_CUDA_TRY(cudaMemsetAsync(vol, 0, sizeof(double) * m->n_nodes, s));
        if (bnormal) EM_CUDA_TRY(cudaMemsetAsync(bnormal, 0, sizeof(double) * m->n_bnodes * dim, s));
        if (ne > 0 && (n || vol)) {
            double* nn = n;
            if (!nn) return fail(EM_ERR_ARG, "partial forward: n_edge is required when vol is given");
            if (dim == 3) {
                if (fp64) k_fwd_atomic3<EM_PREC_FP64><<<G, T, 0, s>>>(ne, el, e2e, x, nn, vol, nullptr, nullptr, nullptr, nullptr);
                else k_fwd_atomic3<EM_PREC_MIXED><<<G, T, 0, s>>>(ne, el, e2e, x, nn, vol, nullptr, nullptr, nullptr, nullptr);
            } else {
                if (fp64) k_fwd_atomic2<EM_PREC_FP64><<<G, T, 0, s>>>(ne, el, e2e, x, nn, vol, nullptr, nullptr, nullptr, nullptr);
                else k_fwd_atomic2<EM_PREC_MIXED><<<G, T, 0, s>>>(ne, el, e2e, x, nn, vol, nullptr, nullptr, nullptr, nullptr);
            }
            note_launches(1);
        }
        if (m->n_bfaces && ne > 0 && (n || bnormal)) {
            if (dim == 3)
                k_bnd_atomic<3><<<grid_for(m->n_bfaces, T), T, 0, s>>>(m->n_bfaces, m->bface, m->bface_owner, m->elems,
                                                                      m->elem2edge, x, m->n_bnodes, m->bnode, n,
                                                                      bnormal, e0, e1);
            else
                k_bnd_atomic<2><<<grid_for(m->n_bfaces, T), T, 0, s>>>(m->n_bfaces, m->bface, m->bface_owner, m->elems,
                                                                      m->elem2edge, x, m->n_bnodes, m->bnode, n,
                                                                      bnormal, e0, e1);
            note_launches(1);
        }
    }
    if (g) {
        EM_CUDA_TRY(cudaMemsetAsync(g, 0, sizeof(double) * m->n_nodes * dim, s));
        if (ne > 0) {
            if (dim == 3) {
                if (fp64) k_adj_atomic3<EM_PREC_FP64><<<G, T, 0, s>>>(ne, el, e2e, x, w, c, g);
                else k_adj_atomic3<EM_PREC_MIXED><<<G, T, 0, s>>>(ne, el, e2e, x, w, c, g);
            } else {
                if (fp64) k_adj_atomic2<EM_PREC_FP64><<<G, T, 0, s>>>(ne, el, e2e, x, w, c, g);
                else k_adj_atomic2<EM_PREC_MIXED><<<G, T, 0, s>>>(ne, el, e2e, x, w, c, g);
            }
            note_launches(1);
            if (m->n_bfaces) {
                if (dim == 3)
                    k_bnd_adj_atomic<3><<<grid_for(m->n_bfaces, T), T, 0, s>>>(m->n_bfaces, m->bface, m->bface_owner,
                                                                              m->elem2edge, x, w, g, e0, e1);
                else
                    k_bnd_adj_atomic<2><<<grid_for(m->n_bfaces, T), T, 0, s>>>(m->n_bfaces, m->bface, m->bface_owner,
                                                                              m->elem2edge, x, w, g, e0, e1);
                note_launches(1);
            }
        }
    }
    EM_CUDA_TRY(cudaGetLastError());
    return EM_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free form of the compensated-FP32 forward: the (hi, lo)
// accumulators live in this file-scope device array instead of a caller
// workspace.  Host code must not pass the symbol itself to a kernel (on the
// host it names a stand-in object, not device memory): it looks up the
// device address once per device with cudaGetSymbolAddress and passes that.
// ---------------------------------------------------------------------------
static __device__ __align__(256) float g_noalloc_scratch[EM_NOALLOC_SCRATCH_BYTES / sizeof(float)];

namespace {
std::mutex g_noalloc_mutex;
constexpr int NOALLOC_MAX_DEVICES = 64;
float* g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {};

int noalloc_scratch(float** out) {
    int dev = 0;
    EM_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return fail(EM_ERR_ARG, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return fail(EM_ERR_CUDA, std::string("cudaGetSymbolAddress(scratch) failed: ") + cudaGetErrorString(e));
        g_noalloc_ptr[dev] = static_cast<float*>(p);
    }
    *out = g_noalloc_ptr[dev];
    return EM_OK;
}
}  // namespace

int atomic_fwd_noalloc(const em_mesh* m, const double* x, double* n, double* vol, double* bnormal, cudaStream_t s) {
    const int dim = m->dim;
    const size_t ne_f = size_t(m->n_edges) * dim, nv_f = size_t(m->n_nodes);
    const size_t need = (2 * ne_f + 2 * nv_f) * sizeof(float);
    if (need > EM_NOALLOC_SCRATCH_BYTES)
        return fail(EM_ERR_ARG, "grid needs " + std::to_string(need) + " bytes of scratch; the allocation-free forward "
                                "holds " + std::to_string((unsigned long long)EM_NOALLOC_SCRATCH_BYTES) +
                                " (use em_edge_metrics with a workspace)");
    float* base = nullptr;
    EM_TRY(noalloc_scratch(&base));
    float* nhi = base;
    float* nlo = nhi + ne_f;
    float* vhi = nlo + ne_f;
    float* vlo = vhi + nv_f;
    EM_CUDA_TRY(cudaMemsetAsync(base, 0, need, s));
    EM_CUDA_TRY(cudaMemsetAsync(bnormal, 0, sizeof(double) * m->n_bnodes * dim, s));
    const int T = 256;
    const unsigned G = grid_for(m->n_elems, T, int64_t(num_sms()) * 16);
    if (dim == 3)
        k_fwd_atomic3<EM_PREC_MIXED_COMP32><<<G, T, 0, s>>>(m->n_elems, m->elems, m->elem2edge, x, n, nullptr, nhi, nlo,
                                                            vhi, vlo);
    else
        k_fwd_atomic2<EM_PREC_MIXED_COMP32><<<G, T, 0, s>>>(m->n_elems, m->elems, m->elem2edge, x, n, nullptr, nhi, nlo,
                                                            vhi, vlo);
    k_comp_finalize<<<grid_for(int64_t(ne_f), T), T, 0, s>>>(int64_t(ne_f), nhi, nlo, n);
    k_comp_finalize<<<grid_for(int64_t(nv_f), T), T, 0, s>>>(int64_t(nv_f), vhi, vlo, vol);
    note_launches(3);
    if (m->n_bfaces) {
        if (dim == 3)
            k_bnd_atomic<3><<<grid_for(m->n_bfaces, T), T, 0, s>>>(m->n_bfaces, m->bface, m->bface_owner, m->elems,
                                                                  m->elem2edge, x, m->n_bnodes, m->bnode, n, bnormal, 0,
                                                                  INT64_MAX);
        else
            k_bnd_atomic<2><<<grid_for(m->n_bfaces, T), T, 0, s>>>(m->n_bfaces, m->bface, m->bface_owner, m->elems,
                                                                  m->elem2edge, x, m->n_bnodes, m->bnode, n, bnormal, 0,
                                                                  INT64_MAX);
        note_launches(1);
    }
    EM_CUDA_TRY(cudaGetLastError());
    return EM_OK;
}

}  // namespace em

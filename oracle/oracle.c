/*
 * CPU oracle for the edge-based grid metrics of
 *   H. Nishikawa, "An Efficient Implementation of Edge-Based Discretization
 *   without Forming Dual Control Volumes" (arXiv 2502.00778).
 *
 * TEST INFRASTRUCTURE ONLY.  Plain, serial, double precision C written from
 * the paper.  Only the test-suite, the smoke check and the benchmark's CPU
 * baseline / reference arm may load this library; the GPU product path never
 * does and shares no code with it.
 *
 * What is here (all loops follow the paper's order):
 *   or_edges            edge list, j<k orientation (Sec. 2), element->edge map
 *   or_bfaces           boundary faces = faces with one incident element,
 *                       oriented outward (the paper takes this list as given)
 *   or_bnodes           nodes on boundary faces
 *   or_direct           proposed algorithm: Eq. efficient_njk_formula_general_D,
 *                       tri: Eqs. njk_eff_algorithm_tria_01/02 + boundary
 *                       Eq. njk_eff_algorithm_tria_02p5_nB; tet: Eqs.
 *                       add_contribution_to_njk_tetra/_nkj_tetra, boundary
 *                       Eq. njk_boundary_correction_3d, scaling Eq.
 *                       apply_1over12_at_the_end_njk_tetra; element-based
 *                       dual volume (Sec. 4.2); boundary dual-face normals
 *                       (1/D) n_B (Sec. 3.2.3)
 *   or_traditional      dual-face construction (Sec. 3.1.1 / 3.1.2)
 *   or_edge_volume      edge-based dual volume (Sec. 4.1)
 *   or_closure          sum of directed areas per node (Sec. 3.2.3)
 *   or_edge_residual    edge-loop residual of the edge-based discretization
 *                       (Sec. 2): central flux 1/2 (F_j + F_k).n_jk out of
 *                       j and into k, plus F_j.bnormal_j at boundary nodes
 *   or_adjoint          analytic gradient of L = sum_e w_e.n_e + sum_i c_i V_i
 *                       (+ sum_b bw_b.bnormal_b when boundary weights are given)
 *   or_loss_subset      L restricted to chosen elements / boundary faces
 *   or_fd_gradient      patch-local central differences of L
 *
 * Readings of the paper used here (the paper's figures are not available):
 *   - n_j^E is the OUTWARD area vector of the face opposite node j, i.e. it
 *     points away from j; its sign is fixed by requiring
 *     n_j^E . (x_k - x_j) > 0 for any other node k of E.
 *   - n_B includes its factor 1/2 in 3D (Eq. tetra_tria_boundary_nB) and is
 *     added to the 2 n_j accumulators before the 1/12 scaling, giving the
 *     general-D correction n_B / (D(D+1)).  In 2D n_B is the full edge normal.
 *   - Traditional dual faces are built in element-local coordinates (the
 *     element's first stored node subtracted) to avoid cancellation when the
 *     grid is offset far from the origin.
 *   - Boundary faces are the faces seen by exactly one element.  A face's
 *     stored node order makes n_B outward; in 3D the first stored node is the
 *     smallest id, in 2D the order (a,b) with n_B = (y_a - y_b, x_b - x_a).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define OR_VERSION 1

int or_version(void) { return OR_VERSION; }

/* local edge numbering over the element's stored node order */
static const int LE3[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
static const int LE2[3][2] = {{0, 1}, {0, 2}, {1, 2}};

static int nloc_edges(int dim) { return dim == 3 ? 6 : 3; }
static const int (*local_edges(int dim))[2] { return dim == 3 ? LE3 : LE2; }

/* ------------------------------------------------------------------------ */
/* small vector helpers                                                      */
/* ------------------------------------------------------------------------ */
static void sub3(const double* a, const double* b, double* r) { r[0] = a[0] - b[0]; r[1] = a[1] - b[1]; r[2] = a[2] - b[2]; }
static void cross3(const double* a, const double* b, double* r) {
    r[0] = a[1] * b[2] - a[2] * b[1];
    r[1] = a[2] * b[0] - a[0] * b[2];
    r[2] = a[0] * b[1] - a[1] * b[0];
}
static double dot(const double* a, const double* b, int d) { double s = 0; for (int i = 0; i < d; i++) s += a[i] * b[i]; return s; }

/* ------------------------------------------------------------------------ */
/* edges                                                                     */
/* ------------------------------------------------------------------------ */
typedef struct { uint64_t key; int64_t slot; } keyslot;

static int cmp_keyslot(const void* pa, const void* pb) {
    const keyslot* a = (const keyslot*)pa; const keyslot* b = (const keyslot*)pb;
    if (a->key < b->key) return -1;
    if (a->key > b->key) return 1;
    return (a->slot < b->slot) ? -1 : (a->slot > b->slot);
}

/* All edges of all elements as (min,max) pairs, sorted and de-duplicated:
 * edges[e] = {j, k} with j < k in lexicographic order; elem2edge[E*nl + l]
 * is the edge of local edge l.  Returns the number of edges, or -1 if
 * `cap` is too small. */
int64_t or_edges(int dim, int64_t ne, const int32_t* elems, int64_t cap, int32_t* edges, int32_t* elem2edge) {
    const int nl = nloc_edges(dim);
    const int (*le)[2] = local_edges(dim);
    int64_t ns = ne * nl;
    keyslot* ks = (keyslot*)malloc(sizeof(keyslot) * (size_t)(ns > 0 ? ns : 1));
    for (int64_t E = 0; E < ne; E++)
        for (int l = 0; l < nl; l++) {
            uint32_t p = (uint32_t)elems[E * 4 + le[l][0]], q = (uint32_t)elems[E * 4 + le[l][1]];
            uint32_t j = p < q ? p : q, k = p < q ? q : p;
            ks[E * nl + l].key = ((uint64_t)j << 32) | k;
            ks[E * nl + l].slot = E * nl + l;
        }
    qsort(ks, (size_t)ns, sizeof(keyslot), cmp_keyslot);
    int64_t m = -1;
    for (int64_t i = 0; i < ns; i++) {
        if (i == 0 || ks[i].key != ks[i - 1].key) {
            m++;
            if (m >= cap) { free(ks); return -1; }
            edges[2 * m] = (int32_t)(ks[i].key >> 32);
            edges[2 * m + 1] = (int32_t)(ks[i].key & 0xffffffffu);
        }
        elem2edge[ks[i].slot] = (int32_t)m;
    }
    free(ks);
    return m + 1;
}

/* id of edge {p,q} in the sorted edge list (binary search), -1 if absent */
static int64_t find_edge(int64_t nedges, const int32_t* edges, int32_t p, int32_t q) {
    int32_t j = p < q ? p : q, k = p < q ? q : p;
    int64_t lo = 0, hi = nedges - 1;
    while (lo <= hi) {
        int64_t mid = (lo + hi) / 2;
        int32_t a = edges[2 * mid], b = edges[2 * mid + 1];
        if (a == j && b == k) return mid;
        if (a < j || (a == j && b < k)) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

/* ------------------------------------------------------------------------ */
/* boundary faces                                                            */
/* ------------------------------------------------------------------------ */
typedef struct { int32_t v[3]; int64_t owner; } facerec;

static int cmp_face(const void* pa, const void* pb) {
    const facerec* a = (const facerec*)pa; const facerec* b = (const facerec*)pb;
    for (int i = 0; i < 3; i++) { if (a->v[i] < b->v[i]) return -1; if (a->v[i] > b->v[i]) return 1; }
    return (a->owner < b->owner) ? -1 : (a->owner > b->owner);
}

static void isort(int32_t* v, int n) {
    for (int i = 1; i < n; i++) { int32_t t = v[i]; int j = i - 1; while (j >= 0 && v[j] > t) { v[j + 1] = v[j]; j--; } v[j + 1] = t; }
}

/* outward area vector of a stored boundary face (Eq. tetra_tria_boundary_nB in
 * 3D, with its 1/2; the full edge normal (y_a - y_b, x_b - x_a) in 2D) */
static void face_area_vector(int dim, const double* x, const int32_t* f, double* nB) {
    if (dim == 3) {
        double u[3], t[3];
        sub3(x + 3 * f[1], x + 3 * f[0], u);
        sub3(x + 3 * f[2], x + 3 * f[0], t);
        cross3(u, t, nB);
        nB[0] *= 0.5; nB[1] *= 0.5; nB[2] *= 0.5;
    } else {
        const double* a = x + 2 * f[0]; const double* b = x + 2 * f[1];
        nB[0] = a[1] - b[1];
        nB[1] = b[0] - a[0];
    }
}

/* Faces seen by exactly one element, sorted by their sorted node ids.
 * bface[B*dim ...] holds the nodes in outward order; bowner[B] = elem*4 + the
 * local index of the owner's node opposite the face.  Returns the count, or
 * -1 if `cap` is too small. */
int64_t or_bfaces(int dim, int64_t ne, const int32_t* elems, const double* x, int64_t cap, int32_t* bface, int32_t* bowner) {
    const int nv = dim + 1;
    int64_t nf = ne * nv;
    facerec* fr = (facerec*)malloc(sizeof(facerec) * (size_t)(nf > 0 ? nf : 1));
    for (int64_t E = 0; E < ne; E++)
        for (int o = 0; o < nv; o++) {
            facerec* r = &fr[E * nv + o];
            int c = 0;
            for (int i = 0; i < nv; i++) if (i != o) r->v[c++] = elems[E * 4 + i];
            if (dim == 2) r->v[2] = -1;
            isort(r->v, dim);
            r->owner = E * 4 + o;
        }
    qsort(fr, (size_t)nf, sizeof(facerec), cmp_face);
    int64_t nb = 0;
    for (int64_t i = 0; i < nf;) {
        int64_t j = i + 1;
        while (j < nf && memcmp(fr[j].v, fr[i].v, sizeof(int32_t) * 3) == 0) j++;
        if (j - i == 1) {
            if (nb >= cap) { free(fr); return -1; }
            int64_t E = fr[i].owner / 4; int o = (int)(fr[i].owner % 4);
            int32_t f[3] = {fr[i].v[0], fr[i].v[1], fr[i].v[2]};
            const double* xo = x + dim * elems[E * 4 + o];
            double nB[3] = {0, 0, 0}, d[3] = {0, 0, 0};
            face_area_vector(dim, x, f, nB);
            for (int c = 0; c < dim; c++) d[c] = xo[c] - x[dim * f[0] + c];
            if (dot(nB, d, dim) > 0) {          /* points towards the element: flip */
                if (dim == 3) { int32_t t = f[1]; f[1] = f[2]; f[2] = t; }
                else { int32_t t = f[0]; f[0] = f[1]; f[1] = t; }
            }
            for (int c = 0; c < dim; c++) bface[nb * dim + c] = f[c];
            bowner[nb] = (int32_t)fr[i].owner;
            nb++;
        }
        i = j;
    }
    free(fr);
    return nb;
}

/* sorted list of nodes touched by boundary faces; returns count */
int64_t or_bnodes(int dim, int64_t nv, int64_t nb, const int32_t* bface, int32_t* bnode) {
    char* mark = (char*)calloc((size_t)(nv > 0 ? nv : 1), 1);
    for (int64_t i = 0; i < nb * dim; i++) mark[bface[i]] = 1;
    int64_t m = 0;
    for (int64_t v = 0; v < nv; v++) if (mark[v]) bnode[m++] = (int32_t)v;
    free(mark);
    return m;
}

/* ------------------------------------------------------------------------ */
/* element geometry                                                          */
/* ------------------------------------------------------------------------ */

/* outward area vector of the face of element E opposite its local node o:
 *   3D: (1/2) (x_l - x_k) x (x_r - x_k) over the other three nodes k,l,r;
 *   2D: the edge {k,r} rotated by 90 degrees (length = edge length);
 * the sign is chosen so that it points away from node o. */
static void face_opposite(int dim, const double* x, const int32_t* el, int o, double* n) {
    int oth[3], c = 0;
    for (int i = 0; i < dim + 1; i++) if (i != o) oth[c++] = i;
    const double* xo = x + dim * el[o];
    const double* xk = x + dim * el[oth[0]];
    double d[3] = {0, 0, 0};
    for (int i = 0; i < dim; i++) d[i] = xk[i] - xo[i];
    if (dim == 3) {
        double u[3], t[3];
        sub3(x + 3 * el[oth[1]], xk, u);
        sub3(x + 3 * el[oth[2]], xk, t);
        cross3(u, t, n);
        n[0] *= 0.5; n[1] *= 0.5; n[2] *= 0.5;
    } else {
        const double* xr = x + 2 * el[oth[1]];
        n[0] = xr[1] - xk[1];
        n[1] = xk[0] - xr[0];
    }
    if (dot(n, d, dim) < 0) for (int i = 0; i < dim; i++) n[i] = -n[i];
}

/* element volume (area in 2D), unsigned */
static double elem_volume(int dim, const double* x, const int32_t* el) {
    if (dim == 3) {
        double a[3], b[3], c[3], bc[3];
        sub3(x + 3 * el[1], x + 3 * el[0], a);
        sub3(x + 3 * el[2], x + 3 * el[0], b);
        sub3(x + 3 * el[3], x + 3 * el[0], c);
        cross3(b, c, bc);
        return fabs(dot(a, bc, 3)) / 6.0;
    }
    const double* p0 = x + 2 * el[0]; const double* p1 = x + 2 * el[1]; const double* p2 = x + 2 * el[2];
    double ax = p1[0] - p0[0], ay = p1[1] - p0[1], bx = p2[0] - p0[0], by = p2[1] - p0[1];
    return fabs(ax * by - ay * bx) / 2.0;
}

/* local index (within the element) of the lower-id end of local edge l */
static int low_end(const int32_t* el, const int* le) { return el[le[0]] < el[le[1]] ? le[0] : le[1]; }

/* ------------------------------------------------------------------------ */
/* proposed (direct) algorithm                                              */
/* ------------------------------------------------------------------------ */

/* n_edge[nedges*dim], vol[nv], bnormal_full[nv*dim] (zero except at boundary
 * nodes) are overwritten. */
void or_direct(int dim, int64_t nv, const double* x, int64_t ne, const int32_t* elems, const int32_t* elem2edge,
               int64_t nedges, const int32_t* edges, int64_t nb, const int32_t* bface,
               double* n_edge, double* vol, double* bnormal_full) {
    const int nl = nloc_edges(dim);
    const int (*le)[2] = local_edges(dim);
    memset(n_edge, 0, sizeof(double) * (size_t)(nedges * dim));
    memset(vol, 0, sizeof(double) * (size_t)nv);
    memset(bnormal_full, 0, sizeof(double) * (size_t)(nv * dim));

    /* element loop: add the (scaled) area vector of the face opposite the
     * lower-numbered end j of every edge {j,k} */
    for (int64_t E = 0; E < ne; E++) {
        const int32_t* el = elems + 4 * E;
        for (int l = 0; l < nl; l++) {
            double nj[3] = {0, 0, 0};
            face_opposite(dim, x, el, low_end(el, le[l]), nj);
            double* ne_ = n_edge + dim * (int64_t)elem2edge[E * nl + l];
            if (dim == 3) {                 /* accumulate 2 n_j^E, scale by 1/12 later */
                for (int c = 0; c < 3; c++) ne_[c] += 2.0 * nj[c];
            } else {                        /* add n_j^E / 3 directly */
                for (int c = 0; c < 2; c++) ne_[c] += nj[c] / 3.0;
            }
        }
    }
    /* boundary loop: correction on every edge of every boundary face, and the
     * boundary dual-face normal (1/D) n_B at its nodes */
    for (int64_t B = 0; B < nb; B++) {
        const int32_t* f = bface + dim * B;
        double nB[3] = {0, 0, 0};
        face_area_vector(dim, x, f, nB);
        if (dim == 3) {
            for (int a = 0; a < 3; a++) {
                int64_t e = find_edge(nedges, edges, f[a], f[(a + 1) % 3]);
                for (int c = 0; c < 3; c++) n_edge[3 * e + c] += nB[c];
            }
        } else {
            int64_t e = find_edge(nedges, edges, f[0], f[1]);
            for (int c = 0; c < 2; c++) n_edge[2 * e + c] += nB[c] / 6.0;
        }
        for (int a = 0; a < dim; a++)
            for (int c = 0; c < dim; c++) bnormal_full[dim * (int64_t)f[a] + c] += nB[c] / (double)dim;
    }
    /* 3D: edge loop applying 1/12 */
    if (dim == 3)
        for (int64_t e = 0; e < nedges * 3; e++) n_edge[e] *= (1.0 / 12.0);

    /* element-based dual volume: V_E / (D+1) to each node of E */
    for (int64_t E = 0; E < ne; E++) {
        const int32_t* el = elems + 4 * E;
        double vE = elem_volume(dim, x, el);
        for (int i = 0; i < dim + 1; i++) vol[el[i]] += vE / (double)(dim + 1);
    }
}

/* ------------------------------------------------------------------------ */
/* traditional algorithm (dual faces)                                        */
/* ------------------------------------------------------------------------ */
void or_traditional(int dim, int64_t nv, const double* x, int64_t ne, const int32_t* elems, const int32_t* elem2edge,
                    int64_t nedges, double* n_edge) {
    (void)nv;
    const int nl = nloc_edges(dim);
    const int (*le)[2] = local_edges(dim);
    memset(n_edge, 0, sizeof(double) * (size_t)(nedges * dim));
    for (int64_t E = 0; E < ne; E++) {
        const int32_t* el = elems + 4 * E;
        /* element-local coordinates */
        double p[4][3] = {{0}};
        for (int i = 0; i < dim + 1; i++)
            for (int c = 0; c < dim; c++) p[i][c] = x[dim * el[i] + c] - x[dim * el[0] + c];
        for (int l = 0; l < nl; l++) {
            int jl = low_end(el, le[l]);
            int kl = (jl == le[l][0]) ? le[l][1] : le[l][0];
            double* ne_ = n_edge + dim * (int64_t)elem2edge[E * nl + l];
            double djk[3] = {0, 0, 0};
            for (int c = 0; c < dim; c++) djk[c] = p[kl][c] - p[jl][c];
            if (dim == 2) {
                int rl = 3 - jl - kl;
                double xm = (p[jl][0] + p[kl][0]) / 2, ym = (p[jl][1] + p[kl][1]) / 2;
                double xE = (p[jl][0] + p[kl][0] + p[rl][0]) / 3, yE = (p[jl][1] + p[kl][1] + p[rl][1]) / 3;
                double n[2] = {ym - yE, xE - xm};
                if (dot(n, djk, 2) < 0) { n[0] = -n[0]; n[1] = -n[1]; }
                ne_[0] += n[0]; ne_[1] += n[1];
            } else {
                int o[2], c2 = 0;
                for (int i = 0; i < 4; i++) if (i != jl && i != kl) o[c2++] = i;
                int ll = o[0], rl = o[1];
                double xm[3], xE[3], xL[3], xR[3];
                for (int c = 0; c < 3; c++) {
                    xm[c] = (p[jl][c] + p[kl][c]) / 2;
                    xE[c] = (p[jl][c] + p[kl][c] + p[ll][c] + p[rl][c]) / 4;
                    xL[c] = (p[jl][c] + p[ll][c] + p[kl][c]) / 3;
                    xR[c] = (p[jl][c] + p[rl][c] + p[kl][c]) / 3;
                }
                double Em[3], Lm[3], Rm[3], nEL[3], nER[3];
                sub3(xE, xm, Em); sub3(xL, xm, Lm); sub3(xR, xm, Rm);
                cross3(Em, Lm, nEL);
                cross3(Rm, Em, nER);
                for (int c = 0; c < 3; c++) { nEL[c] *= 0.5; nER[c] *= 0.5; }
                /* each dual triangle is directed from j to k */
                if (dot(nEL, djk, 3) < 0) for (int c = 0; c < 3; c++) nEL[c] = -nEL[c];
                if (dot(nER, djk, 3) < 0) for (int c = 0; c < 3; c++) nER[c] = -nER[c];
                for (int c = 0; c < 3; c++) ne_[c] += nEL[c] + nER[c];
            }
        }
    }
}

/* ------------------------------------------------------------------------ */
/* edge-based dual volume (Sec. 4.1) and closure (Sec. 3.2.3)               */
/* ------------------------------------------------------------------------ */
void or_edge_volume(int dim, int64_t nv, const double* x, int64_t nedges, const int32_t* edges, const double* n_edge, double* vol) {
    memset(vol, 0, sizeof(double) * (size_t)nv);
    for (int64_t e = 0; e < nedges; e++) {
        int32_t j = edges[2 * e], k = edges[2 * e + 1];
        double s = 0;
        for (int c = 0; c < dim; c++) s += (x[dim * k + c] - x[dim * j + c]) * n_edge[dim * e + c];
        vol[j] += s;
        vol[k] += s;
    }
    for (int64_t v = 0; v < nv; v++) vol[v] *= 1.0 / (2.0 * dim);
}

/* Edge-loop residual (Sec. 2): every edge {j,k} carries the central flux
 * phi = sum_c 1/2 (F_j[c] + F_k[c]) n_jk[c] out of node j's dual volume and
 * into node k's; a boundary node adds F_j . bnormal_j.  For a linear F the
 * sum equals V_j div F at interior nodes (closure plus the linear exactness
 * of the lumped areas); boundary nodes need a boundary quadrature that this
 * simple closure does not provide. */
void or_edge_residual(int dim, int64_t nv, int64_t nedges, const int32_t* edges, const double* n_edge, const double* F,
                      int64_t nbn, const int32_t* bnode, const double* bnormal, double* res) {
    memset(res, 0, sizeof(double) * (size_t)nv);
    for (int64_t e = 0; e < nedges; e++) {
        int32_t j = edges[2 * e], k = edges[2 * e + 1];
        double phi = 0;
        for (int c = 0; c < dim; c++) phi += 0.5 * (F[dim * j + c] + F[dim * k + c]) * n_edge[dim * e + c];
        res[j] += phi;
        res[k] -= phi;
    }
    for (int64_t b = 0; b < nbn; b++) {
        int32_t j = bnode[b];
        double s = 0;
        for (int c = 0; c < dim; c++) s += F[dim * j + c] * bnormal[dim * b + c];
        res[j] += s;
    }
}

void or_closure(int dim, int64_t nv, const double* x, int64_t nedges, const int32_t* edges, const double* n_edge,
                int64_t nb, const int32_t* bface, double* a) {
    memset(a, 0, sizeof(double) * (size_t)(nv * dim));
    for (int64_t e = 0; e < nedges; e++) {
        int32_t j = edges[2 * e], k = edges[2 * e + 1];
        for (int c = 0; c < dim; c++) { a[dim * j + c] += n_edge[dim * e + c]; a[dim * k + c] -= n_edge[dim * e + c]; }
    }
    for (int64_t B = 0; B < nb; B++) {
        const int32_t* f = bface + dim * B;
        double nB[3] = {0, 0, 0};
        face_area_vector(dim, x, f, nB);
        for (int i = 0; i < dim; i++)
            for (int c = 0; c < dim; c++) a[dim * f[i] + c] += nB[c] / (double)dim;
    }
}

/* ------------------------------------------------------------------------ */
/* loss L = sum_e w_e . n_e + sum_i c_i V_i and its gradient                */
/* ------------------------------------------------------------------------ */

/* d/dx of w.(alpha * n) where n is the outward area vector of the face of E
 * opposite local node o (built exactly as in face_opposite), added to g */
static void face_opposite_grad(int dim, const double* x, const int32_t* el, int o, const double* w, double alpha, double* g) {
    int oth[3], c = 0;
    for (int i = 0; i < dim + 1; i++) if (i != o) oth[c++] = i;
    double n[3] = {0, 0, 0};
    face_opposite(dim, x, el, o, n);
    /* recover the orientation sign s used by face_opposite */
    const double* xk = x + dim * el[oth[0]];
    double s;
    if (dim == 3) {
        double u[3], t[3], cr[3], gu[3], gt[3];
        sub3(x + 3 * el[oth[1]], xk, u);
        sub3(x + 3 * el[oth[2]], xk, t);
        cross3(u, t, cr);
        s = (dot(cr, n, 3) >= 0) ? 1.0 : -1.0;
        /* w.(u x t) = u.(t x w) = t.(w x u) */
        cross3(t, w, gu);
        cross3(w, u, gt);
        for (int i = 0; i < 3; i++) {
            double fu = alpha * s * 0.5 * gu[i], ft = alpha * s * 0.5 * gt[i];
            g[3 * el[oth[1]] + i] += fu;
            g[3 * el[oth[2]] + i] += ft;
            g[3 * el[oth[0]] + i] -= fu + ft;
        }
    } else {
        const double* xr = x + 2 * el[oth[1]];
        double base[2] = {xr[1] - xk[1], xk[0] - xr[0]};
        s = (base[0] * n[0] + base[1] * n[1] >= 0) ? 1.0 : -1.0;
        /* n = s (dy, -dx) with d = x_r - x_k: d/dd of w.n = s (-w_y, w_x) */
        double gd[2] = {-s * w[1] * alpha, s * w[0] * alpha};
        for (int i = 0; i < 2; i++) { g[2 * el[oth[1]] + i] += gd[i]; g[2 * el[oth[0]] + i] -= gd[i]; }
    }
}

/* d/dx of w . (alpha n_B) for a stored (outward) boundary face, added to g */
static void bface_grad(int dim, const double* x, const int32_t* f, const double* w, double alpha, double* g) {
    if (dim == 3) {
        double u[3], t[3], gu[3], gt[3];
        sub3(x + 3 * f[1], x + 3 * f[0], u);
        sub3(x + 3 * f[2], x + 3 * f[0], t);
        cross3(t, w, gu);
        cross3(w, u, gt);
        for (int i = 0; i < 3; i++) {
            double fu = alpha * 0.5 * gu[i], ft = alpha * 0.5 * gt[i];
            g[3 * f[1] + i] += fu;
            g[3 * f[2] + i] += ft;
            g[3 * f[0] + i] -= fu + ft;
        }
    } else {
        /* n_B = (-d_y, d_x) with d = x_b - x_a */
        double gd[2] = {w[1] * alpha, -w[0] * alpha};
        for (int i = 0; i < 2; i++) { g[2 * f[1] + i] += gd[i]; g[2 * f[0] + i] -= gd[i]; }
    }
}

static void elem_grad(int dim, const double* x, const int32_t* el, const int32_t* e2e_row, const double* w, const double* c, double* g) {
    const int nl = nloc_edges(dim);
    const int (*le)[2] = local_edges(dim);
    const double alpha = 2.0 / (dim * (dim + 1.0));
    for (int l = 0; l < nl; l++)
        face_opposite_grad(dim, x, el, low_end(el, le[l]), w + dim * (int64_t)e2e_row[l], alpha, g);
    /* dV_E/dx_i = -n_i^E / D */
    double csum = 0;
    for (int i = 0; i < dim + 1; i++) csum += c[el[i]];
    for (int i = 0; i < dim + 1; i++) {
        double ni[3] = {0, 0, 0};
        face_opposite(dim, x, el, i, ni);
        for (int q = 0; q < dim; q++) g[dim * el[i] + q] += csum / (dim + 1.0) * (-ni[q] / dim);
    }
}

static void bface_edge_weight(int dim, int64_t nedges, const int32_t* edges, const int32_t* f, const double* w, double* wB) {
    wB[0] = wB[1] = wB[2] = 0;
    int ned = dim == 3 ? 3 : 1;
    for (int a = 0; a < ned; a++) {
        int64_t e = find_edge(nedges, edges, f[a], f[(a + 1) % dim]);
        for (int q = 0; q < dim; q++) wB[q] += w[dim * e + q];
    }
}

/* g[nv*dim] overwritten with dL/dx */
/* K_B = w_B / (D(D+1)) + (1/D) sum_{b in B} bw_b: the vector that multiplies a
 * boundary face's n_B in L (its edges' n_jk corrections and, with boundary-
 * normal weights bw given per node, the 1/D n_B of its nodes' bnormal) */
static void bface_coeff(int dim, int64_t nedges, const int32_t* edges, const int32_t* f, const double* w,
                        const double* bw_node, double* K) {
    double wB[3];
    bface_edge_weight(dim, nedges, edges, f, w, wB);
    for (int q = 0; q < dim; q++) {
        double bs = 0;
        for (int a = 0; a < dim; a++) bs += bw_node[dim * (int64_t)f[a] + q];
        K[q] = wB[q] / (dim * (dim + 1.0)) + bs / dim;
    }
}

void or_adjoint(int dim, int64_t nv, const double* x, int64_t ne, const int32_t* elems, const int32_t* elem2edge,
                int64_t nedges, const int32_t* edges, int64_t nb, const int32_t* bface,
                const double* w, const double* c, const double* bw_node, double* g) {
    const int nl = nloc_edges(dim);
    memset(g, 0, sizeof(double) * (size_t)(nv * dim));
    for (int64_t E = 0; E < ne; E++) elem_grad(dim, x, elems + 4 * E, elem2edge + nl * E, w, c, g);
    const double beta = 1.0 / (dim * (dim + 1.0));
    for (int64_t B = 0; B < nb; B++) {
        if (bw_node) {
            double K[3];
            bface_coeff(dim, nedges, edges, bface + dim * B, w, bw_node, K);
            bface_grad(dim, x, bface + dim * B, K, 1.0, g);
        } else {
            double wB[3];
            bface_edge_weight(dim, nedges, edges, bface + dim * B, w, wB);
            bface_grad(dim, x, bface + dim * B, wB, beta, g);
        }
    }
}

/* L restricted to a subset of elements and boundary faces (same formulas as
 * or_direct, contribution by contribution) */
double or_loss_subset(int dim, const double* x, const int32_t* elems, const int32_t* elem2edge,
                      int64_t nsel, const int64_t* sel, int64_t nedges, const int32_t* edges, const int32_t* bface,
                      int64_t nbsel, const int64_t* bsel, const double* w, const double* c, const double* bw_node) {
    const int nl = nloc_edges(dim);
    const int (*le)[2] = local_edges(dim);
    const double alpha = 2.0 / (dim * (dim + 1.0));
    double L = 0;
    for (int64_t s = 0; s < nsel; s++) {
        int64_t E = sel[s];
        const int32_t* el = elems + 4 * E;
        for (int l = 0; l < nl; l++) {
            double nj[3] = {0, 0, 0};
            face_opposite(dim, x, el, low_end(el, le[l]), nj);
            L += alpha * dot(w + dim * (int64_t)elem2edge[nl * E + l], nj, dim);
        }
        double vE = elem_volume(dim, x, el);
        for (int i = 0; i < dim + 1; i++) L += c[el[i]] * vE / (dim + 1.0);
    }
    const double beta = 1.0 / (dim * (dim + 1.0));
    for (int64_t s = 0; s < nbsel; s++) {
        const int32_t* f = bface + dim * bsel[s];
        double nB[3] = {0, 0, 0}, wB[3];
        face_area_vector(dim, x, f, nB);
        if (bw_node) {
            bface_coeff(dim, nedges, edges, f, w, bw_node, wB);
            L += dot(wB, nB, dim);
        } else {
            bface_edge_weight(dim, nedges, edges, f, w, wB);
            L += beta * dot(wB, nB, dim);
        }
    }
    return L;
}

/* Patch-local central differences of L at the listed nodes: only elements
 * and boundary faces containing the node are summed.  x is perturbed in
 * place and restored.  g_fd[nn*dim] overwritten. */
void or_fd_gradient(int dim, int64_t nv, double* x, int64_t ne, const int32_t* elems, const int32_t* elem2edge,
                    int64_t nedges, const int32_t* edges, int64_t nb, const int32_t* bface,
                    const double* w, const double* c, const double* bw_node, int64_t nn, const int64_t* nodes,
                    double delta, double* g_fd) {
    int64_t* pos = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nv > 0 ? nv : 1));
    for (int64_t v = 0; v < nv; v++) pos[v] = -1;
    for (int64_t i = 0; i < nn; i++) pos[nodes[i]] = i;
    int64_t* ecnt = (int64_t*)calloc((size_t)nn + 1, sizeof(int64_t));
    int64_t* bcnt = (int64_t*)calloc((size_t)nn + 1, sizeof(int64_t));
    for (int64_t E = 0; E < ne; E++) for (int i = 0; i < dim + 1; i++) { int64_t p = pos[elems[4 * E + i]]; if (p >= 0) ecnt[p + 1]++; }
    for (int64_t B = 0; B < nb; B++) for (int i = 0; i < dim; i++) { int64_t p = pos[bface[dim * B + i]]; if (p >= 0) bcnt[p + 1]++; }
    for (int64_t i = 0; i < nn; i++) { ecnt[i + 1] += ecnt[i]; bcnt[i + 1] += bcnt[i]; }
    int64_t* elist = (int64_t*)malloc(sizeof(int64_t) * (size_t)(ecnt[nn] + 1));
    int64_t* blist = (int64_t*)malloc(sizeof(int64_t) * (size_t)(bcnt[nn] + 1));
    int64_t* efill = (int64_t*)calloc((size_t)nn + 1, sizeof(int64_t));
    int64_t* bfill = (int64_t*)calloc((size_t)nn + 1, sizeof(int64_t));
    for (int64_t E = 0; E < ne; E++) for (int i = 0; i < dim + 1; i++) { int64_t p = pos[elems[4 * E + i]]; if (p >= 0) elist[ecnt[p] + efill[p]++] = E; }
    for (int64_t B = 0; B < nb; B++) for (int i = 0; i < dim; i++) { int64_t p = pos[bface[dim * B + i]]; if (p >= 0) blist[bcnt[p] + bfill[p]++] = B; }
    for (int64_t i = 0; i < nn; i++) {
        int64_t v = nodes[i];
        for (int q = 0; q < dim; q++) {
            double x0 = x[dim * v + q];
            x[dim * v + q] = x0 + delta;
            double Lp = or_loss_subset(dim, x, elems, elem2edge, ecnt[i + 1] - ecnt[i], elist + ecnt[i], nedges, edges, bface,
                                       bcnt[i + 1] - bcnt[i], blist + bcnt[i], w, c, bw_node);
            x[dim * v + q] = x0 - delta;
            double Lm = or_loss_subset(dim, x, elems, elem2edge, ecnt[i + 1] - ecnt[i], elist + ecnt[i], nedges, edges, bface,
                                       bcnt[i + 1] - bcnt[i], blist + bcnt[i], w, c, bw_node);
            x[dim * v + q] = x0;
            g_fd[dim * i + q] = (Lp - Lm) / (2.0 * delta);
        }
    }
    free(pos); free(ecnt); free(bcnt); free(elist); free(blist); free(efill); free(bfill);
}

/* ------------------------------------------------------------------------ */
/* sampled evaluation (one output at a time, from the elements around it)  */
/* ------------------------------------------------------------------------ */

/* SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
 * generators", OOPSLA 2014): the counter-based generator used to define the
 * loss weights of the sampled checks, w(j,k) and c(v), as a function of the
 * edge's end nodes / the node id, so no edge numbering is needed. */
static uint64_t splitmix64(uint64_t z) {
    z += 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}
/* uniform in [-1, 1): 53 random bits */
static double u11(uint64_t z) { return (double)(splitmix64(z) >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0; }

void or_hash_w(int dim, int32_t j, int32_t k, uint64_t seed, double* w) {
    uint64_t key = ((uint64_t)(uint32_t)j << 32) | (uint32_t)k;
    for (int c = 0; c < dim; c++) w[c] = u11(seed ^ (key * 4u + (uint64_t)c));
}
double or_hash_c(int32_t v, uint64_t seed) { return u11(seed ^ (((uint64_t)(uint32_t)v << 2) | 3u) ^ 0x5bd1e995ULL); }

/* elements containing each marked node: CSR over the marked nodes */
typedef struct { int64_t* ptr; int64_t* list; int64_t* pos; } nodestar;

static nodestar build_stars(int dim, int64_t nv, int64_t ne, const int32_t* elems, int64_t nn, const int32_t* nodes) {
    nodestar s;
    s.pos = (int64_t*)malloc(sizeof(int64_t) * (size_t)nv);
    for (int64_t v = 0; v < nv; v++) s.pos[v] = -1;
    for (int64_t i = 0; i < nn; i++) s.pos[nodes[i]] = i;
    s.ptr = (int64_t*)calloc((size_t)nn + 1, sizeof(int64_t));
    for (int64_t E = 0; E < ne; E++)
        for (int i = 0; i < dim + 1; i++) { int64_t p = s.pos[elems[4 * E + i]]; if (p >= 0) s.ptr[p + 1]++; }
    for (int64_t i = 0; i < nn; i++) s.ptr[i + 1] += s.ptr[i];
    s.list = (int64_t*)malloc(sizeof(int64_t) * (size_t)(s.ptr[nn] + 1));
    int64_t* fill = (int64_t*)calloc((size_t)nn + 1, sizeof(int64_t));
    for (int64_t E = 0; E < ne; E++)
        for (int i = 0; i < dim + 1; i++) { int64_t p = s.pos[elems[4 * E + i]]; if (p >= 0) s.list[s.ptr[p] + fill[p]++] = E; }
    free(fill);
    return s;
}
static void free_stars(nodestar* s) { free(s->ptr); free(s->list); free(s->pos); }

static int elem_has(int dim, const int32_t* el, int32_t v) { for (int i = 0; i < dim + 1; i++) if (el[i] == v) return 1; return 0; }

/* faces of the star of node j that contain j and are seen by exactly one star
 * element: the boundary faces through j.  Calls fn for each, with the face's
 * nodes in outward order (the stored order of the boundary face list). */
static int face_key_eq(const int32_t* a, const int32_t* b, int n) { for (int i = 0; i < n; i++) if (a[i] != b[i]) return 0; return 1; }

static int64_t star_bfaces(int dim, const double* x, const int32_t* elems, const int64_t* star, int64_t ns, int32_t j,
                           int32_t* out /* [cap][dim] outward order */, int64_t cap) {
    int64_t nb = 0;
    for (int64_t a = 0; a < ns; a++) {
        const int32_t* el = elems + 4 * star[a];
        for (int o = 0; o < dim + 1; o++) {
            if (el[o] == j) continue;                 /* faces through j only */
            int32_t f[3] = {0, 0, 0}; int c = 0;
            for (int i = 0; i < dim + 1; i++) if (i != o) f[c++] = el[i];
            isort(f, dim);
            int count = 0;
            for (int64_t b = 0; b < ns; b++) {
                const int32_t* eb = elems + 4 * star[b];
                int all = 1;
                for (int i = 0; i < dim; i++) all &= elem_has(dim, eb, f[i]);
                count += all;
            }
            if (count != 1) continue;
            /* orient outward exactly as or_bfaces does */
            double nB[3] = {0, 0, 0}, d[3] = {0, 0, 0};
            face_area_vector(dim, x, f, nB);
            for (int q = 0; q < dim; q++) d[q] = x[dim * el[o] + q] - x[dim * f[0] + q];
            if (dot(nB, d, dim) > 0) {
                if (dim == 3) { int32_t t = f[1]; f[1] = f[2]; f[2] = t; }
                else { int32_t t = f[0]; f[0] = f[1]; f[1] = t; }
            }
            if (nb < cap) for (int q = 0; q < dim; q++) out[nb * dim + q] = f[q];
            nb++;
        }
    }
    return nb;
}

/* n at sampled edges (sj < sk), V and bnormal at sampled nodes, gradient of
 * L (with w(j,k), c(v) from or_hash_w / or_hash_c) at sampled nodes; every
 * value is computed from the elements around its edge or node with the same
 * formulas as or_direct / or_adjoint. */
void or_sample(int dim, int64_t nv, const double* x, int64_t ne, const int32_t* elems,
               int64_t nse, const int32_t* sj, const int32_t* sk, double* n_out,
               int64_t nsn, const int32_t* sn, double* v_out, double* b_out, uint64_t seed, double* g_out) {
    const int nl = nloc_edges(dim);
    const int (*le)[2] = local_edges(dim);
    int64_t nq = nse + nsn;
    int32_t* nodes = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nq > 0 ? nq : 1));
    for (int64_t i = 0; i < nse; i++) nodes[i] = sj[i];
    for (int64_t i = 0; i < nsn; i++) nodes[nse + i] = sn[i];
    /* de-duplicate the marked set through pos[] (last index wins) */
    nodestar st = build_stars(dim, nv, ne, elems, nq, nodes);
    int32_t fb[64 * 3];
    for (int64_t s = 0; s < nse; s++) {
        int32_t j = sj[s], k = sk[s];
        int64_t p = st.pos[j];
        const int64_t* star = st.list + st.ptr[p];
        int64_t ns = st.ptr[p + 1] - st.ptr[p];
        double acc[3] = {0, 0, 0};
        for (int64_t a = 0; a < ns; a++) {
            const int32_t* el = elems + 4 * star[a];
            if (!elem_has(dim, el, k)) continue;
            for (int l = 0; l < nl; l++) {
                int32_t u = el[le[l][0]], w2 = el[le[l][1]];
                if (!((u == j && w2 == k) || (u == k && w2 == j))) continue;
                double nj[3] = {0, 0, 0};
                face_opposite(dim, x, el, low_end(el, le[l]), nj);
                for (int c = 0; c < dim; c++) acc[c] += (dim == 3) ? 2.0 * nj[c] : nj[c] / 3.0;
            }
        }
        int64_t nb = star_bfaces(dim, x, elems, star, ns, j, fb, 64);
        for (int64_t b = 0; b < nb && b < 64; b++) {
            const int32_t* f = fb + dim * b;
            int hasj = 0, hask = 0;
            for (int q = 0; q < dim; q++) { hasj |= f[q] == j; hask |= f[q] == k; }
            if (!(hasj && hask)) continue;
            double nB[3] = {0, 0, 0};
            face_area_vector(dim, x, f, nB);
            for (int c = 0; c < dim; c++) acc[c] += (dim == 3) ? nB[c] : nB[c] / 6.0;
        }
        for (int c = 0; c < dim; c++) n_out[dim * s + c] = (dim == 3) ? acc[c] * (1.0 / 12.0) : acc[c];
    }
    for (int64_t s = 0; s < nsn; s++) {
        int32_t v = sn[s];
        int64_t p = st.pos[v];
        const int64_t* star = st.list + st.ptr[p];
        int64_t ns = st.ptr[p + 1] - st.ptr[p];
        double vol = 0, bn[3] = {0, 0, 0};
        double* g = g_out + dim * s;
        double gg[3] = {0, 0, 0};
        for (int64_t a = 0; a < ns; a++) {
            const int32_t* el = elems + 4 * star[a];
            vol += elem_volume(dim, x, el) / (double)(dim + 1);
            /* gradient of this element's share of L, read at node v: build a
             * local gradient over the element's nodes with or_adjoint's rules */
            double wl[6][3];
            int32_t e2e_local[6];
            for (int l = 0; l < nl; l++) {
                int32_t a0 = el[le[l][0]], a1 = el[le[l][1]];
                or_hash_w(dim, a0 < a1 ? a0 : a1, a0 < a1 ? a1 : a0, seed, wl[l]);
                e2e_local[l] = l;
            }
            double cl[4];
            for (int i = 0; i < dim + 1; i++) cl[i] = or_hash_c(el[i], seed);
            /* local copies indexed 0..dim with node ids 0..dim */
            double xl[12];
            int32_t ell[4] = {0, 1, 2, dim == 3 ? 3 : -1};
            for (int i = 0; i < dim + 1; i++) for (int q = 0; q < dim; q++) xl[dim * i + q] = x[dim * el[i] + q];
            /* lower-end choice must follow the GLOBAL ids: reorder the local
             * copy so that local order equals global order */
            int ord[4] = {0, 1, 2, 3};
            for (int i2 = 1; i2 < dim + 1; i2++) { int t = ord[i2], q2 = i2 - 1; while (q2 >= 0 && el[ord[q2]] > el[t]) { ord[q2 + 1] = ord[q2]; q2--; } ord[q2 + 1] = t; }
            double xs[12]; double cs[4]; int32_t gid[4];
            for (int i = 0; i < dim + 1; i++) { gid[i] = el[ord[i]]; cs[i] = cl[ord[i]]; for (int q = 0; q < dim; q++) xs[dim * i + q] = xl[dim * ord[i] + q]; }
            double ws[6][3];
            for (int l = 0; l < nl; l++) {
                int32_t a0 = gid[le[l][0]], a1 = gid[le[l][1]];
                or_hash_w(dim, a0 < a1 ? a0 : a1, a0 < a1 ? a1 : a0, seed, ws[l]);
            }
            double glocal[12] = {0};
            double wflat[18];
            for (int l = 0; l < nl; l++) for (int q = 0; q < dim; q++) wflat[dim * l + q] = ws[l][q];
            elem_grad(dim, xs, ell, e2e_local, wflat, cs, glocal);
            int iv = -1;
            for (int i = 0; i < dim + 1; i++) if (gid[i] == v) iv = i;
            for (int q = 0; q < dim; q++) gg[q] += glocal[dim * iv + q];
            (void)wl;
        }
        int64_t nb = star_bfaces(dim, x, elems, star, ns, v, fb, 64);
        for (int64_t b = 0; b < nb && b < 64; b++) {
            const int32_t* f = fb + dim * b;
            double nB[3] = {0, 0, 0};
            face_area_vector(dim, x, f, nB);
            for (int c = 0; c < dim; c++) bn[c] += nB[c] / (double)dim;
            /* boundary-face share of L at v */
            double wB[3] = {0, 0, 0}, wt[3];
            int ned = dim == 3 ? 3 : 1;
            for (int a = 0; a < ned; a++) {
                int32_t a0 = f[a], a1 = f[(a + 1) % dim];
                or_hash_w(dim, a0 < a1 ? a0 : a1, a0 < a1 ? a1 : a0, seed, wt);
                for (int q = 0; q < dim; q++) wB[q] += wt[q];
            }
            double xl[9]; int32_t fl[3] = {0, 1, 2};
            for (int i = 0; i < dim; i++) for (int q = 0; q < dim; q++) xl[dim * i + q] = x[dim * f[i] + q];
            double glocal[9] = {0};
            bface_grad(dim, xl, fl, wB, 1.0 / (dim * (dim + 1.0)), glocal);
            for (int i = 0; i < dim; i++) if (f[i] == v) for (int q = 0; q < dim; q++) gg[q] += glocal[dim * i + q];
        }
        v_out[s] = vol;
        for (int c = 0; c < dim; c++) { b_out[dim * s + c] = bn[c]; g[c] = gg[c]; }
    }
    free_stars(&st);
    free(nodes);
}

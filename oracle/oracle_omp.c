/*
 * Multi-core CPU baseline of the proposed algorithm (forward + adjoint).
 *
 * TEST INFRASTRUCTURE ONLY, like the rest of oracle/: the benchmark times it
 * as the all-cores CPU comparison point; the GPU product path never loads it.
 * It is not a parity reference (the serial functions of oracle.c are): its
 * accumulation order depends on the thread schedule.
 *
 * It reuses the oracle's per-element arithmetic unchanged -- this file
 * includes oracle.c and calls its element helpers -- and only splits the
 * loops of or_direct and or_adjoint over threads:
 *   - element loop (Eq. efficient_njk_formula_general_D, Sec. 4.2 volumes,
 *     the element part of the adjoint): static ranges of elements per
 *     thread, every contribution added with an atomic update;
 *   - boundary loop (Sec. 3.2.3 correction and boundary normals, the
 *     boundary part of the adjoint): static ranges of faces, atomic updates;
 *   - 3D edge loop applying 1/12: split over edges.
 * Built with -fopenmp into liboracle_omp.so; without OpenMP the pragmas are
 * ignored and it runs on one thread.
 */
#include "oracle.c"

#ifdef _OPENMP
#include <omp.h>
#endif

static void atomic_add(double* p, double v) {
#pragma omp atomic update
    *p += v;
}

/* gradient of one element's part of L, as elem_grad computes it, on a copy of
 * the element whose nodes are renumbered 0..D in the order of their global ids
 * (so every lower-end test takes the same branch) and whose edges are 0..nl-1 */
static void elem_grad_local(int dim, const double* x, const int32_t* el, const int32_t* e2e_row, const double* w,
                            const double* c, double* gl /* [(dim+1)*dim] */) {
    const int nl = nloc_edges(dim);
    const int nn = dim + 1;
    double xl[4 * 3], wl[6 * 3], cl[4];
    int32_t ell[4] = {0, 0, 0, -1}, e2el[6];
    for (int i = 0; i < nn; i++) {
        int r = 0;
        for (int k = 0; k < nn; k++) r += el[k] < el[i];
        ell[i] = r;
        for (int q = 0; q < dim; q++) xl[dim * r + q] = x[dim * (int64_t)el[i] + q];
        cl[r] = c[el[i]];
    }
    for (int l = 0; l < nl; l++) {
        e2el[l] = l;
        for (int q = 0; q < dim; q++) wl[dim * l + q] = w[dim * (int64_t)e2e_row[l] + q];
    }
    for (int i = 0; i < nn * dim; i++) gl[i] = 0.0;
    elem_grad(dim, xl, ell, e2el, wl, cl, gl);
}

/* Forward (n_edge [nedges*dim], vol [nv], bnormal_full [nv*dim]) and
 * gradient g [nv*dim] of L = sum w.n + sum c V, all overwritten, on
 * `nthreads` threads (<= 0: the OpenMP default). */
void or_fused_omp(int nthreads, int dim, int64_t nv, const double* x, int64_t ne, const int32_t* elems,
                  const int32_t* elem2edge, int64_t nedges, const int32_t* edges, int64_t nb, const int32_t* bface,
                  const double* w, const double* c, double* n_edge, double* vol, double* bnormal_full, double* g) {
    const int nl = nloc_edges(dim);
    const int (*le)[2] = local_edges(dim);
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel
    {
#pragma omp for schedule(static)
        for (int64_t i = 0; i < nedges * dim; i++) n_edge[i] = 0.0;
#pragma omp for schedule(static)
        for (int64_t i = 0; i < nv; i++) vol[i] = 0.0;
#pragma omp for schedule(static)
        for (int64_t i = 0; i < nv * dim; i++) { bnormal_full[i] = 0.0; g[i] = 0.0; }

        /* element loop */
#pragma omp for schedule(static)
        for (int64_t E = 0; E < ne; E++) {
            const int32_t* el = elems + 4 * E;
            for (int l = 0; l < nl; l++) {
                double nj[3] = {0, 0, 0};
                face_opposite(dim, x, el, low_end(el, le[l]), nj);
                double* ne_ = n_edge + dim * (int64_t)elem2edge[E * nl + l];
                if (dim == 3)
                    for (int q = 0; q < 3; q++) atomic_add(&ne_[q], 2.0 * nj[q]);
                else
                    for (int q = 0; q < 2; q++) atomic_add(&ne_[q], nj[q] / 3.0);
            }
            const double vE = elem_volume(dim, x, el);
            for (int i = 0; i < dim + 1; i++) atomic_add(&vol[el[i]], vE / (double)(dim + 1));
            double gl[4 * 3];
            elem_grad_local(dim, x, el, elem2edge + nl * E, w, c, gl);
            for (int i = 0; i < dim + 1; i++) {
                int r = 0;
                for (int k = 0; k < dim + 1; k++) r += el[k] < el[i];
                for (int q = 0; q < dim; q++) atomic_add(&g[dim * (int64_t)el[i] + q], gl[dim * r + q]);
            }
        }

        /* boundary loop */
        const double beta = 1.0 / (dim * (dim + 1.0));
#pragma omp for schedule(static)
        for (int64_t B = 0; B < nb; B++) {
            const int32_t* f = bface + dim * B;
            double nB[3] = {0, 0, 0};
            face_area_vector(dim, x, f, nB);
            if (dim == 3) {
                for (int a = 0; a < 3; a++) {
                    const int64_t e = find_edge(nedges, edges, f[a], f[(a + 1) % 3]);
                    for (int q = 0; q < 3; q++) atomic_add(&n_edge[3 * e + q], nB[q]);
                }
            } else {
                const int64_t e = find_edge(nedges, edges, f[0], f[1]);
                for (int q = 0; q < 2; q++) atomic_add(&n_edge[2 * e + q], nB[q] / 6.0);
            }
            for (int a = 0; a < dim; a++)
                for (int q = 0; q < dim; q++) atomic_add(&bnormal_full[dim * (int64_t)f[a] + q], nB[q] / (double)dim);
            /* adjoint: the face's part, on a copy of the face renumbered 0..D-1 */
            double wB[3], xf[3 * 3], gf[3 * 3] = {0};
            int32_t fl[3] = {0, 1, 2};
            bface_edge_weight(dim, nedges, edges, f, w, wB);
            for (int a = 0; a < dim; a++)
                for (int q = 0; q < dim; q++) xf[dim * a + q] = x[dim * (int64_t)f[a] + q];
            bface_grad(dim, xf, fl, wB, beta, gf);
            for (int a = 0; a < dim; a++)
                for (int q = 0; q < dim; q++) atomic_add(&g[dim * (int64_t)f[a] + q], gf[dim * a + q]);
        }

        /* 3D: edge loop applying 1/12 */
        if (dim == 3) {
#pragma omp for schedule(static)
            for (int64_t e = 0; e < nedges * 3; e++) n_edge[e] *= (1.0 / 12.0);
        }
    }
}

/* threads an OpenMP parallel region gets by default (1 without OpenMP) */
int or_omp_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

// The ordered tile gather (EM_PATH_GATHER; plan layout in em_plan.cuh).  One
// CTA per tile; a tile owns a range of nodes, the edges whose lower end it
// owns and its boundary nodes, and computes every element that touches an
// owned node.  The tile's node coordinates (and, for the adjoint, w and c)
// are staged in shared memory (relative to the tile's first node for the
// FP32-based forms).  Elements are processed in chunks of one element per
// thread; each thread stages its element's three needed face area vectors,
// its volume (and, for the adjoint, its gradient terms) in shared memory,
// then every owned edge / node / boundary node sums its own slots of the
// chunk in the fixed order of the plan's gather lists.  Each output is
// produced by one CTA and written once, with no atomics, and the result is
// bit-identical from run to run.  (The scatter tiles of EM_PATH_TILED are in
// em_scatter.cu.)
//
// Element formulas (local nodes in ascending global id, so the lower end of
// edge (p,q), p<q, is local node p), 3D: a,b,c = x1-x0, x2-x0, x3-x0,
//   N1 = b x c, N2 = c x a, N3 = a x b, det = a.N1, s = sign(det);
//   the outward area vector of the face opposite node i is -s N_i / 2 and
//   n_0 = -(n_1+n_2+n_3), so the proposed algorithm's contribution
//   2/(D(D+1)) n_p to edge (p,q) is m_p/12 with
//   m_0 = s(N1+N2+N3), m_1 = -s N1, m_2 = -s N2      (Eq. efficient_njk_formula_general_D)
//   V_E/(D+1) = |det|/24                                  (Sec. 4.2)
//   boundary face B: + n_B/12 on its edges, n_B/3 on its nodes (Sec. 3.2.3).
// 2D: n_1 = -s (b_y,-b_x), n_2 = -s (-a_y,a_x), n_0 = -(n_1+n_2), edge
// contribution n_p/3, V_E/3 = |det|/6, boundary n_B/6 on the edge, n_B/2 on
// its nodes.
// Adjoint: see em_atomic.cu (W_i, A_i, C and the closed-form element gradient).
#include "em_common.cuh"
#include "em_dw.cuh"
#include "em_kernels.cuh"
#include "em_plan.cuh"
#include "em_tile_forms.cuh"

namespace em {

namespace {

constexpr int NT = 256;   // threads per CTA = elements per chunk

// shared-memory layout, computed identically on host and device
struct Smem {
    size_t xs, ws, cs, st_m, st_v, st_g, acc_e, cur_e, acc_v, acc_g, cur_n, acc_b, cur_b;
    size_t eptr, eslot, nptr, nslot, bptr, bslot, total;
};

struct Dims {
    int max_nodes, max_edges, max_eo, max_own, max_bo, max_es, max_ns, max_bs;
};

template <int DIM, int PREC, int WHAT>
__host__ __device__ inline Smem smem_layout(const Dims& D) {
    const int max_nodes = D.max_nodes, max_edges = D.max_edges, max_eo = D.max_eo, max_own = D.max_own,
              max_bo = D.max_bo;
    using F = Form<PREC>;
    constexpr int NN = DIM;          // staged face vectors per element (3D: m0,m1,m2; 2D: m0,m1)
    Smem s;
    size_t o = 0;
    auto take = [&](size_t bytes) { o = (o + 15) & ~size_t(15); size_t r = o; o += bytes; return r; };
    s.xs = take(sizeof(typename F::C) * DIM * max_nodes);
    s.ws = (WHAT & DO_ADJ) ? take(sizeof(typename F::V) * DIM * max_edges) : 0;
    s.cs = (WHAT & DO_ADJ) ? take(sizeof(typename F::V) * max_nodes) : 0;
    s.st_m = (WHAT & DO_FWD) ? take(sizeof(typename F::V) * NN * DIM * NT) : 0;
    s.st_v = (WHAT & DO_FWD) ? take(sizeof(typename F::V) * NT) : 0;
    s.st_g = (WHAT & DO_ADJ) ? take(sizeof(typename F::V) * (DIM + 1) * DIM * NT) : 0;
    s.acc_e = (WHAT & DO_FWD) ? take(sizeof(typename F::A) * DIM * max_eo) : 0;
    s.cur_e = (WHAT & DO_FWD) ? take(sizeof(int) * max_eo * DIM) : 0;
    s.acc_v = (WHAT & DO_FWD) ? take(sizeof(typename F::A) * max_own) : 0;
    s.acc_g = (WHAT & DO_ADJ) ? take(sizeof(typename F::A) * DIM * max_own) : 0;
    s.cur_n = take(sizeof(int) * max_own * (((WHAT & DO_FWD) ? 1 : 0) + ((WHAT & DO_ADJ) ? DIM : 0)));
    s.acc_b = (WHAT & DO_FWD) ? take(sizeof(typename F::A) * DIM * max_bo) : 0;
    s.cur_b = take(sizeof(int) * max_bo * (((WHAT & DO_FWD) ? DIM : 0) + ((WHAT & DO_ADJ) ? DIM : 0)));
    s.eptr = (WHAT & DO_FWD) ? take(sizeof(int) * (max_eo + 1)) : 0;
    s.eslot = (WHAT & DO_FWD) ? take(sizeof(uint16_t) * D.max_es) : 0;
    s.nptr = take(sizeof(int) * (max_own + 1));
    s.nslot = take(sizeof(uint16_t) * D.max_ns);
    s.bptr = take(sizeof(int) * (max_bo + 1));
    s.bslot = take(sizeof(uint16_t) * D.max_bs);
    s.total = (o + 15) & ~size_t(15);
    return s;
}

struct TileArgs {
    const void* plan;
    const int32_t* bnode;
    const double* x;
    const double* w;
    const double* c;
    double* n_out;
    double* vol;
    double* bnormal;
    double* grad;
    Dims D;
    int n_tiles;
    int64_t tile_base;      // first tile handled by blockIdx.x == 0
};

template <int DIM, int PREC, int WHAT>
__device__ __forceinline__ void run_tile(const TileArgs& A, int t, char* smem) {
    using F = Form<PREC>;
    using C = typename F::C;
    using V = typename F::V;
    using Acc = typename F::A;
    constexpr int NN = DIM;
    const PlanHeader* H = static_cast<const PlanHeader*>(A.plan);
    const TileInfo ti = plan_at<TileInfo>(A.plan, H->off_tiles)[t];
    const ElemConn* conn = plan_at<ElemConn>(A.plan, H->off_conn) + ti.elem_off;
    const ElemEdges* tedge = plan_at<ElemEdges>(A.plan, H->off_tedge) + ti.elem_off;
    const int32_t* halo = plan_at<int32_t>(A.plan, H->off_halo) + ti.halo_off;
    const int32_t* hedge = plan_at<int32_t>(A.plan, H->off_hedge) + ti.hedge_off;
    const int32_t* eptr = plan_at<int32_t>(A.plan, H->off_eslot_ptr);
    const uint16_t* eslot = plan_at<uint16_t>(A.plan, H->off_eslot);
    const int32_t* nptr = plan_at<int32_t>(A.plan, H->off_nslot_ptr);
    const uint16_t* nslot = plan_at<uint16_t>(A.plan, H->off_nslot);
    const TileBFace* tbf = plan_at<TileBFace>(A.plan, H->off_tbf) + ti.bf_off;
    const int32_t* bptr = plan_at<int32_t>(A.plan, H->off_bslot_ptr);
    const uint16_t* bslot = plan_at<uint16_t>(A.plan, H->off_bslot);

    const Smem L = smem_layout<DIM, PREC, WHAT>(A.D);
    C* xs = reinterpret_cast<C*>(smem + L.xs);
    V* ws = reinterpret_cast<V*>(smem + L.ws);
    V* cs = reinterpret_cast<V*>(smem + L.cs);
    V* st_m = reinterpret_cast<V*>(smem + L.st_m);
    V* st_v = reinterpret_cast<V*>(smem + L.st_v);
    V* st_g = reinterpret_cast<V*>(smem + L.st_g);
    Acc* acc_e = reinterpret_cast<Acc*>(smem + L.acc_e);
    int* cur_e = reinterpret_cast<int*>(smem + L.cur_e);
    Acc* acc_v = reinterpret_cast<Acc*>(smem + L.acc_v);
    Acc* acc_g = reinterpret_cast<Acc*>(smem + L.acc_g);
    int* cur_n = reinterpret_cast<int*>(smem + L.cur_n);
    Acc* acc_b = reinterpret_cast<Acc*>(smem + L.acc_b);
    int* cur_b = reinterpret_cast<int*>(smem + L.cur_b);
    int* s_eptr = reinterpret_cast<int*>(smem + L.eptr);
    uint16_t* s_eslot = reinterpret_cast<uint16_t*>(smem + L.eslot);
    int* s_nptr = reinterpret_cast<int*>(smem + L.nptr);
    uint16_t* s_nslot = reinterpret_cast<uint16_t*>(smem + L.nslot);
    int* s_bptr = reinterpret_cast<int*>(smem + L.bptr);
    uint16_t* s_bslot = reinterpret_cast<uint16_t*>(smem + L.bslot);

    const int tid = threadIdx.x;
    const int nnodes = ti.n_own + ti.n_halo;
    // gather work items: one per (output, component)
    constexpr int NCN = ((WHAT & DO_FWD) ? 1 : 0) + ((WHAT & DO_ADJ) ? DIM : 0);   // node: [grad comps..., V]
    constexpr int NCB = ((WHAT & DO_FWD) ? DIM : 0) + ((WHAT & DO_ADJ) ? DIM : 0);  // boundary node: [bnormal, grad]
    double org[DIM];
    tile_origin<DIM>(A.x, ti.node0, ti.n_own, org);

    // ---- stage coordinates (and w, c), reset accumulators ----------------
    for (int i = tid; i < nnodes; i += NT) {
        int64_t v = i < ti.n_own ? int64_t(ti.node0) + i : int64_t(halo[i - ti.n_own]);
#pragma unroll
        for (int d = 0; d < DIM; d++) xs[i * DIM + d] = F::coord(A.x[v * DIM + d], org[d]);
        if (WHAT & DO_ADJ) cs[i] = A.c ? F::from_double(A.c[v]) : F::cst(0.0);
    }
    if (WHAT & DO_ADJ) {
        const int nte = ti.n_eo + ti.n_hedge;
        for (int i = tid; i < nte; i += NT) {
            int64_t e = i < ti.n_eo ? int64_t(ti.edge0) + i : int64_t(hedge[i - ti.n_eo]);
#pragma unroll
            for (int d = 0; d < DIM; d++) ws[i * DIM + d] = F::from_double(A.w[e * DIM + d]);
        }
    }
    // gather lists of the tile, copied to shared memory (offsets made local)
    if (WHAT & DO_FWD) {
        const int e_base = eptr[ti.edge0];
        const int ne_sl = eptr[ti.edge0 + ti.n_eo] - e_base;
        for (int i = tid; i <= ti.n_eo; i += NT) s_eptr[i] = eptr[ti.edge0 + i] - e_base;
        for (int q = tid; q < ne_sl; q += NT) s_eslot[q] = eslot[e_base + q];
        for (int q = tid; q < ti.n_eo * DIM; q += NT) {
            acc_e[q] = F::zero();
            cur_e[q] = eptr[ti.edge0 + q / DIM] - e_base;
        }
    }
    {
        const int n_base = nptr[ti.node0];
        const int nn_sl = nptr[ti.node0 + ti.n_own] - n_base;
        for (int i = tid; i <= ti.n_own; i += NT) s_nptr[i] = nptr[ti.node0 + i] - n_base;
        for (int q = tid; q < nn_sl; q += NT) s_nslot[q] = nslot[n_base + q];
        for (int i = tid; i < ti.n_own; i += NT) {
            if (WHAT & DO_FWD) acc_v[i] = F::zero();
            if (WHAT & DO_ADJ) {
#pragma unroll
                for (int d = 0; d < DIM; d++) acc_g[i * DIM + d] = F::zero();
            }
        }
        for (int q = tid; q < ti.n_own * NCN; q += NT) cur_n[q] = nptr[ti.node0 + q / NCN] - n_base;
    }
    if (ti.n_bo) {
        const int b_base = bptr[ti.bnode0];
        const int nb_sl = bptr[ti.bnode0 + ti.n_bo] - b_base;
        for (int i = tid; i <= ti.n_bo; i += NT) s_bptr[i] = bptr[ti.bnode0 + i] - b_base;
        for (int q = tid; q < nb_sl; q += NT) s_bslot[q] = bslot[b_base + q];
        for (int k = tid; k < ti.n_bo; k += NT) {
            if (WHAT & DO_FWD) {
#pragma unroll
                for (int d = 0; d < DIM; d++) acc_b[k * DIM + d] = F::zero();
            }
        }
        for (int q = tid; q < ti.n_bo * NCB; q += NT) cur_b[q] = bptr[ti.bnode0 + q / NCB] - b_base;
    }
    __syncthreads();

    // ---- element chunks ------------------------------------------------------
    ElemConn cn_next;
    ElemEdges ee_next;
    if (tid < ti.n_el) {
        cn_next = conn[tid];
        if (WHAT & DO_ADJ) ee_next = tedge[tid];
    }
    for (int cb = 0; cb < ti.n_el; cb += NT) {
        const int j = tid;
        const ElemConn cn_cur = cn_next;
        const ElemEdges ee_cur = ee_next;
        if (cb + NT + j < ti.n_el) {          // prefetch the next chunk's records
            cn_next = conn[cb + NT + j];
            if (WHAT & DO_ADJ) ee_next = tedge[cb + NT + j];
        }
        if (cb + j < ti.n_el) {
            const ElemConn cn = cn_cur;
            if (DIM == 3) {
                V a[3], b[3], c[3];
#pragma unroll
                for (int d = 0; d < 3; d++) {
                    a[d] = F::diff(xs[cn.v[1] * 3 + d], xs[cn.v[0] * 3 + d]);
                    b[d] = F::diff(xs[cn.v[2] * 3 + d], xs[cn.v[0] * 3 + d]);
                    c[d] = F::diff(xs[cn.v[3] * 3 + d], xs[cn.v[0] * 3 + d]);
                }
                V N1[3] = {F::det2(b[1], c[2], b[2], c[1]), F::det2(b[2], c[0], b[0], c[2]), F::det2(b[0], c[1], b[1], c[0])};
                V N2[3] = {F::det2(c[1], a[2], c[2], a[1]), F::det2(c[2], a[0], c[0], a[2]), F::det2(c[0], a[1], c[1], a[0])};
                V N3[3] = {F::det2(a[1], b[2], a[2], b[1]), F::det2(a[2], b[0], a[0], b[2]), F::det2(a[0], b[1], a[1], b[0])};
                V det = F::add(F::add(F::mul(a[0], N1[0]), F::mul(a[1], N1[1])), F::mul(a[2], N1[2]));
                const float s = F::sign_of(det);
                if (WHAT & DO_FWD) {
                    V* m = st_m + j * (NN * 3);
#pragma unroll
                    for (int d = 0; d < 3; d++) {
                        m[0 * 3 + d] = F::sgn(F::add(F::add(N1[d], N2[d]), N3[d]), s);
                        m[1 * 3 + d] = F::sgn(N1[d], -s);
                        m[2 * 3 + d] = F::sgn(N2[d], -s);
                    }
                    st_v[j] = F::sgn(det, s);
                }
                if (WHAT & DO_ADJ) {
                    const ElemEdges ee = ee_cur;
                    V W0[3], W1[3], W2[3];
#pragma unroll
                    for (int d = 0; d < 3; d++) {
                        W0[d] = F::add(F::add(ws[ee.e[0] * 3 + d], ws[ee.e[1] * 3 + d]), ws[ee.e[2] * 3 + d]);
                        W1[d] = F::add(ws[ee.e[3] * 3 + d], ws[ee.e[4] * 3 + d]);
                        W2[d] = ws[ee.e[5] * 3 + d];
                    }
                    V A1[3], A2[3], A3[3];
#pragma unroll
                    for (int d = 0; d < 3; d++) {
                        A1[d] = F::sub(W1[d], W0[d]);
                        A2[d] = F::sub(W2[d], W0[d]);
                        A3[d] = F::sgn(W0[d], -1.f);
                    }
                    V Cs = F::add(F::add(cs[cn.v[0]], cs[cn.v[1]]), F::add(cs[cn.v[2]], cs[cn.v[3]]));
                    const V f12 = F::cst(-1.0 / 12.0), f24 = F::cst(1.0 / 24.0);
                    V h = F::sgn(F::mul(Cs, f24), s);
                    V g[4][3];
#pragma unroll
                    for (int d = 0; d < 3; d++) {
                        const int d1 = (d + 1) % 3, d2 = (d + 2) % 3;
                        // (u x v)_d = u_d1 v_d2 - u_d2 v_d1
                        V ga = F::sub(F::det2(A2[d1], c[d2], A2[d2], c[d1]), F::det2(A3[d1], b[d2], A3[d2], b[d1]));
                        V gb = F::sub(F::det2(A3[d1], a[d2], A3[d2], a[d1]), F::det2(A1[d1], c[d2], A1[d2], c[d1]));
                        V gc = F::sub(F::det2(A1[d1], b[d2], A1[d2], b[d1]), F::det2(A2[d1], a[d2], A2[d2], a[d1]));
                        g[1][d] = F::add(F::sgn(F::mul(ga, f12), s), F::mul(h, N1[d]));
                        g[2][d] = F::add(F::sgn(F::mul(gb, f12), s), F::mul(h, N2[d]));
                        g[3][d] = F::add(F::sgn(F::mul(gc, f12), s), F::mul(h, N3[d]));
                        g[0][d] = F::sgn(F::add(F::add(g[1][d], g[2][d]), g[3][d]), -1.f);
                    }
                    V* gg = st_g + j * 12;
#pragma unroll
                    for (int r = 0; r < 4; r++)
#pragma unroll
                        for (int d = 0; d < 3; d++) gg[r * 3 + d] = g[r][d];
                }
            } else {
                V a[2], b[2];
#pragma unroll
                for (int d = 0; d < 2; d++) {
                    a[d] = F::diff(xs[cn.v[1] * 2 + d], xs[cn.v[0] * 2 + d]);
                    b[d] = F::diff(xs[cn.v[2] * 2 + d], xs[cn.v[0] * 2 + d]);
                }
                V det = F::det2(a[0], b[1], a[1], b[0]);
                const float s = F::sign_of(det);
                if (WHAT & DO_FWD) {
                    // n_1 = -s (b_y, -b_x), n_2 = -s (-a_y, a_x), n_0 = -(n_1 + n_2)
                    V n1x = F::sgn(b[1], -s), n1y = F::sgn(b[0], s);
                    V n2x = F::sgn(a[1], s), n2y = F::sgn(a[0], -s);
                    V* m = st_m + j * (NN * 2);
                    m[0] = F::sgn(F::add(n1x, n2x), -1.f);
                    m[1] = F::sgn(F::add(n1y, n2y), -1.f);
                    m[2] = n1x;
                    m[3] = n1y;
                    st_v[j] = F::sgn(det, s);
                }
                if (WHAT & DO_ADJ) {
                    const ElemEdges ee = ee_cur;
                    V W0[2], W1[2];
#pragma unroll
                    for (int d = 0; d < 2; d++) {
                        W0[d] = F::add(ws[ee.e[0] * 2 + d], ws[ee.e[1] * 2 + d]);
                        W1[d] = ws[ee.e[2] * 2 + d];
                    }
                    V A1[2] = {F::sub(W1[0], W0[0]), F::sub(W1[1], W0[1])};
                    V A2[2] = {F::sgn(W0[0], -1.f), F::sgn(W0[1], -1.f)};
                    V Cs = F::add(F::add(cs[cn.v[0]], cs[cn.v[1]]), cs[cn.v[2]]);
                    const V f3 = F::cst(1.0 / 3.0), f6 = F::cst(1.0 / 6.0);
                    V h = F::sgn(F::mul(Cs, f6), s);
                    // g_a = (s/3)(-A2y, A2x) + h (b_y, -b_x); g_b = (s/3)(A1y, -A1x) + h (-a_y, a_x)
                    V gax = F::add(F::sgn(F::mul(A2[1], f3), -s), F::mul(h, b[1]));
                    V gay = F::add(F::sgn(F::mul(A2[0], f3), s), F::sgn(F::mul(h, b[0]), -1.f));
                    V gbx = F::add(F::sgn(F::mul(A1[1], f3), s), F::sgn(F::mul(h, a[1]), -1.f));
                    V gby = F::add(F::sgn(F::mul(A1[0], f3), -s), F::mul(h, a[0]));
                    V* gg = st_g + j * 6;
                    gg[0] = F::sgn(F::add(gax, gbx), -1.f);
                    gg[1] = F::sgn(F::add(gay, gby), -1.f);
                    gg[2] = gax; gg[3] = gay;
                    gg[4] = gbx; gg[5] = gby;
                }
            }
        }
        __syncthreads();
        const int cend = cb + NT;
        if (WHAT & DO_FWD) {
            for (int q = tid; q < ti.n_eo * DIM; q += NT) {
                const int le = q / DIM, d = q - le * DIM;
                int cur = cur_e[q];
                const int end = s_eptr[le + 1];
                Acc a = acc_e[q];
                while (cur < end) {
                    const unsigned sl = s_eslot[cur];
                    const int code = sl & 3, idx = (int)(sl >> 2);
                    if (code == 3 || idx >= cend) break;
                    F::acc(a, st_m[(idx - cb) * (NN * DIM) + code * DIM + d]);
                    cur++;
                }
                acc_e[q] = a;
                cur_e[q] = cur;
            }
        }
        for (int q = tid; q < ti.n_own * NCN; q += NT) {
            const int i = q / NCN, k = q - i * NCN;
            int cur = cur_n[q];
            const int end = s_nptr[i + 1];
            const bool isv = (WHAT & DO_FWD) && k == NCN - 1;
            Acc a = isv ? acc_v[i] : acc_g[i * DIM + k];
            while (cur < end) {
                const unsigned sl = s_nslot[cur];
                const int r = sl & 3, idx = (int)(sl >> 2);
                if (idx >= cend) break;
                if (isv) F::acc(a, st_v[idx - cb]);
                else F::acc(a, st_g[(idx - cb) * ((DIM + 1) * DIM) + r * DIM + k]);
                cur++;
            }
            if (isv) acc_v[i] = a;
            else acc_g[i * DIM + k] = a;
            cur_n[q] = cur;
        }
        __syncthreads();
    }

    // ---- boundary faces --------------------------------------------------------
    for (int bb = 0; bb < ti.n_bf; bb += NT) {
        const int j = tid;
        if (bb + j < ti.n_bf) {
            const TileBFace f = tbf[bb + j];
            if (DIM == 3) {
                V u[3], tt[3];
#pragma unroll
                for (int d = 0; d < 3; d++) {
                    u[d] = F::diff(xs[f.v[1] * 3 + d], xs[f.v[0] * 3 + d]);
                    tt[d] = F::diff(xs[f.v[2] * 3 + d], xs[f.v[0] * 3 + d]);
                }
                if (WHAT & DO_FWD) {
                    V* m = st_m + j * (NN * 3);
                    m[0] = F::half(F::det2(u[1], tt[2], u[2], tt[1]));
                    m[1] = F::half(F::det2(u[2], tt[0], u[0], tt[2]));
                    m[2] = F::half(F::det2(u[0], tt[1], u[1], tt[0]));
                }
                if (WHAT & DO_ADJ) {
                    V WB[3];
#pragma unroll
                    for (int d = 0; d < 3; d++)
                        WB[d] = F::add(F::add(ws[f.e[0] * 3 + d], ws[f.e[1] * 3 + d]), ws[f.e[2] * 3 + d]);
                    const V f24 = F::cst(1.0 / 24.0);
                    V* gg = st_g + j * 12;
#pragma unroll
                    for (int d = 0; d < 3; d++) {
                        const int d1 = (d + 1) % 3, d2 = (d + 2) % 3;
                        V gq = F::mul(F::det2(tt[d1], WB[d2], tt[d2], WB[d1]), f24);   // (t x W)/24
                        V gr = F::mul(F::det2(WB[d1], u[d2], WB[d2], u[d1]), f24);     // (W x u)/24
                        gg[1 * 3 + d] = gq;
                        gg[2 * 3 + d] = gr;
                        gg[0 * 3 + d] = F::sgn(F::add(gq, gr), -1.f);
                    }
                }
            } else {
                if (WHAT & DO_FWD) {
                    V* m = st_m + j * (NN * 2);
                    m[0] = F::diff(xs[f.v[0] * 2 + 1], xs[f.v[1] * 2 + 1]);   // y_a - y_b
                    m[1] = F::diff(xs[f.v[1] * 2 + 0], xs[f.v[0] * 2 + 0]);   // x_b - x_a
                }
                if (WHAT & DO_ADJ) {
                    const V f6 = F::cst(1.0 / 6.0);
                    V gx = F::mul(ws[f.e[0] * 2 + 1], f6);
                    V gy = F::sgn(F::mul(ws[f.e[0] * 2 + 0], f6), -1.f);
                    V* gg = st_g + j * 6;
                    gg[2] = gx; gg[3] = gy;
                    gg[0] = F::sgn(gx, -1.f);
                    gg[1] = F::sgn(gy, -1.f);
                }
            }
        }
        __syncthreads();
        const int bend = bb + NT;
        if (WHAT & DO_FWD) {
            for (int q = tid; q < ti.n_eo * DIM; q += NT) {
                const int le = q / DIM, d = q - le * DIM;
                int cur = cur_e[q];
                const int end = s_eptr[le + 1];
                Acc a = acc_e[q];
                while (cur < end) {
                    const unsigned sl = s_eslot[cur];
                    const int idx = (int)(sl >> 2);
                    if (idx >= bend) break;
                    const V m = st_m[(idx - bb) * (NN * DIM) + d];
                    F::acc(a, DIM == 3 ? m : F::half(m));
                    cur++;
                }
                acc_e[q] = a;
                cur_e[q] = cur;
            }
        }
        for (int q = tid; q < ti.n_bo * NCB; q += NT) {
            const int kb = q / NCB, k = q - kb * NCB;
            int cur = cur_b[q];
            const int end = s_bptr[kb + 1];
            const bool isb = (WHAT & DO_FWD) && k < DIM;
            const int d = isb ? k : k - ((WHAT & DO_FWD) ? DIM : 0);
            const int i = A.bnode[ti.bnode0 + kb] - ti.node0;
            Acc a = isb ? acc_b[kb * DIM + d] : acc_g[i * DIM + d];
            while (cur < end) {
                const unsigned sl = s_bslot[cur];
                const int pos = sl & 3, idx = (int)(sl >> 2);
                if (idx >= bend) break;
                if (isb) F::acc(a, st_m[(idx - bb) * (NN * DIM) + d]);
                else F::acc(a, st_g[(idx - bb) * ((DIM + 1) * DIM) + pos * DIM + d]);
                cur++;
            }
            if (isb) acc_b[kb * DIM + d] = a;
            else acc_g[i * DIM + d] = a;
            cur_b[q] = cur;
        }
        __syncthreads();
    }

    // ---- write every owned output once ---------------------------------------
    const double esc = DIM == 3 ? 1.0 / 12.0 : 1.0 / 3.0;
    const double vsc = DIM == 3 ? 1.0 / 24.0 : 1.0 / 6.0;
    const double bsc = DIM == 3 ? 1.0 / 3.0 : 1.0 / 2.0;
    if (WHAT & DO_FWD) {
        for (int le = tid; le < ti.n_eo; le += NT) {
#pragma unroll
            for (int d = 0; d < DIM; d++)
                A.n_out[(int64_t(ti.edge0) + le) * DIM + d] = F::out(acc_e[le * DIM + d], esc);
        }
        for (int k = tid; k < ti.n_bo; k += NT) {
#pragma unroll
            for (int d = 0; d < DIM; d++)
                A.bnormal[(int64_t(ti.bnode0) + k) * DIM + d] = F::out(acc_b[k * DIM + d], bsc);
        }
    }
    for (int i = tid; i < ti.n_own; i += NT) {
        if (WHAT & DO_FWD) A.vol[int64_t(ti.node0) + i] = F::out(acc_v[i], vsc);
        if (WHAT & DO_ADJ) {
#pragma unroll
            for (int d = 0; d < DIM; d++) A.grad[(int64_t(ti.node0) + i) * DIM + d] = F::out(acc_g[i * DIM + d], 1.0);
        }
    }
}


template <int DIM, int PREC, int WHAT>
__global__ void __launch_bounds__(NT) k_tile(TileArgs A) {
    extern __shared__ __align__(16) char smem[];
    run_tile<DIM, PREC, WHAT>(A, (int)(A.tile_base + blockIdx.x), smem);
}

template <int DIM, int PREC, int WHAT>
int launch_tiles(const em_mesh* m, TileArgs& A, cudaStream_t s) {
    const Smem L = smem_layout<DIM, PREC, WHAT>(A.D);
    static size_t configured = 0;
    if (L.total > 227 * 1024)
        return fail(EM_ERR_ARG, "tile needs " + std::to_string(L.total) +
                                    " bytes of shared memory (> 227 KB): rebuild the plan with a smaller tile_nodes");
    if (L.total > 48 * 1024 && L.total > configured) {
        EM_CUDA_TRY(cudaFuncSetAttribute(k_tile<DIM, PREC, WHAT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         227 * 1024));
        configured = 227 * 1024;
    }
    const int64_t n_tiles = m->plan_info[EM_PLAN_INFO_TILES];
    const int64_t chunk = 1 << 30;
    for (int64_t base = 0; base < n_tiles; base += chunk) {
        A.tile_base = base;
        int64_t nb = n_tiles - base < chunk ? n_tiles - base : chunk;
        k_tile<DIM, PREC, WHAT><<<(unsigned)nb, NT, L.total, s>>>(A);
        note_launches(1);
    }
    EM_CUDA_TRY(cudaGetLastError());
    return EM_OK;
}


template <int DIM, int PREC>
int dispatch_what(const em_mesh* m, int what, TileArgs& A, cudaStream_t s) {
    if (what == GATHER_FWD) return launch_tiles<DIM, PREC, DO_FWD>(m, A, s);
    if (what == GATHER_ADJ) return launch_tiles<DIM, PREC, DO_ADJ>(m, A, s);
    return launch_tiles<DIM, PREC, DO_FWD | DO_ADJ>(m, A, s);
}

}  // namespace

size_t gather_ws_bytes(const em_mesh* m, int what) {
    return (what & GATHER_SCATTER) ? scatter_ws_bytes(m) : 0;
}

int gather_run(const em_mesh* m, int prec, int what, const double* x, const double* w, const double* c, double* n,
               double* vol, double* bnormal, double* g, void* ws, cudaStream_t s, const BwAux* bw) {
    const int64_t* pi = m->plan_info;
    if (pi[EM_PLAN_INFO_TILES] <= 0 || pi[EM_PLAN_INFO_CHECK] <= 0 || (size_t)pi[EM_PLAN_INFO_CHECK] > m->plan_bytes)
        return fail(EM_ERR_ARG, "mesh->plan_info does not describe mesh->plan (copy em_plan_build's plan_info)");
    if (m->n_bnodes && !m->bnode) return fail(EM_ERR_ARG, "gather path needs bnode");
    if (what & GATHER_SCATTER) return scatter_run(m, prec, what & (GATHER_FWD | GATHER_ADJ), x, w, c, n, vol, bnormal, g, ws, s, bw);
    if (bw && bw->bw) return fail(EM_ERR_ARG, "boundary-normal weights are supported by the TILED and ATOMIC paths");
    TileArgs A;
    A.plan = m->plan;
    A.bnode = m->bnode;
    A.x = x; A.w = w; A.c = c;
    A.n_out = n; A.vol = vol; A.bnormal = bnormal; A.grad = g;
    A.D.max_nodes = (int)pi[EM_PLAN_INFO_MAX_NODES];
    A.D.max_edges = (int)pi[EM_PLAN_INFO_MAX_EDGES];
    A.D.max_eo = (int)pi[EM_PLAN_INFO_MAX_OWNED_EDGES];
    A.D.max_own = (int)pi[EM_PLAN_INFO_MAX_OWNED_NODES];
    A.D.max_bo = (int)pi[EM_PLAN_INFO_MAX_OWNED_BNODES];
    A.D.max_es = (int)pi[EM_PLAN_INFO_MAX_ESLOTS];
    A.D.max_ns = (int)pi[EM_PLAN_INFO_MAX_NSLOTS];
    A.D.max_bs = (int)pi[EM_PLAN_INFO_MAX_BSLOTS];
    A.n_tiles = (int)pi[EM_PLAN_INFO_TILES];
    A.tile_base = 0;
    (void)ws;
    if (m->dim == 3) {
        if (prec == EM_PREC_FP64) return dispatch_what<3, EM_PREC_FP64>(m, what, A, s);
        if (prec == EM_PREC_DW) return dispatch_what<3, EM_PREC_DW>(m, what, A, s);
        return dispatch_what<3, EM_PREC_MIXED>(m, what, A, s);
    }
    if (prec == EM_PREC_FP64) return dispatch_what<2, EM_PREC_FP64>(m, what, A, s);
    if (prec == EM_PREC_DW) return dispatch_what<2, EM_PREC_DW>(m, what, A, s);
    return dispatch_what<2, EM_PREC_MIXED>(m, what, A, s);
}

}  // namespace em

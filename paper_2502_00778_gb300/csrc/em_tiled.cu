// The tiled paths (plan layout in em_plan.cuh).  One CTA per tile; a tile
// owns a range of nodes, the edges whose lower end it owns and its boundary
// nodes, and computes every element that touches an owned node.  The tile's
// node coordinates (and, for the adjoint, w and c) are staged in shared
// memory (relative to the tile's first node for the FP32-based forms).  Two
// ways of summing the element contributions into the owned outputs:
//
// EM_PATH_GATHER (run_tile): elements are processed in chunks of one element
// per thread; each thread stages its element's three needed face area
// vectors, its volume (and, for the adjoint, its gradient terms) in shared
// memory, then every owned edge / node / boundary node sums its own slots of
// the chunk in the fixed order of the plan's gather lists.
//
// EM_PATH_TILED (run_tile_scatter): each element adds its contributions to
// the owned targets directly, with shared-memory integer atomics on exact
// fixed-point limbs (see the scatter section below); elements are grouped by
// which of their nodes the tile owns, so warps skip unowned outputs together.
//
// Either way each output is produced by one CTA and written once, with no
// global atomics, and the result is bit-identical from run to run.
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

namespace em {

namespace {

constexpr int NT = 256;   // threads per CTA = elements per chunk

// ---------------------------------------------------------------------------
// precision forms
// ---------------------------------------------------------------------------
template <int PREC>
struct Form;

template <>
struct Form<EM_PREC_FP64> {
    // explicitly rounded operations: every kernel that inlines this form
    // evaluates the same expressions (no compiler-chosen FMA contraction)
    using C = double;  // staged coordinate (raw)
    using V = double;  // element value
    using A = double;  // accumulator
    static __device__ __forceinline__ C coord(double x, double) { return x; }
    static __device__ __forceinline__ V diff(C a, C b) { return __dsub_rn(a, b); }
    static __device__ __forceinline__ V add(V a, V b) { return __dadd_rn(a, b); }
    static __device__ __forceinline__ V sub(V a, V b) { return __dsub_rn(a, b); }
    static __device__ __forceinline__ V mul(V a, V b) { return __dmul_rn(a, b); }
    static __device__ __forceinline__ V det2(V p, V q, V r, V s) { return __fma_rn(p, q, -__dmul_rn(r, s)); }
    static __device__ __forceinline__ V sgn(V a, float s) { return s < 0.f ? -a : a; }
    static __device__ __forceinline__ V half(V a) { return __dmul_rn(0.5, a); }
    static __device__ __forceinline__ float sign_of(V a) { return a > 0.0 ? 1.f : -1.f; }
    static __device__ __forceinline__ V from_double(double d) { return d; }
    static __device__ __forceinline__ V cst(double d) { return d; }
    static __device__ __forceinline__ A zero() { return 0.0; }
    static __device__ __forceinline__ void acc(A& a, V v) { a = __dadd_rn(a, v); }
    static __device__ __forceinline__ double out(A a, double sc) { return __dmul_rn(a, sc); }
};

template <>
struct Form<EM_PREC_DW> {
    using C = dw;
    using V = dw;
    using A = dw;
    static __device__ __forceinline__ C coord(double x, double o) { return dw_from_double(x - o); }
    static __device__ __forceinline__ V diff(C a, C b) { return dw_sub_n(a, b); }
    static __device__ __forceinline__ V add(V a, V b) { return dw_add(a, b); }
    static __device__ __forceinline__ V sub(V a, V b) { return dw_sub(a, b); }
    static __device__ __forceinline__ V mul(V a, V b) { return dw_mul(a, b); }
    static __device__ __forceinline__ V det2(V p, V q, V r, V s) { return dw_det2(p, q, r, s); }
    static __device__ __forceinline__ V sgn(V a, float s) { return dw_sgn(a, s); }
    static __device__ __forceinline__ V half(V a) { return {__fmul_rn(0.5f, a.h), __fmul_rn(0.5f, a.l)}; }
    static __device__ __forceinline__ float sign_of(V a) { return (a.h > 0.f || (a.h == 0.f && a.l > 0.f)) ? 1.f : -1.f; }
    static __device__ __forceinline__ V from_double(double d) { return dw_from_double(d); }
    static __device__ __forceinline__ V cst(double d) { return dw_from_double(d); }
    static __device__ __forceinline__ A zero() { return {0.f, 0.f}; }
    static __device__ __forceinline__ void acc(A& a, V v) { dw_acc(a, v); }
    static __device__ __forceinline__ double out(A a, double sc) {
        dw s = dw_from_double(sc);
        return dw_to_double(dw_mulc(a, s.h, s.l));
    }
};

template <>
struct Form<EM_PREC_MIXED> {
    using C = dw;     // tile-relative coordinates kept exact, element math in FP32
    using V = float;
    using A = dw;     // compensated FP32 accumulation
    static __device__ __forceinline__ C coord(double x, double o) { return dw_from_double(x - o); }
    static __device__ __forceinline__ V diff(C a, C b) { return (a.h - b.h) + (a.l - b.l); }
    static __device__ __forceinline__ V add(V a, V b) { return a + b; }
    static __device__ __forceinline__ V sub(V a, V b) { return a - b; }
    static __device__ __forceinline__ V mul(V a, V b) { return a * b; }
    static __device__ __forceinline__ V det2(V p, V q, V r, V s) { return fmaf(p, q, -r * s); }
    static __device__ __forceinline__ V sgn(V a, float s) { return a * s; }
    static __device__ __forceinline__ V half(V a) { return 0.5f * a; }
    static __device__ __forceinline__ float sign_of(V a) { return a > 0.f ? 1.f : -1.f; }
    static __device__ __forceinline__ V from_double(double d) { return f_from_double(d); }
    static __device__ __forceinline__ V cst(double d) { return f_from_double(d); }
    static __device__ __forceinline__ A zero() { return {0.f, 0.f}; }
    static __device__ __forceinline__ void acc(A& a, V v) { dw_acc_f(a, v); }
    static __device__ __forceinline__ double out(A a, double sc) {
        dw s = dw_from_double(sc);
        return dw_to_double(dw_mulc(a, s.h, s.l));
    }
};

enum { DO_FWD = 1, DO_ADJ = 2 };

// NaN tests of staged values (staging turns every non-finite input into NaN)
__device__ __forceinline__ bool is_nan(double v) { return v != v; }
__device__ __forceinline__ bool is_nan(float v) { return v != v; }
__device__ __forceinline__ bool is_nan(dw v) { return v.h != v.h; }
__device__ __forceinline__ double qnan_d() { return __longlong_as_double(0x7ff8000000000000LL); }
// FP64 form: infinities become NaN too (the FP32-based forms' conversions
// already map every non-finite or out-of-range value to NaN)
__device__ __forceinline__ double finite_or_nan(double v) { return isfinite(v) ? v : qnan_d(); }
__device__ __forceinline__ float finite_or_nan(float v) { return v; }
__device__ __forceinline__ dw finite_or_nan(dw v) { return v; }

// The tile's coordinate origin, per component: the first owned node whose
// coordinate is finite (0 if none is), so that one non-finite coordinate does
// not reach the other staged nodes through the subtraction.
template <int DIM>
__device__ __forceinline__ void tile_origin(const double* x, int node0, int n_own, double* org) {
#pragma unroll
    for (int d = 0; d < DIM; d++) {
        double o = x[int64_t(node0) * DIM + d];
        for (int k = 1; !isfinite(o) && k < n_own; k++) o = x[(int64_t(node0) + k) * DIM + d];
        org[d] = isfinite(o) ? o : 0.0;
    }
}

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
    int val_e, val_v;          // largest edge / node valence of the grid
    int64_t tile_base;      // first tile handled by blockIdx.x == 0
    BwAux bwa;              // boundary-normal weights of the adjoint (bwa.bw NULL: none)
    int ahead;              // > 0: each tile prefetches tile t + ahead's inputs into L2
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

// ---------------------------------------------------------------------------
// scatter mode: every tile element adds its contributions to the tile's owned
// accumulators with shared-memory atomics on EXACT fixed-point integers.  A
// tile chooses, for each output kind, a power-of-two scale 2^sigma from the
// largest coordinate difference along its elements' edges (and the largest
// |w|, |c| it stages) and the grid's largest valences, such that no
// accumulated sum can reach 2^62 (2^41 for the FP32 form).  Each contribution
// is rounded once to a multiple of 2^-sigma and split into signed 21-bit
// limbs (units 2^42, 2^21, 1; the FP32 form uses the lower two), each summed
// with a native 32-bit integer atomic into its own shared-memory plane.  A
// limb plane holds up to 1023 contributions per entry without overflow, so
// no carries are propagated; the planes are recombined into one int64 at the
// end.  Integer sums do not depend on the order of the additions, so the
// results are bit-reproducible.
//
// The float -> limb split uses the classical "magic number" rounding on the
// FP32 pipe: adding 1.5*2^23 to a float t with |t| < 2^22 rounds it to an
// integer held in the low mantissa bits, and t - round(t) is exact.  (A
// float -> int64 conversion instruction would run on the FP64 pipe, which is
// 50x slower than the FP32 pipe on this GPU.)
// ---------------------------------------------------------------------------
struct Lq {
    int a, b, c;   // value = a*2^42 + b*2^21 + c (in units of 2^-sigma)
};

constexpr float FX_MAGIC = 12582912.0f;   // 1.5 * 2^23

__device__ __forceinline__ int fx_round(float t, float& rem) {
    const float y = __fadd_rn(t, FX_MAGIC);
    rem = __fsub_rn(t, __fsub_rn(y, FX_MAGIC));
    return __float_as_int(y) - 0x4B400000;
}

template <int NL>
__device__ __forceinline__ void acc_add(int* p, int stride, int i, const Lq& q) {
    atomicAdd(p + i, q.a);
    atomicAdd(p + stride + i, q.b);
    if (NL == 3) atomicAdd(p + 2 * stride + i, q.c);
}

template <int NL>
__device__ __forceinline__ long long acc_load(const int* p, int stride, int i) {
    if (NL == 3)
        return (long long)((unsigned long long)(long long)p[i] << 42) +
               (long long)((unsigned long long)(long long)p[stride + i] << 21) + (long long)p[2 * stride + i];
    return (long long)((unsigned long long)(long long)p[i] << 21) + (long long)p[stride + i];
}

// 2^k as float / double, k in the normal range
__device__ __forceinline__ float pow2f(int k) { return __uint_as_float((unsigned)(k + 127) << 23); }
__device__ __forceinline__ double pow2d(int k) {
    return __longlong_as_double((long long)((unsigned long long)(k + 1023) << 52));
}

__device__ __forceinline__ int sg_clamp(int sg, int lo, int hi) { return sg > hi ? hi : (sg < lo ? lo : sg); }

// Magnitudes as order-preserving 32-bit keys: the upper word of |v| as an
// IEEE double (exponent and 20 mantissa bits).  Non-negative doubles order
// like their bit patterns, so an integer max gives the max magnitude.  Every
// value with key k is below the double whose upper word is k + 1, and that
// double is below 2^key_exp(k).  Integer pipe only, and valid over the whole
// finite double range.  NaN and infinities get key 0, so they never enter a
// maximum: the scales bound the finite values, and the outputs that depend on
// a non-finite input are set to NaN separately (see the poison pass below).
// key_exp therefore only sees keys below 0x7ff00000 (exponents up to 1025).
__device__ __forceinline__ unsigned mkey(double v) {
    const unsigned k = (unsigned)((unsigned long long)__double_as_longlong(v) >> 32) & 0x7fffffffu;
    return k < 0x7ff00000u ? k : 0u;
}
__device__ __forceinline__ int key_exp(unsigned k) { return (int)(((k + 1u) >> 20) & 0x7ffu) - 1022; }


template <int PREC>
struct Fix;

template <>
struct Fix<EM_PREC_FP64> {
    static constexpr int NL = 3, TOP = 62, LO = -900, HI = 900;
    static __device__ __forceinline__ Lq q(double v, int sg) {
        const long long z = __double2ll_rn(__dmul_rn(v, pow2d(sg)));   // FP64 pipe: this form is FP64-bound anyway
        return {(int)(z >> 42), (int)((z >> 21) & 0x1fffff), (int)(z & 0x1fffff)};
    }
    static __device__ __forceinline__ unsigned mag(double v) { return mkey(v); }
    static __device__ __forceinline__ double out(long long q, int sg, double sc) {
        return __dmul_rn(__ll2double_rn(q), __dmul_rn(pow2d(-sg), sc));
    }
};

template <>
struct Fix<EM_PREC_DW> {
    // LO, HI: the float powers of two 2^(sg - 42) and 2^(sg - 21) below stay normal
    static constexpr int NL = 3, TOP = 62, LO = -80, HI = 148;
    static __device__ __forceinline__ Lq q(dw v, int sg) {
        float r;
        const float th = __fmul_rn(v.h, pow2f(sg - 42));
        const int a = fx_round(th, r);
        const int b = fx_round(__fmul_rn(r, 2097152.0f), r);
        const int c = fx_round(__fmul_rn(r, 2097152.0f), r);
        const float tl = __fmul_rn(v.l, pow2f(sg - 21));
        const int b2 = fx_round(tl, r);
        const int c2 = fx_round(__fmul_rn(r, 2097152.0f), r);
        return {a, b + b2, c + c2};
    }
    static __device__ __forceinline__ unsigned mag(dw v) {
        return mkey(f_to_double((fabsf(v.h) + fabsf(v.l)) * 1.000001f));
    }
    // once per output: the FP64 pipe is otherwise idle in this form
    static __device__ __forceinline__ double out(long long q, int sg, double sc) {
        return __dmul_rn(__ll2double_rn(q), __dmul_rn(pow2d(-sg), sc));
    }
};

template <>
struct Fix<EM_PREC_MIXED> {
    static constexpr int NL = 2, TOP = 41, LO = -80, HI = 148;
    static __device__ __forceinline__ Lq q(float v, int sg) {
        float r;
        const int a = fx_round(__fmul_rn(v, pow2f(sg - 21)), r);
        const int b = fx_round(__fmul_rn(r, 2097152.0f), r);
        return {a, b, 0};
    }
    static __device__ __forceinline__ unsigned mag(float v) { return mkey(f_to_double(v)); }
    static __device__ __forceinline__ double out(long long q, int sg, double sc) {
        return __dmul_rn(__ll2double_rn(q), __dmul_rn(pow2d(-sg), sc));
    }
};

// block-wide maxima without a cleared slot: each warp writes its maximum to
// its own entry of slot s (16 entries per slot), and readers take the max of
// the entries after a barrier
constexpr int RED_WARPS = 16;
__device__ __forceinline__ void block_max(unsigned* wred, int s, unsigned v) {
    v = __reduce_max_sync(0xffffffffu, v);
    if ((threadIdx.x & 31) == 0) wred[s * RED_WARPS + (threadIdx.x >> 5)] = v;
}
__device__ __forceinline__ unsigned red_max(const unsigned* wred, int s, int nwarps) {
    unsigned m = 0u;
    for (int w = 0; w < nwarps; w++) m = max(m, wred[s * RED_WARPS + w]);
    return m;
}

// ---- L2 prefetch of a later tile's inputs -----------------------------------
// Tiles are dispatched in index order, so while tile t computes, tile
// t + (resident CTAs) is about to start on some SM.  Used when one CTA fills an
// SM (no second CTA computes while the first stages).  One warp of tile t asks
// L2 for that tile's contiguous records (bulk prefetches of whole 16-byte
// blocks inside each range) and for the halo coordinates and weights it will
// gather, so its staging and element-record loads hit L2 instead of DRAM.
// Prefetches are hints: they move no data into the program's view and raise
// no errors for the valid addresses used here.
__device__ __forceinline__ void l2_prefetch_range(const void* p, long long bytes) {
    if (bytes <= 0) return;
    const unsigned long long b = (unsigned long long)__cvta_generic_to_global(p);
    unsigned long long a = (b + 15) & ~15ull;
    const unsigned long long e = (b + (unsigned long long)bytes) & ~15ull;
    while (a < e) {
        const unsigned n = (unsigned)(e - a < 65536ull ? e - a : 65536ull);
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a), "r"(n) : "memory");
        a += n;
    }
}

__device__ __forceinline__ void l2_prefetch_line(const void* p) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"((unsigned long long)__cvta_generic_to_global(p)));
}

template <int DIM, bool ADJ>
__device__ void prefetch_tile_l2(const TileArgs& A, int t2, int lane) {
    if (t2 >= A.n_tiles) return;
    const PlanHeader* H = static_cast<const PlanHeader*>(A.plan);
    const TileInfo ti = plan_at<TileInfo>(A.plan, H->off_tiles)[t2];
    const int32_t* halo = plan_at<int32_t>(A.plan, H->off_halo) + ti.halo_off;
    const int32_t* hedge = plan_at<int32_t>(A.plan, H->off_hedge) + ti.hedge_off;
    // contiguous ranges, one lane each
    switch (lane) {
        case 0: l2_prefetch_range(plan_at<ElemConn>(A.plan, H->off_conn) + ti.elem_off, (long long)sizeof(ElemConn) * ti.n_el); break;
        case 1:
            if (ADJ) l2_prefetch_range(plan_at<ElemEdges>(A.plan, H->off_tedge) + ti.elem_off, (long long)sizeof(ElemEdges) * ti.n_el);
            break;
        case 2: l2_prefetch_range(A.x + int64_t(ti.node0) * DIM, 8ll * DIM * ti.n_own); break;
        case 3:
            if (ADJ) l2_prefetch_range(A.w + int64_t(ti.edge0) * DIM, 8ll * DIM * ti.n_eo);
            break;
        case 4: l2_prefetch_range(halo, 4ll * ti.n_halo); break;
        case 5:
            if (ADJ) l2_prefetch_range(hedge, 4ll * ti.n_hedge);
            break;
        case 6:
            if (ADJ && A.c) l2_prefetch_range(A.c + ti.node0, 8ll * ti.n_own);
            break;
        case 7: l2_prefetch_range(plan_at<TileBFace>(A.plan, H->off_tbf) + ti.bf_off, (long long)sizeof(TileBFace) * ti.n_bf); break;
        case 8: l2_prefetch_range(A.bnode + ti.bnode0, 4ll * ti.n_bo); break;
        default: break;
    }
    // gathered rows: the index loads are issued 8 per lane before their prefetches
    constexpr int PB = 8;
    for (int i0 = lane; i0 < ti.n_halo; i0 += PB * 32) {
        int v[PB];
#pragma unroll
        for (int u = 0; u < PB; u++) v[u] = i0 + u * 32 < ti.n_halo ? halo[i0 + u * 32] : -1;
#pragma unroll
        for (int u = 0; u < PB; u++) {
            if (v[u] < 0) continue;
            l2_prefetch_line(A.x + int64_t(v[u]) * DIM);
            if (ADJ && A.c) l2_prefetch_line(A.c + v[u]);
        }
    }
    if (ADJ) {
        for (int i0 = lane; i0 < ti.n_hedge; i0 += PB * 32) {
            int e[PB];
#pragma unroll
            for (int u = 0; u < PB; u++) e[u] = i0 + u * 32 < ti.n_hedge ? hedge[i0 + u * 32] : -1;
#pragma unroll
            for (int u = 0; u < PB; u++)
                if (e[u] >= 0) l2_prefetch_line(A.w + int64_t(e[u]) * DIM);
        }
    }
}

struct SmemS {
    size_t xs, ws, cs, acc_e, acc_v, acc_g, acc_b, bmap, red, total;
};

template <int DIM, int PREC, int WHAT>
__host__ __device__ inline SmemS smem_layout_s(const Dims& D) {
    using F = Form<PREC>;
    SmemS s;
    size_t o = 0;
    auto take = [&](size_t bytes) { o = (o + 15) & ~size_t(15); size_t r = o; o += bytes; return r; };
    const size_t wb = Fix<PREC>::NL * sizeof(int);
    s.xs = take(sizeof(typename F::C) * DIM * D.max_nodes);
    s.ws = (WHAT & DO_ADJ) ? take(sizeof(typename F::V) * DIM * D.max_edges) : 0;
    s.cs = (WHAT & DO_ADJ) ? take(sizeof(typename F::V) * D.max_nodes) : 0;
    s.acc_e = (WHAT & DO_FWD) ? take(wb * DIM * D.max_eo) : 0;
    s.acc_v = (WHAT & DO_FWD) ? take(wb * D.max_own) : 0;
    s.acc_g = (WHAT & DO_ADJ) ? take(wb * DIM * D.max_own) : 0;
    s.acc_b = (WHAT & DO_FWD) ? take(wb * DIM * D.max_bo) : 0;
    s.bmap = take(sizeof(int) * D.max_own);
    s.red = take(sizeof(unsigned) * (16 + 5 * RED_WARPS));
    s.total = (o + 15) & ~size_t(15);
    return s;
}

// pf(lane) is called by the last warp once the tile's staging is done: it may
// prefetch a later tile's inputs into L2 while the other warps compute
template <int DIM, int PREC, int WHAT, int NTH, class PF>
__device__ __forceinline__ void run_tile_scatter(const TileArgs& A, int t, char* smem, const PF& pf) {
    using F = Form<PREC>;
    using FX = Fix<PREC>;
    using C = typename F::C;
    using V = typename F::V;
    const PlanHeader* H = static_cast<const PlanHeader*>(A.plan);
    const TileInfo ti = plan_at<TileInfo>(A.plan, H->off_tiles)[t];
    const ElemConn* conn = plan_at<ElemConn>(A.plan, H->off_conn) + ti.elem_off;
    const ElemEdges* tedge = plan_at<ElemEdges>(A.plan, H->off_tedge) + ti.elem_off;
    const int32_t* halo = plan_at<int32_t>(A.plan, H->off_halo) + ti.halo_off;
    const int32_t* hedge = plan_at<int32_t>(A.plan, H->off_hedge) + ti.hedge_off;
    const TileBFace* tbf = plan_at<TileBFace>(A.plan, H->off_tbf) + ti.bf_off;

    const SmemS L = smem_layout_s<DIM, PREC, WHAT>(A.D);
    C* xs = reinterpret_cast<C*>(smem + L.xs);
    V* ws = reinterpret_cast<V*>(smem + L.ws);
    V* cs = reinterpret_cast<V*>(smem + L.cs);
    constexpr int NL = FX::NL;
    int* acc_e = reinterpret_cast<int*>(smem + L.acc_e);
    int* acc_v = reinterpret_cast<int*>(smem + L.acc_v);
    int* acc_g = reinterpret_cast<int*>(smem + L.acc_g);
    int* acc_b = reinterpret_cast<int*>(smem + L.acc_b);
    const int se = DIM * A.D.max_eo, sv = A.D.max_own, sgs = DIM * A.D.max_own, sb = DIM * A.D.max_bo;
    int* bmap = reinterpret_cast<int*>(smem + L.bmap);
    unsigned* red = reinterpret_cast<unsigned*>(smem + L.red);
    unsigned* wred = red + 16;
    static_assert(NTH / 32 <= RED_WARPS, "one maximum slot per warp");

    const int tid = threadIdx.x;
    const int nnodes = ti.n_own + ti.n_halo;

    // ---- clear accumulators --------------------------------------------------
    if (tid < 16) red[tid] = 0u;
    if (WHAT & DO_FWD) {
        for (int q = tid; q < NL * se; q += NTH) acc_e[q] = 0;
        for (int q = tid; q < NL * sv; q += NTH) acc_v[q] = 0;
        for (int q = tid; q < NL * sb; q += NTH) acc_b[q] = 0;
    }
    if (WHAT & DO_ADJ)
        for (int q = tid; q < NL * sgs; q += NTH) acc_g[q] = 0;
    for (int i = tid; i < ti.n_own; i += NTH) bmap[i] = -1;
    // (no barrier: the cleared planes are first used after the staging and
    // extent barriers below, and the boundary-node map is filled after them)

    // 512-thread tiles (one CTA per SM, nothing hides their latency): this
    // thread's first element records of the extent pass below are requested
    // now, so that they arrive while the staging gathers are in flight (the
    // 256-thread forms have no registers to spare for them)
    constexpr int EB = 8;
    constexpr bool HOIST = NTH > NT;
    ElemConn ecb[HOIST ? EB : 1];
    if constexpr (HOIST) {
#pragma unroll
        for (int u = 0; u < EB; u++)
            if (tid + u * NTH < ti.n_el) ecb[u] = conn[tid + u * NTH];
    }

    // ---- stage coordinates (and w, c) and find the tile's magnitudes --------
    double org[DIM];
    tile_origin<DIM>(A.x, ti.node0, ti.n_own, org);
    // gathers are issued in batches of SB per thread so that several loads are
    // in flight before the first one is used
    constexpr int SB = 4, SBW = 8;
    unsigned wm = 0u, cm = 0u;
    float xl = 0.f;      // DW / MIXED forms: largest |low part| of a staged coordinate
    bool nf = false;     // a staged value is non-finite (staged as NaN)
    for (int i0 = tid; i0 < nnodes; i0 += SB * NTH) {
        int64_t v[SB];
#pragma unroll
        for (int u = 0; u < SB; u++) {
            const int i = i0 + u * NTH;
            v[u] = i >= nnodes ? -1 : (i < ti.n_own ? int64_t(ti.node0) + i : int64_t(halo[i - ti.n_own]));
        }
        double xv[SB][DIM], cv[SB];
#pragma unroll
        for (int u = 0; u < SB; u++) {
            if (v[u] < 0) continue;
#pragma unroll
            for (int d = 0; d < DIM; d++) xv[u][d] = A.x[v[u] * DIM + d];
            if (WHAT & DO_ADJ) cv[u] = A.c ? A.c[v[u]] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < SB; u++) {
            if (v[u] < 0) continue;
            const int i = i0 + u * NTH;
#pragma unroll
            for (int d = 0; d < DIM; d++) {
                const C xc = finite_or_nan(F::coord(xv[u][d], org[d]));
                xs[i * DIM + d] = xc;
                nf |= is_nan(xc);
                if constexpr (PREC != EM_PREC_FP64) xl = fmaxf(xl, fabsf(xc.l));
            }
            if (WHAT & DO_ADJ) {
                const V c1 = finite_or_nan(F::from_double(cv[u]));
                cs[i] = c1;
                nf |= is_nan(c1);
                cm = max(cm, FX::mag(c1));
            }
        }
    }
    if (WHAT & DO_ADJ) {
        const int nte = ti.n_eo + ti.n_hedge;
        for (int i0 = tid; i0 < nte; i0 += SBW * NTH) {
            int64_t e[SBW];
#pragma unroll
            for (int u = 0; u < SBW; u++) {
                const int i = i0 + u * NTH;
                e[u] = i >= nte ? -1 : (i < ti.n_eo ? int64_t(ti.edge0) + i : int64_t(hedge[i - ti.n_eo]));
            }
            double wv[SBW][DIM];
#pragma unroll
            for (int u = 0; u < SBW; u++)
                if (e[u] >= 0)
#pragma unroll
                    for (int d = 0; d < DIM; d++) wv[u][d] = A.w[e[u] * DIM + d];
#pragma unroll
            for (int u = 0; u < SBW; u++) {
                if (e[u] < 0) continue;
                const int i = i0 + u * NTH;
#pragma unroll
                for (int d = 0; d < DIM; d++) {
                    const V w1 = finite_or_nan(F::from_double(wv[u][d]));
                    ws[i * DIM + d] = w1;
                    nf |= is_nan(w1);
                    wm = max(wm, FX::mag(w1));
                }
            }
        }
    }
    if (WHAT & DO_ADJ) {
        block_max(wred, 1, wm);
        block_max(wred, 2, cm);
    }
    if constexpr (PREC != EM_PREC_FP64) block_max(wred, 3, mkey(f_to_double(xl)));
    block_max(wred, 4, nf ? 1u : 0u);
    __syncthreads();
    for (int k = tid; k < ti.n_bo; k += NTH) bmap[A.bnode[ti.bnode0 + k] - ti.node0] = k;

    // ---- element extent: Lx bounds every coordinate difference along an edge
    // from local node 0 of a tile element; every face vector, volume and
    // gradient term below is bounded by a power of Lx (edges not at node 0 and
    // boundary-face edges by 2 Lx), so the scales follow the element size, not
    // the extent of the tile.  The element records are loaded EB at a time so
    // that their loads are in flight together.
    {
        unsigned lk = 0u;
        float lf = 0.f;
        for (int i0 = tid; i0 < ti.n_el; i0 += EB * NTH) {
            ElemConn cb[EB];
#pragma unroll
            for (int u = 0; u < EB; u++)
                if (i0 + u * NTH < ti.n_el) cb[u] = (HOIST && i0 == tid) ? ecb[HOIST ? u : 0] : conn[i0 + u * NTH];
#pragma unroll
            for (int u = 0; u < EB; u++) {
                if (i0 + u * NTH >= ti.n_el) continue;
#pragma unroll
                for (int r = 1; r <= DIM; r++)
#pragma unroll
                    for (int d = 0; d < DIM; d++) {
                        if constexpr (PREC == EM_PREC_FP64)
                            lk = max(lk, mkey(xs[cb[u].v[r] * DIM + d] - xs[cb[u].v[0] * DIM + d]));
                        else
                            lf = fmaxf(lf, fabsf(__fsub_rn(xs[cb[u].v[r] * DIM + d].h, xs[cb[u].v[0] * DIM + d].h)));
                    }
            }
        }
        // DW / MIXED: |a - b| <= |a.h - b.h| (1 + 2^-23) + 2 max|low part|
        block_max(wred, 0, PREC == EM_PREC_FP64 ? lk : mkey(f_to_double(lf)));
    }
    __syncthreads();

    // ---- scales: no accumulated sum can reach 2^TOP -------------------------
    // Each bound is a product (or a sum of three products) of factors with
    // power-of-two upper bounds, so its exponent is a sum of exponents: every
    // thread derives the same scales with integer arithmetic, with no FP64
    // instruction and no further barrier.  (Rounding each factor up to a power
    // of two gives away at most a few of the 62 bits.)
    constexpr int TP = FX::TOP, LO = FX::LO, HI = FX::HI;
    // DW / MIXED: Lx <= b0 (1 + 2^-20) + 2 b3 < 2^(max(E0, E3) + 2), with b0 < 2^E0
    // bounding the high-part extent (slot 0) and b3 < 2^E3 the low parts (slot 3)
    constexpr int NW = NTH / 32;
    const int eL = PREC == EM_PREC_FP64 ? key_exp(red_max(wred, 0, NW))
                                        : max(key_exp(red_max(wred, 0, NW)), key_exp(red_max(wred, 3, NW))) + 2;
    const int eKe = 32 - __clz(A.val_e > 1 ? A.val_e : 1), eKv = 32 - __clz(A.val_v > 1 ? A.val_v : 1);
    int eg = 0;
    if (WHAT & DO_ADJ) {
        // |w|, |c|, |bw| < 2^Ew, 2^Ec, 2^Eb
        const int Ew = key_exp(red_max(wred, 1, NW)), Ec = key_exp(red_max(wred, 2, NW));
        const int Eb = A.bwa.bw ? key_exp(*A.bwa.key) : -2000;
        if (DIM == 3)   // (16 |w| Lx + 8 |c| Lx^2 + 16 |bw| Lx) 2 Kv
            eg = max(max(4 + Ew + eL, 3 + Ec + 2 * eL), 4 + Eb + eL) + 2 + 1 + eKv;
        else            // (4 |w| + 4 |c| Lx + 4 |bw|) 2 Kv
            eg = max(max(2 + Ew, 2 + Ec + eL), 2 + Eb) + 2 + 1 + eKv;
    }
    // 3D: |N_i| components <= 2 Lx^2, |det| <= 3 sqrt(3) Lx^3 < 8 Lx^3,
    // |n_B| <= 8 Lx^2 with up to 3 boundary faces per element at a node;
    // 2D: |n_i| <= 2 Lx, |det| <= 2 Lx^2, boundary edge <= 2 Lx
    const int u_e = TP - (DIM == 3 ? 5 + 2 * eL + eKe : 3 + eL + eKe);
    const int u_v = TP - (DIM == 3 ? 3 + 3 * eL + eKv : 4 + 2 * eL + eKv);
    const int u_b = TP - (DIM == 3 ? 5 + 2 * eL + eKv : 3 + eL + eKv);
    const int sg_e = sg_clamp(u_e, LO, HI), sg_v = sg_clamp(u_v, LO, HI), sg_b = sg_clamp(u_b, LO, HI);
    const int sg_g = (WHAT & DO_ADJ) ? sg_clamp(TP - eg, LO, HI) : 0;
    // Element extents outside the form's range (a scale outside [LO, HI]:
    // the values would overflow the fixed point, or lose the digits the
    // contract needs) make every output of the tile NaN instead of silently
    // wrong; for the FP32-based forms that is an element extent outside about
    // 2^-34 .. 2^40, for the FP64 form outside about 2^-290 .. 2^290.  A tile
    // whose elements all have zero extent contributes exact zeros at any scale.
    // Non-finite staged values mark the tile for the poison pass below.
    const bool lx0 = red_max(wred, 0, NW) == 0u;
    const bool range_bad = (!lx0 && (u_e < LO || u_e > HI || u_v < LO || u_v > HI || u_b < LO || u_b > HI)) ||
                           ((WHAT & DO_ADJ) && TP - eg < LO);
    const bool nf_tile = red_max(wred, 4, NW) != 0u;
    if ((tid >> 5) == (NTH >> 5) - 1) pf(tid & 31);

    // ---- elements: compute and scatter to owned targets -------------------
    // warps take chunks of 32 consecutive elements from a shared counter (the
    // elements are grouped by owned mask, so work per chunk varies); the next
    // chunk's records are loaded while the current one is computed
    const int lane = tid & 31;
    unsigned* chunk_ctr = red + 8;
    auto grab = [&]() {
        int b = 0;
        if (lane == 0) b = (int)atomicAdd(chunk_ctr, 32u);
        return __shfl_sync(0xffffffffu, b, 0);
    };
    int cur = grab();
    ElemConn cn_nx{};
    ElemEdges ee_nx{};
    if (cur + lane < ti.n_el) {
        cn_nx = conn[cur + lane];
        ee_nx = tedge[cur + lane];
    }
    while (cur < ti.n_el) {
        const int nxt = grab();
        const int i = cur + lane;
        const ElemConn cn = cn_nx;
        const ElemEdges ee = ee_nx;
        if (nxt + lane < ti.n_el) {
            cn_nx = conn[nxt + lane];
            ee_nx = tedge[nxt + lane];
        }
        cur = nxt;
        if (i >= ti.n_el) continue;
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
            // ownership of the sorted nodes; edges are owned by their lower end,
            // so edges (0,1),(0,2),(0,3) are owned iff node 0 is, (1,2),(1,3)
            // iff node 1 is, (2,3) iff node 2 is.  Tile elements are grouped by
            // this mask, so the branches below are warp-uniform almost always.
            const bool o0 = cn.v[0] < ti.n_own, o1 = cn.v[1] < ti.n_own, o2 = cn.v[2] < ti.n_own,
                       o3 = cn.v[3] < ti.n_own;
            if (WHAT & DO_FWD) {
                // edges (0,1),(0,2),(0,3) <- m0; (1,2),(1,3) <- m1; (2,3) <- m2.
                // An edge is owned exactly when its lower end is, and owned
                // edges have local ids below n_eo (plan invariant).
                if (o0) {
#pragma unroll
                    for (int d = 0; d < 3; d++) {
                        const Lq q0 = FX::q(F::sgn(F::add(F::add(N1[d], N2[d]), N3[d]), s), sg_e);
                        acc_add<NL>(acc_e, se, ee.e[0] * 3 + d, q0);
                        acc_add<NL>(acc_e, se, ee.e[1] * 3 + d, q0);
                        acc_add<NL>(acc_e, se, ee.e[2] * 3 + d, q0);
                    }
                }
                if (o1) {
#pragma unroll
                    for (int d = 0; d < 3; d++) {
                        const Lq q1 = FX::q(F::sgn(N1[d], -s), sg_e);
                        acc_add<NL>(acc_e, se, ee.e[3] * 3 + d, q1);
                        acc_add<NL>(acc_e, se, ee.e[4] * 3 + d, q1);
                    }
                }
                if (o2) {
#pragma unroll
                    for (int d = 0; d < 3; d++) acc_add<NL>(acc_e, se, ee.e[5] * 3 + d, FX::q(F::sgn(N2[d], -s), sg_e));
                }
                const Lq qv = FX::q(F::sgn(det, s), sg_v);
                if (o0) acc_add<NL>(acc_v, sv, cn.v[0], qv);
                if (o1) acc_add<NL>(acc_v, sv, cn.v[1], qv);
                if (o2) acc_add<NL>(acc_v, sv, cn.v[2], qv);
                if (o3) acc_add<NL>(acc_v, sv, cn.v[3], qv);
            }
            if (WHAT & DO_ADJ) {
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
                // g_k = -s/12 (A_{k+1} x X_{k+2} - A_{k+2} x X_{k+1}) + h N_k for
                // k = 1, 2, 3 (indices cyclic, X = (a, b, c)): one loop body with
                // the operand vectors rotated by one position per iteration; g_k
                // is needed for owned node k, and all three for node 0
                V Ar[3][3], Xr[3][3], Nr[3][3];
#pragma unroll
                for (int d = 0; d < 3; d++) {
                    Ar[0][d] = A1[d]; Ar[1][d] = A2[d]; Ar[2][d] = A3[d];
                    Xr[0][d] = a[d]; Xr[1][d] = b[d]; Xr[2][d] = c[d];
                    Nr[0][d] = N1[d]; Nr[1][d] = N2[d]; Nr[2][d] = N3[d];
                }
                int vr0 = cn.v[1], vr1 = cn.v[2], vr2 = cn.v[3];
                V gs[3] = {F::cst(0.0), F::cst(0.0), F::cst(0.0)};
#pragma unroll 1
                for (int k = 0; k < 3; k++) {
                    const bool own = vr0 < ti.n_own;
                    if (o0 || own) {
                        V gk[3];
#pragma unroll
                        for (int d = 0; d < 3; d++) {
                            const int d1 = (d + 1) % 3, d2 = (d + 2) % 3;
                            V g = F::sub(F::det2(Ar[1][d1], Xr[2][d2], Ar[1][d2], Xr[2][d1]),
                                         F::det2(Ar[2][d1], Xr[1][d2], Ar[2][d2], Xr[1][d1]));
                            gk[d] = F::add(F::sgn(F::mul(g, f12), s), F::mul(h, Nr[0][d]));
                        }
                        if (own) {
#pragma unroll
                            for (int d = 0; d < 3; d++) acc_add<NL>(acc_g, sgs, vr0 * 3 + d, FX::q(gk[d], sg_g));
                        }
                        if (o0) {
#pragma unroll
                            for (int d = 0; d < 3; d++) gs[d] = F::add(gs[d], gk[d]);
                        }
                    }
                    // rotate: position 0 takes the next k
#pragma unroll
                    for (int d = 0; d < 3; d++) {
                        V t0 = Ar[0][d]; Ar[0][d] = Ar[1][d]; Ar[1][d] = Ar[2][d]; Ar[2][d] = t0;
                        V t1 = Xr[0][d]; Xr[0][d] = Xr[1][d]; Xr[1][d] = Xr[2][d]; Xr[2][d] = t1;
                        V t2 = Nr[0][d]; Nr[0][d] = Nr[1][d]; Nr[1][d] = Nr[2][d]; Nr[2][d] = t2;
                    }
                    const int tv = vr0; vr0 = vr1; vr1 = vr2; vr2 = tv;
                }
                if (o0) {
#pragma unroll
                    for (int d = 0; d < 3; d++) acc_add<NL>(acc_g, sgs, cn.v[0] * 3 + d, FX::q(F::sgn(gs[d], -1.f), sg_g));
                }
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
            // edges (0,1),(0,2) are owned iff node 0 is, (1,2) iff node 1 is
            const bool o0 = cn.v[0] < ti.n_own, o1 = cn.v[1] < ti.n_own, o2 = cn.v[2] < ti.n_own;
            if (WHAT & DO_FWD) {
                V n1[2] = {F::sgn(b[1], -s), F::sgn(b[0], s)};
                V n2[2] = {F::sgn(a[1], s), F::sgn(a[0], -s)};
                if (o0) {
#pragma unroll
                    for (int d = 0; d < 2; d++) {
                        const Lq q0 = FX::q(F::sgn(F::add(n1[d], n2[d]), -1.f), sg_e);
                        acc_add<NL>(acc_e, se, ee.e[0] * 2 + d, q0);
                        acc_add<NL>(acc_e, se, ee.e[1] * 2 + d, q0);
                    }
                }
                if (o1) {
#pragma unroll
                    for (int d = 0; d < 2; d++) acc_add<NL>(acc_e, se, ee.e[2] * 2 + d, FX::q(n1[d], sg_e));
                }
                const Lq qv = FX::q(F::sgn(det, s), sg_v);
                if (o0) acc_add<NL>(acc_v, sv, cn.v[0], qv);
                if (o1) acc_add<NL>(acc_v, sv, cn.v[1], qv);
                if (o2) acc_add<NL>(acc_v, sv, cn.v[2], qv);
            }
            if (WHAT & DO_ADJ) {
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
                V gax = F::cst(0.0), gay = F::cst(0.0), gbx = F::cst(0.0), gby = F::cst(0.0);
                if (o0 || o1) {
                    gax = F::add(F::sgn(F::mul(A2[1], f3), -s), F::mul(h, b[1]));
                    gay = F::add(F::sgn(F::mul(A2[0], f3), s), F::sgn(F::mul(h, b[0]), -1.f));
                }
                if (o0 || o2) {
                    gbx = F::add(F::sgn(F::mul(A1[1], f3), s), F::sgn(F::mul(h, a[1]), -1.f));
                    gby = F::add(F::sgn(F::mul(A1[0], f3), -s), F::mul(h, a[0]));
                }
                if (o1) {
                    acc_add<NL>(acc_g, sgs, cn.v[1] * 2, FX::q(gax, sg_g));
                    acc_add<NL>(acc_g, sgs, cn.v[1] * 2 + 1, FX::q(gay, sg_g));
                }
                if (o2) {
                    acc_add<NL>(acc_g, sgs, cn.v[2] * 2, FX::q(gbx, sg_g));
                    acc_add<NL>(acc_g, sgs, cn.v[2] * 2 + 1, FX::q(gby, sg_g));
                }
                if (o0) {
                    acc_add<NL>(acc_g, sgs, cn.v[0] * 2, FX::q(F::sgn(F::add(gax, gbx), -1.f), sg_g));
                    acc_add<NL>(acc_g, sgs, cn.v[0] * 2 + 1, FX::q(F::sgn(F::add(gay, gby), -1.f), sg_g));
                }
            }
        }
    }

    // ---- boundary faces ------------------------------------------------------
    for (int j = tid; j < ti.n_bf; j += NTH) {
        const TileBFace f = tbf[j];
        if (DIM == 3) {
            V u[3], tt[3];
#pragma unroll
            for (int d = 0; d < 3; d++) {
                u[d] = F::diff(xs[f.v[1] * 3 + d], xs[f.v[0] * 3 + d]);
                tt[d] = F::diff(xs[f.v[2] * 3 + d], xs[f.v[0] * 3 + d]);
            }
            if (WHAT & DO_FWD) {
                V nB[3] = {F::half(F::det2(u[1], tt[2], u[2], tt[1])), F::half(F::det2(u[2], tt[0], u[0], tt[2])),
                           F::half(F::det2(u[0], tt[1], u[1], tt[0]))};
#pragma unroll
                for (int d = 0; d < 3; d++) {
                    const Lq qe = FX::q(nB[d], sg_e), qb = FX::q(nB[d], sg_b);
#pragma unroll
                    for (int k = 0; k < 3; k++)
                        if (f.e[k] < ti.n_eo) acc_add<NL>(acc_e, se, f.e[k] * 3 + d, qe);
#pragma unroll
                    for (int k = 0; k < 3; k++)
                        if (f.v[k] < ti.n_own && bmap[f.v[k]] >= 0) acc_add<NL>(acc_b, sb, bmap[f.v[k]] * 3 + d, qb);
                }
            }
            if (WHAT & DO_ADJ) {
                V WB[3];
#pragma unroll
                for (int d = 0; d < 3; d++)
                    WB[d] = F::add(F::add(ws[f.e[0] * 3 + d], ws[f.e[1] * 3 + d]), ws[f.e[2] * 3 + d]);
                const V f24 = F::cst(1.0 / 24.0);
                // boundary-normal weights: K = 1/3 sum of bw at the face's nodes
                V K[3];
                const bool hasK = A.bwa.bw != nullptr;
                if (hasK) {
                    double Kd[3] = {0.0, 0.0, 0.0};
#pragma unroll
                    for (int k = 0; k < 3; k++) {
                        const int lv = f.v[k];
                        const int64_t gv = lv < ti.n_own ? int64_t(ti.node0) + lv : int64_t(halo[lv - ti.n_own]);
                        const int64_t b = A.bwa.map[gv];
#pragma unroll
                        for (int d = 0; d < 3; d++) Kd[d] += A.bwa.bw[3 * b + d];
                    }
#pragma unroll
                    for (int d = 0; d < 3; d++) K[d] = F::from_double(Kd[d] / 3.0);
                    if (!(isfinite(Kd[0]) && isfinite(Kd[1]) && isfinite(Kd[2]))) atomicOr(red + 11, 1u);
                }
#pragma unroll
                for (int d = 0; d < 3; d++) {
                    const int d1 = (d + 1) % 3, d2 = (d + 2) % 3;
                    V gq = F::mul(F::det2(tt[d1], WB[d2], tt[d2], WB[d1]), f24);
                    V gr = F::mul(F::det2(WB[d1], u[d2], WB[d2], u[d1]), f24);
                    if (hasK) {
                        gq = F::add(gq, F::half(F::det2(tt[d1], K[d2], tt[d2], K[d1])));
                        gr = F::add(gr, F::half(F::det2(K[d1], u[d2], K[d2], u[d1])));
                    }
                    if (f.v[1] < ti.n_own) acc_add<NL>(acc_g, sgs, f.v[1] * 3 + d, FX::q(gq, sg_g));
                    if (f.v[2] < ti.n_own) acc_add<NL>(acc_g, sgs, f.v[2] * 3 + d, FX::q(gr, sg_g));
                    if (f.v[0] < ti.n_own) acc_add<NL>(acc_g, sgs, f.v[0] * 3 + d, FX::q(F::sgn(F::add(gq, gr), -1.f), sg_g));
                }
            }
        } else {
            if (WHAT & DO_FWD) {
                V nB[2] = {F::diff(xs[f.v[0] * 2 + 1], xs[f.v[1] * 2 + 1]), F::diff(xs[f.v[1] * 2 + 0], xs[f.v[0] * 2 + 0])};
#pragma unroll
                for (int d = 0; d < 2; d++) {
                    if (f.e[0] < ti.n_eo) acc_add<NL>(acc_e, se, f.e[0] * 2 + d, FX::q(F::half(nB[d]), sg_e));
                    const Lq qb = FX::q(nB[d], sg_b);
#pragma unroll
                    for (int k = 0; k < 2; k++)
                        if (f.v[k] < ti.n_own && bmap[f.v[k]] >= 0) acc_add<NL>(acc_b, sb, bmap[f.v[k]] * 2 + d, qb);
                }
            }
            if (WHAT & DO_ADJ) {
                const V f6 = F::cst(1.0 / 6.0);
                V gx = F::mul(ws[f.e[0] * 2 + 1], f6);
                V gy = F::sgn(F::mul(ws[f.e[0] * 2 + 0], f6), -1.f);
                if (A.bwa.bw) {   // boundary-normal weights: K = 1/2 (bw_a + bw_b)
                    double Kd[2] = {0.0, 0.0};
#pragma unroll
                    for (int k = 0; k < 2; k++) {
                        const int lv = f.v[k];
                        const int64_t gv = lv < ti.n_own ? int64_t(ti.node0) + lv : int64_t(halo[lv - ti.n_own]);
                        const int64_t b = A.bwa.map[gv];
                        Kd[0] += A.bwa.bw[2 * b];
                        Kd[1] += A.bwa.bw[2 * b + 1];
                    }
                    gx = F::add(gx, F::from_double(0.5 * Kd[1]));
                    gy = F::add(gy, F::from_double(-0.5 * Kd[0]));
                    if (!(isfinite(Kd[0]) && isfinite(Kd[1]))) atomicOr(red + 11, 1u);
                }
                if (f.v[1] < ti.n_own) {
                    acc_add<NL>(acc_g, sgs, f.v[1] * 2, FX::q(gx, sg_g));
                    acc_add<NL>(acc_g, sgs, f.v[1] * 2 + 1, FX::q(gy, sg_g));
                }
                if (f.v[0] < ti.n_own) {
                    acc_add<NL>(acc_g, sgs, f.v[0] * 2, FX::q(F::sgn(gx, -1.f), sg_g));
                    acc_add<NL>(acc_g, sgs, f.v[0] * 2 + 1, FX::q(F::sgn(gy, -1.f), sg_g));
                }
            }
        }
    }
    __syncthreads();

    // ---- non-finite inputs (rare; tile-uniform branch) -----------------------
    // Every output to which an element or boundary face with a non-finite
    // input contributes is NaN: forward outputs (n, V, bnormal) from the
    // coordinates, gradients from the coordinates, w, c and the boundary-normal
    // weights.  Such contributions went into the integer sums as arbitrary
    // values (the scales above bound the finite ones only); their targets are
    // marked with a first-limb value no sum can reach (|limb sums| < 2^31 by
    // the headroom argument above) and written as NaN.
    constexpr int MARK = -2147483647 - 1;
    const bool poison = nf_tile || (red[11] != 0u);
    if (poison && !range_bad) {
        constexpr int NLE = DIM == 3 ? 6 : 3;
        for (int i = tid; i < ti.n_el; i += NTH) {
            const ElemConn cn = conn[i];
            const ElemEdges ee = tedge[i];
            bool px = false, pa = false;
#pragma unroll
            for (int r = 0; r <= DIM; r++)
#pragma unroll
                for (int d = 0; d < DIM; d++) px |= is_nan(xs[cn.v[r] * DIM + d]);
            if (WHAT & DO_ADJ) {
#pragma unroll
                for (int l = 0; l < NLE; l++)
#pragma unroll
                    for (int d = 0; d < DIM; d++) pa |= is_nan(ws[ee.e[l] * DIM + d]);
#pragma unroll
                for (int r = 0; r <= DIM; r++) pa |= is_nan(cs[cn.v[r]]);
            }
            pa |= px;
            if ((WHAT & DO_FWD) && px) {
#pragma unroll
                for (int l = 0; l < NLE; l++)
                    if (ee.e[l] < ti.n_eo)
#pragma unroll
                        for (int d = 0; d < DIM; d++) acc_e[ee.e[l] * DIM + d] = MARK;
#pragma unroll
                for (int r = 0; r <= DIM; r++)
                    if (cn.v[r] < ti.n_own) acc_v[cn.v[r]] = MARK;
            }
            if ((WHAT & DO_ADJ) && pa) {
#pragma unroll
                for (int r = 0; r <= DIM; r++)
                    if (cn.v[r] < ti.n_own)
#pragma unroll
                        for (int d = 0; d < DIM; d++) acc_g[cn.v[r] * DIM + d] = MARK;
            }
        }
        for (int j = tid; j < ti.n_bf; j += NTH) {
            const TileBFace f = tbf[j];
            constexpr int FE = DIM == 3 ? 3 : 1;
            bool px = false, pa = false;
#pragma unroll
            for (int k = 0; k < DIM; k++)
#pragma unroll
                for (int d = 0; d < DIM; d++) px |= is_nan(xs[f.v[k] * DIM + d]);
            if (WHAT & DO_ADJ) {
#pragma unroll
                for (int k = 0; k < FE; k++)
#pragma unroll
                    for (int d = 0; d < DIM; d++) pa |= is_nan(ws[f.e[k] * DIM + d]);
                if (A.bwa.bw) {
#pragma unroll
                    for (int k = 0; k < DIM; k++) {
                        const int lv = f.v[k];
                        const int64_t gv = lv < ti.n_own ? int64_t(ti.node0) + lv : int64_t(halo[lv - ti.n_own]);
                        const int64_t b = A.bwa.map[gv];
#pragma unroll
                        for (int d = 0; d < DIM; d++) pa |= !isfinite(A.bwa.bw[DIM * b + d]);
                    }
                }
            }
            pa |= px;
            if ((WHAT & DO_FWD) && px) {
#pragma unroll
                for (int k = 0; k < FE; k++)
                    if (f.e[k] < ti.n_eo)
#pragma unroll
                        for (int d = 0; d < DIM; d++) acc_e[f.e[k] * DIM + d] = MARK;
#pragma unroll
                for (int k = 0; k < DIM; k++)
                    if (f.v[k] < ti.n_own && bmap[f.v[k]] >= 0)
#pragma unroll
                        for (int d = 0; d < DIM; d++) acc_b[bmap[f.v[k]] * DIM + d] = MARK;
            }
            if ((WHAT & DO_ADJ) && pa) {
#pragma unroll
                for (int k = 0; k < DIM; k++)
                    if (f.v[k] < ti.n_own)
#pragma unroll
                        for (int d = 0; d < DIM; d++) acc_g[f.v[k] * DIM + d] = MARK;
            }
        }
        __syncthreads();
    }

    const double esc = DIM == 3 ? 1.0 / 12.0 : 1.0 / 3.0;
    const double vsc = DIM == 3 ? 1.0 / 24.0 : 1.0 / 6.0;
    const double bsc = DIM == 3 ? 1.0 / 3.0 : 1.0 / 2.0;
    // out(p, q): output q of the planes p at scale sg, NaN where marked
    auto outv = [&](const int* p, int stride, int q, int sg, double sc) {
        if (range_bad || (poison && p[q] == MARK)) return qnan_d();
        return FX::out(acc_load<NL>(p, stride, q), sg, sc);
    };
    if (WHAT & DO_FWD) {
        for (int q = tid; q < ti.n_eo * DIM; q += NTH) A.n_out[int64_t(ti.edge0) * DIM + q] = outv(acc_e, se, q, sg_e, esc);
        for (int q = tid; q < ti.n_bo * DIM; q += NTH) A.bnormal[int64_t(ti.bnode0) * DIM + q] = outv(acc_b, sb, q, sg_b, bsc);
        for (int q = tid; q < ti.n_own; q += NTH) A.vol[int64_t(ti.node0) + q] = outv(acc_v, sv, q, sg_v, vsc);
    }
    if (WHAT & DO_ADJ)
        for (int q = tid; q < ti.n_own * DIM; q += NTH) A.grad[int64_t(ti.node0) * DIM + q] = outv(acc_g, sgs, q, sg_g, 1.0);
}

// resident CTAs per SM the register allocation must allow: the forward alone
// and the FP32 form need little shared memory and fit three CTAs, the other
// adjoint-carrying forms fit two
template <int PREC, int WHAT>
constexpr int scatter_min_ctas() { return (PREC == EM_PREC_MIXED || WHAT == DO_FWD) ? 3 : 2; }

// NTH = 2 NT for tiles so large that one CTA fills an SM's shared memory:
// the register file then still holds 16 warps per SM
template <int DIM, int PREC, int WHAT, int NTH>
__global__ void __launch_bounds__(NTH, NTH == NT ? scatter_min_ctas<PREC, WHAT>() : 1) k_tile_scatter(TileArgs A) {
    extern __shared__ __align__(16) char smem[];
    const int t = (int)(A.tile_base + blockIdx.x);
    auto pf = [&](int lane) {
        if (A.ahead > 0) prefetch_tile_l2<DIM, (WHAT & DO_ADJ) != 0>(A, t + A.ahead, lane);
    };
    run_tile_scatter<DIM, PREC, WHAT, NTH>(A, t, smem, pf);
}

template <int DIM, int PREC, int WHAT>
int launch_tiles_scatter(const em_mesh* m, TileArgs& A, cudaStream_t s) {
    const SmemS L = smem_layout_s<DIM, PREC, WHAT>(A.D);
    static size_t configured = 0;
    // a limb plane entry holds < 1024 contributions of magnitude <= 2^21
    if (A.val_e > 1000 || A.val_v > 250)
        return fail(EM_ERR_ARG, "tiled path: an edge with more than 1000 elements or a node with more than 250 "
                                "elements exceeds its fixed-point headroom; use the gather path");
    if (L.total > 227 * 1024)
        return fail(EM_ERR_ARG, "tile needs " + std::to_string(L.total) +
                                    " bytes of shared memory (> 227 KB): rebuild the plan with a smaller tile_nodes");
    if (L.total > 48 * 1024 && L.total > configured) {
        EM_CUDA_TRY(cudaFuncSetAttribute(k_tile_scatter<DIM, PREC, WHAT, NT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
        if constexpr (DIM == 3)
            EM_CUDA_TRY(cudaFuncSetAttribute(k_tile_scatter<DIM, PREC, WHAT, 2 * NT>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
        configured = 227 * 1024;
    }
    // one resident CTA of NT threads per SM leaves half the register file
    // idle: such tiles run with 2 NT threads (3D; the results do not depend
    // on the thread count)
    bool wide = false;
    int per_sm = 0;
    EM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tile_scatter<DIM, PREC, WHAT, NT>, NT, L.total));
    if constexpr (DIM == 3) {
        if (per_sm < 2) {
            wide = true;
            EM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tile_scatter<DIM, PREC, WHAT, 2 * NT>,
                                                                      2 * NT, L.total));
        }
    }
    // with one CTA per SM nothing hides a tile's staging latency: tile t
    // prefetches the tile that starts after it (tiles resident at once ahead)
    A.ahead = per_sm == 1 ? num_sms() : 0;
    const int64_t n_tiles = m->plan_info[EM_PLAN_INFO_TILES];
    const int64_t chunk = 1 << 30;
    for (int64_t base = 0; base < n_tiles; base += chunk) {
        A.tile_base = base;
        int64_t nb = n_tiles - base < chunk ? n_tiles - base : chunk;
        if constexpr (DIM == 3) {
            if (wide)
                k_tile_scatter<DIM, PREC, WHAT, 2 * NT><<<(unsigned)nb, 2 * NT, L.total, s>>>(A);
            else
                k_tile_scatter<DIM, PREC, WHAT, NT><<<(unsigned)nb, NT, L.total, s>>>(A);
        } else {
            k_tile_scatter<DIM, PREC, WHAT, NT><<<(unsigned)nb, NT, L.total, s>>>(A);
        }
        note_launches(1);
    }
    EM_CUDA_TRY(cudaGetLastError());
    return EM_OK;
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
    if (what & GATHER_SCATTER) {
        const int w = what & (GATHER_FWD | GATHER_ADJ);
        if (w == GATHER_FWD) return launch_tiles_scatter<DIM, PREC, DO_FWD>(m, A, s);
        if (w == GATHER_ADJ) return launch_tiles_scatter<DIM, PREC, DO_ADJ>(m, A, s);
        return launch_tiles_scatter<DIM, PREC, DO_FWD | DO_ADJ>(m, A, s);
    }
    if (what == GATHER_FWD) return launch_tiles<DIM, PREC, DO_FWD>(m, A, s);
    if (what == GATHER_ADJ) return launch_tiles<DIM, PREC, DO_ADJ>(m, A, s);
    return launch_tiles<DIM, PREC, DO_FWD | DO_ADJ>(m, A, s);
}

// ---- batched: the tiles of many grids in one launch --------------------------
// Work item = (grid, tile), numbered through the grids' tile prefix sums.  Two
// launch shapes run each item through the same tiled scatter, so both give
// the results of the single-grid tiled path bit for bit:
//   item grid (default): one CTA per item, dispatched by the hardware in item
//     order;
//   persistent: a fixed set of CTAs claims items through one atomic counter.
// The persistent loop around the element loop leaves the register allocator
// less room (it spills at this register budget), so the item grid is faster.
__device__ __forceinline__ void args_from_mesh(const em_batch_item& it, TileArgs& A) {
    A.plan = it.mesh.plan;
    A.bnode = it.mesh.bnode;
    A.x = it.x; A.w = it.w; A.c = it.c;
    A.n_out = it.n_edge; A.vol = it.vol; A.bnormal = it.bnormal; A.grad = it.grad_x;
    A.n_tiles = (int)it.mesh.plan_info[EM_PLAN_INFO_TILES];
    A.val_e = (int)it.mesh.plan_info[EM_PLAN_INFO_MAX_EDGE_VALENCE];
    A.val_v = (int)it.mesh.plan_info[EM_PLAN_INFO_MAX_NODE_VALENCE];
    A.tile_base = 0;
    A.bwa = BwAux{nullptr, nullptr, nullptr};
    A.ahead = 0;
}

// last grid whose prefix <= wk
__device__ __forceinline__ int item_grid(const int64_t* pre, int n_meshes, int64_t wk) {
    int lo = 0, hi = n_meshes - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (pre[mid] <= wk) lo = mid; else hi = mid - 1;
    }
    return lo;
}

template <int DIM>
__device__ void prefetch_item_l2(const em_batch_item* items, const int64_t* pre, int n_meshes, int64_t nx, int lane) {
    const int g = item_grid(pre, n_meshes, nx);
    if (items[g].mesh.dim != DIM) return;
    TileArgs B;
    args_from_mesh(items[g], B);
    prefetch_tile_l2<DIM, true>(B, (int)(nx - pre[g]), lane);
}

// one CTA per work item; `ahead` > 0: prefetch item wk + ahead into L2
template <int DIM, int PREC, int NTH>
__global__ void __launch_bounds__(NTH, (NTH == NT ? scatter_min_ctas<PREC, DO_FWD | DO_ADJ>() : 1))
    k_batched_items(const em_batch_item* __restrict__ items, const int64_t* __restrict__ prefix, int n_meshes,
                    Dims D, int32_t* status, int ahead) {
    extern __shared__ __align__(16) char smem[];
    __shared__ TileArgs sA;     // the item's arguments, read by every thread
    const int64_t wk = blockIdx.x;
    const int64_t total = prefix[n_meshes];
    if (wk >= total) return;    // a grid larger than the item count: nothing to do
    const int g = item_grid(prefix, n_meshes, wk);
    const em_batch_item& it = items[g];
    if (it.mesh.dim != DIM) {   // block-uniform
        if (threadIdx.x == 0) atomicExch(status, EM_ERR_ARG);
        return;
    }
    if (threadIdx.x == 0) {
        args_from_mesh(it, sA);
        sA.D = D;
    }
    __syncthreads();
    auto pf = [&](int lane) {
        if (ahead > 0 && wk + ahead < total) prefetch_item_l2<DIM>(items, prefix, n_meshes, wk + ahead, lane);
    };
    run_tile_scatter<DIM, PREC, DO_FWD | DO_ADJ, NTH>(sA, (int)(wk - prefix[g]), smem, pf);
}

// persistent CTAs draining the work list; `prefetch`: prefetch the item
// claimed next into L2
template <int DIM, int PREC, int NTH>
__global__ void __launch_bounds__(NTH, (NTH == NT ? scatter_min_ctas<PREC, DO_FWD | DO_ADJ>() : 1))
    k_batched(const em_batch_item* __restrict__ items, const int64_t* __restrict__ prefix, int n_meshes, Dims D,
              unsigned long long* counter, int32_t* status, int prefetch) {
    extern __shared__ __align__(16) char smem[];
    __shared__ long long s_next;
    __shared__ TileArgs sA;
    // the tile prefix sums live in shared memory behind the tile's layout
    const SmemS L = smem_layout_s<DIM, PREC, DO_FWD | DO_ADJ>(D);
    int64_t* spre = reinterpret_cast<int64_t*>(smem + L.total);
    for (int i = threadIdx.x; i <= n_meshes; i += blockDim.x) spre[i] = prefix[i];
    if (threadIdx.x == 0) s_next = (long long)atomicAdd(counter, 1ull);
    __syncthreads();
    const int64_t total = spre[n_meshes];
    for (;;) {
        const int64_t wk = s_next;
        __syncthreads();
        if (wk >= total) break;
        // claim the following item now; its atomic completes while this tile runs
        if (threadIdx.x == 0) s_next = (long long)atomicAdd(counter, 1ull);
        const int g = item_grid(spre, n_meshes, wk);
        const em_batch_item& it = items[g];
        if (it.mesh.dim != DIM) {   // block-uniform branch
            if (threadIdx.x == 0) atomicExch(status, EM_ERR_ARG);
            __syncthreads();         // orders the claim above before the next read of s_next
            continue;
        }
        if (threadIdx.x == 0) {
            args_from_mesh(it, sA);
            sA.D = D;
        }
        __syncthreads();
        // s_next (written before the tile's first barrier) is this block's
        // next item
        auto pf = [&](int lane) {
            const long long nx = s_next;
            if (prefetch && nx < total) prefetch_item_l2<DIM>(items, spre, n_meshes, nx, lane);
        };
        run_tile_scatter<DIM, PREC, DO_FWD | DO_ADJ, NTH>(sA, (int)(wk - spre[g]), smem, pf);
        __syncthreads();
    }
}

template <int DIM, int PREC, int NTH>
int launch_batched_as(int n_meshes, const em_batch_item* items, const int64_t* prefix, int64_t n_items, const Dims& D,
                      int blocks, int per_sm, size_t bytes, unsigned long long* counter, int32_t* status,
                      cudaStream_t s) {
    if (blocks == 0) {
        // one CTA per item; with one CTA per SM, item wk prefetches the item
        // that starts after it
        const int ahead = per_sm == 1 ? num_sms() : 0;
        EM_CUDA_TRY(cudaFuncSetAttribute(k_batched_items<DIM, PREC, NTH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)bytes));
        k_batched_items<DIM, PREC, NTH><<<(unsigned)n_items, NTH, bytes, s>>>(items, prefix, n_meshes, D, status,
                                                                               ahead);
    } else {
        if (blocks < 0) blocks = num_sms() * (per_sm > 0 ? per_sm : 1);
        EM_CUDA_TRY(cudaFuncSetAttribute(k_batched<DIM, PREC, NTH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(bytes + sizeof(int64_t) * (size_t)(n_meshes + 1))));
        k_batched<DIM, PREC, NTH><<<blocks, NTH, bytes + sizeof(int64_t) * (size_t)(n_meshes + 1), s>>>(
            items, prefix, n_meshes, D, counter, status, per_sm == 1 ? 1 : 0);
    }
    note_launches(1);
    EM_CUDA_TRY(cudaGetLastError());
    return EM_OK;
}

template <int DIM, int PREC>
int launch_batched(int n_meshes, const em_batch_item* items, const int64_t* prefix, int64_t n_items, const Dims& D,
                   int blocks, unsigned long long* counter, int32_t* status, cudaStream_t s) {
    const SmemS L = smem_layout_s<DIM, PREC, DO_FWD | DO_ADJ>(D);
    const size_t bytes = L.total;
    const size_t need = L.total + (blocks != 0 ? sizeof(int64_t) * (size_t)(n_meshes + 1) : 0);
    if (need > 227 * 1024)
        return fail(EM_ERR_ARG, "batched tiles need " + std::to_string(need) +
                                    " bytes of shared memory (> 227 KB): use a smaller tile_nodes or fewer grids");
    // as for one grid: tiles that fill an SM run with 2 NT threads (3D) and
    // prefetch their next item (the results depend on neither)
    int per_sm = 0;
    EM_CUDA_TRY(cudaFuncSetAttribute(k_batched_items<DIM, PREC, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)need));
    EM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batched_items<DIM, PREC, NT>, NT, need));
    if constexpr (DIM == 3) {
        if (per_sm < 2) {
            EM_CUDA_TRY(cudaFuncSetAttribute(k_batched_items<DIM, PREC, 2 * NT>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need));
            EM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batched_items<DIM, PREC, 2 * NT>,
                                                                      2 * NT, need));
            return launch_batched_as<DIM, PREC, 2 * NT>(n_meshes, items, prefix, n_items, D, blocks, per_sm, bytes,
                                                        counter, status, s);
        }
    }
    return launch_batched_as<DIM, PREC, NT>(n_meshes, items, prefix, n_items, D, blocks, per_sm, bytes, counter,
                                            status, s);
}

}  // namespace

int batched_impl(int n_meshes, const em_batch_item* items, const int64_t* tile_prefix, int64_t n_items,
                 const int64_t* max_info, int dim, int precision, int blocks, int32_t* status, void* ws,
                 size_t* ws_bytes, cudaStream_t s) {
    bool query;
    EM_TRY(check_ws(ws, ws_bytes, 256, &query));
    if (query) return EM_OK;
    if (n_meshes <= 0 || !items || !tile_prefix || !max_info || !status)
        return fail(EM_ERR_ARG, "batched call needs items, tile_prefix, max_info and status");
    if (n_items <= 0 || n_items > 0x7fffffffLL) return fail(EM_ERR_ARG, "n_items must be in [1, 2^31)");
    if (blocks < EM_BATCH_PERSISTENT) return fail(EM_ERR_ARG, "blocks must be >= EM_BATCH_PERSISTENT (-1)");
    if (dim != 2 && dim != 3) return fail(EM_ERR_ARG, "dim must be 2 or 3");
    if (precision != EM_PREC_FP64 && precision != EM_PREC_DW && precision != EM_PREC_MIXED)
        return fail(EM_ERR_ARG, "batched pass supports FP64, DW and MIXED");
    Dims D;
    D.max_nodes = (int)max_info[EM_PLAN_INFO_MAX_NODES];
    D.max_edges = (int)max_info[EM_PLAN_INFO_MAX_EDGES];
    D.max_eo = (int)max_info[EM_PLAN_INFO_MAX_OWNED_EDGES];
    D.max_own = (int)max_info[EM_PLAN_INFO_MAX_OWNED_NODES];
    D.max_bo = (int)max_info[EM_PLAN_INFO_MAX_OWNED_BNODES];
    D.max_es = (int)max_info[EM_PLAN_INFO_MAX_ESLOTS];
    D.max_ns = (int)max_info[EM_PLAN_INFO_MAX_NSLOTS];
    D.max_bs = (int)max_info[EM_PLAN_INFO_MAX_BSLOTS];
    if (D.max_own <= 0 || D.max_nodes <= 0) return fail(EM_ERR_ARG, "max_info is empty");
    // each grid's tiles accumulate in exact fixed point (tiled scatter)
    if (max_info[EM_PLAN_INFO_MAX_EDGE_VALENCE] > 1000 || max_info[EM_PLAN_INFO_MAX_NODE_VALENCE] > 250)
        return fail(EM_ERR_ARG, "batched pass: an edge with more than 1000 elements or a node with more than 250 "
                                "elements exceeds the fixed-point headroom");
    unsigned long long* counter = static_cast<unsigned long long*>(ws);
    EM_CUDA_TRY(cudaMemsetAsync(counter, 0, sizeof(unsigned long long), s));
    EM_CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(int32_t), s));
    if (dim == 3) {
        if (precision == EM_PREC_FP64) return launch_batched<3, EM_PREC_FP64>(n_meshes, items, tile_prefix, n_items, D, blocks, counter, status, s);
        if (precision == EM_PREC_DW) return launch_batched<3, EM_PREC_DW>(n_meshes, items, tile_prefix, n_items, D, blocks, counter, status, s);
        return launch_batched<3, EM_PREC_MIXED>(n_meshes, items, tile_prefix, n_items, D, blocks, counter, status, s);
    }
    if (precision == EM_PREC_FP64) return launch_batched<2, EM_PREC_FP64>(n_meshes, items, tile_prefix, n_items, D, blocks, counter, status, s);
    if (precision == EM_PREC_DW) return launch_batched<2, EM_PREC_DW>(n_meshes, items, tile_prefix, n_items, D, blocks, counter, status, s);
    return launch_batched<2, EM_PREC_MIXED>(n_meshes, items, tile_prefix, n_items, D, blocks, counter, status, s);
}

size_t gather_ws_bytes(const em_mesh*) { return 0; }

int gather_run(const em_mesh* m, int prec, int what, const double* x, const double* w, const double* c, double* n,
               double* vol, double* bnormal, double* g, void* ws, cudaStream_t s, const BwAux* bw) {
    (void)ws;
    const int64_t* pi = m->plan_info;
    if (pi[EM_PLAN_INFO_TILES] <= 0 || pi[EM_PLAN_INFO_CHECK] <= 0 || (size_t)pi[EM_PLAN_INFO_CHECK] > m->plan_bytes)
        return fail(EM_ERR_ARG, "mesh->plan_info does not describe mesh->plan (copy em_plan_build's plan_info)");
    if (m->n_bnodes && !m->bnode) return fail(EM_ERR_ARG, "gather path needs bnode");
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
    A.val_e = (int)(pi[EM_PLAN_INFO_MAX_EDGE_VALENCE] > 0 ? pi[EM_PLAN_INFO_MAX_EDGE_VALENCE] : 64);
    A.val_v = (int)(pi[EM_PLAN_INFO_MAX_NODE_VALENCE] > 0 ? pi[EM_PLAN_INFO_MAX_NODE_VALENCE] : 64);
    A.tile_base = 0;
    A.ahead = 0;
    A.bwa = bw ? *bw : BwAux{nullptr, nullptr, nullptr};
    if (A.bwa.bw && !(what & GATHER_SCATTER))
        return fail(EM_ERR_ARG, "boundary-normal weights are supported by the TILED and ATOMIC paths");
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

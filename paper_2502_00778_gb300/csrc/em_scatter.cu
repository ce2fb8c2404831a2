// Scatter tiles (EM_PATH_TILED; plan sections described in em_plan.cuh).
//
// Every element belongs to exactly one tile (the tile of its lowest node) and
// every boundary face to the tile of its owner element, so each element and
// face is computed exactly once.  One CTA per tile:
//   1. stage the coordinates of the tile's local nodes (owned nodes, then the
//      halo nodes of its elements) in shared memory, relative to the tile's
//      first node (FP32-based forms: as float pairs), and, for the adjoint,
//      the w of its local edges and the c of its local nodes;
//   2. bound the element geometry (largest coordinate difference along an
//      element edge) and derive a power-of-two fixed-point scale per output
//      kind such that no partial sum can overflow;
//   3. warps take 32-element chunks from a shared counter; every element
//      adds ALL its contributions (face vectors to its edges, volume to its
//      nodes, gradient terms to its nodes) to shared-memory accumulators of
//      the tile's local targets as exact integers split into 21-bit limbs,
//      one native 32-bit shared atomic per limb (em_tile_forms.cuh);
//   4. boundary faces likewise;
//   5. owned targets are converted and written as outputs; halo targets
//      (owned by later tiles) are converted and written as records at their
//      position in the plan's halo lists.
// A merge pass then adds, for every target that has records, its records in
// ascending record order (= ascending tile order) to the owner's output.
// Integer sums inside a tile do not depend on the order of the atomics and
// the merge order is fixed, so the results are bit-identical from run to run
// and independent of the launch shape.
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
// Adjoint (gradient of L = sum_e w_e.n_e + sum_i c_i V_i + sum_b bw_b.bnormal_b):
// the element's loss is a sum of triple products, so with W_0 = w01+w02+w03,
// W_1 = w12+w13, W_2 = w23, A_1 = W_1 - W_0, A_2 = W_2 - W_0, A_3 = -W_0 and
// C = c0+c1+c2+c3, the gradient at node k (k = 1, 2, 3, indices cyclic,
// X = (a, b, c)) is g_k = -s/12 (A_{k+1} x X_{k+2} - A_{k+2} x X_{k+1})
// + s C/24 N_k, and at node 0 -(g_1 + g_2 + g_3).  Since N_1 = b x c, etc.,
// the volume term folds into the cross products: with A''_k = A_k - (C/4) X_k,
// g_k = -s/12 (A''_{k+1} x X_{k+2} - A''_{k+2} x X_{k+1}).  The 3D tile sums
// hold 12 g (the 1/12 is applied once per output), and node 0's share is the
// integer sum -(q_1 + q_2 + q_3) of the other nodes' quantised values, as is
// the share of the edges at node 0 in the forward (m0 = -(m1 + m2 + m3)).
#include "em_common.cuh"
#include "em_dw.cuh"
#include "em_kernels.cuh"
#include "em_plan.cuh"
#include "em_tile_forms.cuh"

namespace em {

namespace {

constexpr int NT = 256;   // threads per CTA (512 for tiles that fill an SM, 3D)

struct SDims {
    int max_nodes, max_edges, max_bnodes;   // local targets of the largest tile
};

struct SArgs {
    const void* plan;
    const double* x;
    const double* w;
    const double* c;
    double* n_out;
    double* vol;
    double* bnormal;
    double* grad;
    double* rec_e;          // [edge records][DIM]: n
    double* rec_v;          // [node records]: V
    double* rec_g;          // [node records][DIM]: grad
    double* rec_b;          // [boundary-node records][DIM]: bnormal
    SDims D;
    int n_tiles;
    int val_e, val_v;       // largest edge / node valence of the grid
    int64_t tile_base;      // first tile handled by blockIdx.x == 0
    BwAux bwa;              // boundary-normal weights of the adjoint (bwa.bw NULL: none)
    int ahead;              // > 0: each tile prefetches tile t + ahead's inputs into L2
};

struct SmemS {
    size_t xs, ws, cs, acc_e, acc_v, acc_g, acc_b, red, total;
};

// shared-memory layout, computed identically on host and device; the
// accumulator planes (acc_e .. acc_b) are one contiguous block
template <int DIM, int PREC, int WHAT>
__host__ __device__ inline SmemS s_layout(const SDims& D) {
    using F = Form<PREC>;
    SmemS s;
    size_t o = 0;
    auto take = [&](size_t bytes) { o = (o + 15) & ~size_t(15); size_t r = o; o += bytes; return r; };
    const size_t wb = Fix<PREC>::NL * sizeof(int);
    s.xs = take(sizeof(typename F::C) * DIM * D.max_nodes);
    s.ws = (WHAT & DO_ADJ) ? take(sizeof(typename F::V) * DIM * D.max_edges) : 0;
    s.cs = (WHAT & DO_ADJ) ? take(sizeof(typename F::V) * D.max_nodes) : 0;
    const size_t acc0 = (o + 15) & ~size_t(15);
    s.acc_e = (WHAT & DO_FWD) ? take(wb * DIM * D.max_edges) : acc0;
    s.acc_v = (WHAT & DO_FWD) ? take(wb * D.max_nodes) : acc0;
    s.acc_g = (WHAT & DO_ADJ) ? take(wb * DIM * D.max_nodes) : acc0;
    s.acc_b = (WHAT & DO_FWD) ? take(wb * DIM * D.max_bnodes) : acc0;
    s.red = take(sizeof(unsigned) * (16 + 5 * RED_WARPS));
    s.total = (o + 15) & ~size_t(15);
    return s;
}

// ---- L2 prefetch of a later tile's inputs -----------------------------------
// Tiles are dispatched in index order, so while tile t computes, tile
// t + (resident CTAs) is about to start on some SM.  Used when one CTA fills
// an SM.  One warp of tile t asks L2 for that tile's contiguous records and
// owned rows (bulk prefetches) and for the halo rows it will gather.
template <int DIM, bool ADJ>
__device__ void prefetch_stile_l2(const SArgs& A, int t2, int lane) {
    if (t2 >= A.n_tiles) return;
    const PlanHeader* H = static_cast<const PlanHeader*>(A.plan);
    const STile ti = plan_at<STile>(A.plan, H->off_stiles)[t2];
    const int32_t* halo = plan_at<int32_t>(A.plan, H->off_shalo) + ti.halo_off;
    const int32_t* hedge = plan_at<int32_t>(A.plan, H->off_shedge) + ti.hedge_off;
    switch (lane) {
        case 0: l2_prefetch_range(plan_at<ElemConn>(A.plan, H->off_sconn) + ti.elem_off, (long long)sizeof(ElemConn) * ti.n_el); break;
        case 1: l2_prefetch_range(plan_at<ElemEdges>(A.plan, H->off_stedge) + ti.elem_off, (long long)sizeof(ElemEdges) * ti.n_el); break;
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
        case 7: l2_prefetch_range(plan_at<SFace>(A.plan, H->off_sbf) + ti.bf_off, (long long)sizeof(SFace) * ti.n_bf); break;
        default: break;
    }
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

// pf(lane) is called by the last warp once the tile's staging is done: it may
// prefetch a later tile's inputs into L2 while the other warps compute
template <int DIM, int PREC, int WHAT, int NTH, class PF>
__device__ __forceinline__ void run_stile(const SArgs& A, int t, char* smem, const PF& pf) {
    using F = Form<PREC>;
    using FX = Fix<PREC>;
    using C = typename F::C;
    using V = typename F::V;
    const PlanHeader* H = static_cast<const PlanHeader*>(A.plan);
    const STile ti = plan_at<STile>(A.plan, H->off_stiles)[t];
    const ElemConn* conn = plan_at<ElemConn>(A.plan, H->off_sconn) + ti.elem_off;
    const ElemEdges* tedge = plan_at<ElemEdges>(A.plan, H->off_stedge) + ti.elem_off;
    const int32_t* halo = plan_at<int32_t>(A.plan, H->off_shalo) + ti.halo_off;
    const int32_t* hedge = plan_at<int32_t>(A.plan, H->off_shedge) + ti.hedge_off;
    const int32_t* hbo = plan_at<int32_t>(A.plan, H->off_shbo) + ti.hbo_off;
    const SFace* sbf = plan_at<SFace>(A.plan, H->off_sbf) + ti.bf_off;

    const SmemS L = s_layout<DIM, PREC, WHAT>(A.D);
    C* xs = reinterpret_cast<C*>(smem + L.xs);
    V* ws = reinterpret_cast<V*>(smem + L.ws);
    V* cs = reinterpret_cast<V*>(smem + L.cs);
    constexpr int NL = FX::NL;
    int* acc_e = reinterpret_cast<int*>(smem + L.acc_e);
    int* acc_v = reinterpret_cast<int*>(smem + L.acc_v);
    int* acc_g = reinterpret_cast<int*>(smem + L.acc_g);
    int* acc_b = reinterpret_cast<int*>(smem + L.acc_b);
    // limb plane strides
    const int se = DIM * A.D.max_edges, sv = A.D.max_nodes, sgs = DIM * A.D.max_nodes, sb = DIM * A.D.max_bnodes;
    unsigned* red = reinterpret_cast<unsigned*>(smem + L.red);
    unsigned* wred = red + 16;
    static_assert(NTH / 32 <= RED_WARPS, "one maximum slot per warp");

    const int tid = threadIdx.x;
    const int nnodes = ti.n_own + ti.n_halo;
    const int nedges = ti.n_eo + ti.n_hedge;
    const int nbn = ti.n_bo + ti.n_hbo;

    // ---- clear the accumulator block (16-byte stores) -------------------------
    if (tid < 16) red[tid] = 0u;
    {
        int4* a4 = reinterpret_cast<int4*>(smem + L.acc_e);
        const int n4 = (int)((L.red - L.acc_e) / 16);
        for (int q = tid; q < n4; q += NTH) a4[q] = make_int4(0, 0, 0, 0);
    }
    // (no barrier: the planes are first used after the staging and extent
    // barriers below)

    // 512-thread tiles (one CTA per SM, nothing hides their latency): this
    // thread's first element records of the extent pass below are requested
    // now, so that they arrive while the staging gathers are in flight
    constexpr int EB = 8;
    constexpr bool HOIST = NTH > NT;
    ElemConn ecb[HOIST ? EB : 1];
    if constexpr (HOIST) {
#pragma unroll
        for (int u = 0; u < EB; u++)
            if (tid + u * NTH < ti.n_el) ecb[u] = conn[tid + u * NTH];
    }

    // ---- stage coordinates (and w, c) and find the tile's magnitudes --------
    // Each thread takes up to SB nodes and SBW edges per round.  It first
    // requests the halo indices of all of them (owned rows need none), then all
    // their gathers, and converts last, so a round costs two dependent trips to
    // L2 / HBM however many lists it covers.  The tile origin is loaded with
    // the indices and only replaced when it is not finite (rare).
    constexpr int SB = NTH > NT ? 1 : 2, SBW = (WHAT & DO_ADJ) ? 6 : 1;
    double org[DIM];
#pragma unroll
    for (int d = 0; d < DIM; d++) org[d] = A.x[int64_t(ti.node0) * DIM + d];
    unsigned wm = 0u, cm = 0u;
    float xl = 0.f;      // DW / MIXED forms: largest |low part| of a staged coordinate
    bool nf = false;     // a staged value is non-finite (staged as NaN)
    const int n_rounds = max((nnodes + SB * NTH - 1) / (SB * NTH),
                             (WHAT & DO_ADJ) ? (nedges + SBW * NTH - 1) / (SBW * NTH) : 0);
    for (int r = 0; r < n_rounds; r++) {
        int vn[SB], ve[SBW];
#pragma unroll
        for (int u = 0; u < SB; u++) {
            const int i = r * SB * NTH + tid + u * NTH;
            vn[u] = i >= nnodes ? -1 : (i < ti.n_own ? ti.node0 + i : halo[i - ti.n_own]);
        }
        if (WHAT & DO_ADJ) {
#pragma unroll
            for (int u = 0; u < SBW; u++) {
                const int i = r * SBW * NTH + tid + u * NTH;
                ve[u] = i >= nedges ? -1 : (i < ti.n_eo ? ti.edge0 + i : hedge[i - ti.n_eo]);
            }
        }
        double xv[SB][DIM], cv[SB], wv[SBW][DIM];
#pragma unroll
        for (int u = 0; u < SB; u++) {
            if (vn[u] < 0) continue;
#pragma unroll
            for (int d = 0; d < DIM; d++) xv[u][d] = A.x[int64_t(vn[u]) * DIM + d];
            if (WHAT & DO_ADJ) cv[u] = A.c ? A.c[vn[u]] : 0.0;
        }
        if (WHAT & DO_ADJ) {
#pragma unroll
            for (int u = 0; u < SBW; u++)
                if (ve[u] >= 0)
#pragma unroll
                    for (int d = 0; d < DIM; d++) wv[u][d] = A.w[int64_t(ve[u]) * DIM + d];
        }
        if (r == 0) {
#pragma unroll
            for (int d = 0; d < DIM; d++)
                if (!isfinite(org[d])) org[d] = tile_origin_component<DIM>(A.x, ti.node0, ti.n_own, d);
        }
#pragma unroll
        for (int u = 0; u < SB; u++) {
            if (vn[u] < 0) continue;
            const int i = r * SB * NTH + tid + u * NTH;
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
        if (WHAT & DO_ADJ) {
#pragma unroll
            for (int u = 0; u < SBW; u++) {
                if (ve[u] < 0) continue;
                const int i = r * SBW * NTH + tid + u * NTH;
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
    // Each bound is a product (or a sum of three products) of upper bounds,
    // evaluated as float mantissas rounded up times powers of two: every
    // thread derives the same scales with no FP64 instruction and no further
    // barrier, and each scale gives away less than one of the 62 bits plus
    // the 2^-12 margin below.  A partial sum of a tile holds at most as many
    // contributions as the full sum, so the grid's valences bound it too.
    constexpr int TP = FX::TOP, LO = FX::LO, HI = FX::HI;
    constexpr int NW = NTH / 32;
    // Lx.  FP64 form: slot 0 bounds the computed differences, rounded to
    // nearest, so the exact ones too.  DW / MIXED: |a - b| <= |a.h - b.h| +
    // |a.l| + |b.l| <= fl(a.h - b.h) (1 + 2^-23) + 2 max|low part| (slot 3).
    Ub uL = ub_key(red_max(wred, 0, NW));
    if constexpr (PREC != EM_PREC_FP64) {
        Ub l3 = ub_key(red_max(wred, 3, NW));
        l3.e += 1;
        uL = ub_add(ub_scale(uL, 1.0f + 0x1p-23f), l3);
    }
    // mantissa products m (>= 1, rounded up) and exponent sums e: the bound
    // is below m 2^e; powers of two go to e
    const float mL2 = __fmul_ru(uL.m, uL.m), mL3 = __fmul_ru(mL2, uL.m);
    // contribution counts (the launcher refuses valences above 340 / 170, so
    // these floats are exact), with a 2^-12 margin for the rounding of the
    // computed contributions against the exact quantities bounded here
    const float Ke = __fmul_ru((float)(max(A.val_e, 1) + 1), 1.0f + 0x1p-12f);
    const float Kv = __fmul_ru((float)(max(A.val_v, 1) + 1), 1.0f + 0x1p-12f);
    auto room = [&](float m, int e) { return TP - (e + ub_bits(m)); };
    int u_g = HI;
    if (WHAT & DO_ADJ) {
        // |w|, |c|, |bw| below W, C, B
        const Ub W = ub_key(red_max(wred, 1, NW)), C = ub_key(red_max(wred, 2, NW));
        Ub T;
        if (DIM == 3) {   // 12 (16 |w| Lx + 8 |c| Lx^2 + 16 |bw| Lx) 2 Kv: the 3D sums hold 12 g
            T = ub_add(ub_norm(__fmul_ru(W.m, uL.m), W.e + uL.e + 4), ub_norm(__fmul_ru(C.m, mL2), C.e + 2 * uL.e + 3));
            if (A.bwa.bw) {
                const Ub B = ub_key(*A.bwa.key);
                T = ub_add(T, ub_norm(__fmul_ru(B.m, uL.m), B.e + uL.e + 4));
            }
            u_g = room(__fmul_ru(__fmul_ru(T.m, Kv), 3.0f), T.e + 3);
        } else {          // (4 |w| + 4 |c| Lx + 4 |bw|) 2 Kv
            T = ub_add(W, ub_norm(__fmul_ru(C.m, uL.m), C.e + uL.e));
            if (A.bwa.bw) T = ub_add(T, ub_key(*A.bwa.key));
            u_g = room(__fmul_ru(T.m, Kv), T.e + 3);
        }
    }
    // 3D: |N_i| components <= 2 Lx^2, |det| <= 3 sqrt(3) Lx^3 < 8 Lx^3,
    // |n_B| <= 8 Lx^2 with up to 3 boundary faces per element at a node; the
    // factors 2^5, 2^3, 2^5 cover the shares and the sums' 12 n, 24 V,
    // 3 bnormal; 2D: |n_i| <= 2 Lx, |det| <= 2 Lx^2, boundary edge <= 2 Lx
    // (factors 2^3, 2^4, 2^3)
    const int u_e = DIM == 3 ? room(__fmul_ru(mL2, Ke), 2 * uL.e + 5) : room(__fmul_ru(uL.m, Ke), uL.e + 3);
    const int u_v = DIM == 3 ? room(__fmul_ru(mL3, Kv), 3 * uL.e + 3) : room(__fmul_ru(mL2, Kv), 2 * uL.e + 4);
    const int u_b = DIM == 3 ? room(__fmul_ru(mL2, Kv), 2 * uL.e + 5) : room(__fmul_ru(uL.m, Kv), uL.e + 3);
    const int sg_e = sg_clamp(u_e, LO, HI), sg_v = sg_clamp(u_v, LO, HI), sg_b = sg_clamp(u_b, LO, HI);
    const int sg_g = (WHAT & DO_ADJ) ? sg_clamp(u_g, LO, HI) : 0;
    // Element extents outside the form's range (a scale outside [LO, HI]:
    // the values would overflow the fixed point, or lose the digits the
    // contract needs) make every output of the tile NaN instead of silently
    // wrong; for the FP32-based forms that is an element extent outside about
    // 2^-34 .. 2^40, for the FP64 form outside about 2^-290 .. 2^290.  A tile
    // whose elements all have zero extent contributes exact zeros at any scale.
    // Non-finite staged values mark the tile for the poison pass below.
    const bool lx0 = red_max(wred, 0, NW) == 0u;
    const bool range_bad = (!lx0 && (u_e < LO || u_e > HI || u_v < LO || u_v > HI || u_b < LO || u_b > HI)) ||
                           ((WHAT & DO_ADJ) && u_g < LO);
    const bool nf_tile = red_max(wred, 4, NW) != 0u;
    if ((tid >> 5) == (NTH >> 5) - 1) pf(tid & 31);

    // ---- elements: compute and scatter to the tile's local targets ----------
    // warps take chunks of 32 consecutive elements from a shared counter; the
    // next chunk's records are loaded while the current one is computed
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
            if (WHAT & DO_FWD) {
                // edges (0,1),(0,2),(0,3) <- m0; (1,2),(1,3) <- m1; (2,3) <- m2,
                // m_k = -s N_k and m0 = -(m1 + m2 + m3), summed as integers
#pragma unroll
                for (int d = 0; d < 3; d++) {
                    const Lq q1 = FX::q(F::sgn(N1[d], -s), sg_e);
                    const Lq q2 = FX::q(F::sgn(N2[d], -s), sg_e);
                    const Lq q0 = lq_neg_sum(q1, q2, FX::q(F::sgn(N3[d], -s), sg_e));
                    acc_add<NL>(acc_e, se, ee.e[0] * 3 + d, q0);
                    acc_add<NL>(acc_e, se, ee.e[1] * 3 + d, q0);
                    acc_add<NL>(acc_e, se, ee.e[2] * 3 + d, q0);
                    acc_add<NL>(acc_e, se, ee.e[3] * 3 + d, q1);
                    acc_add<NL>(acc_e, se, ee.e[4] * 3 + d, q1);
                    acc_add<NL>(acc_e, se, ee.e[5] * 3 + d, q2);
                }
                const Lq qv = FX::q(F::sgn(det, s), sg_v);
#pragma unroll
                for (int r = 0; r < 4; r++) acc_add<NL>(acc_v, sv, cn.v[r], qv);
            }
            if (WHAT & DO_ADJ) {
                // 12 g_k = -s (A''_{k+1} x X_{k+2} - A''_{k+2} x X_{k+1}), k = 1, 2, 3
                // (indices cyclic, X = (a, b, c)), with A''_k = A_k - (C/4) X_k:
                // the (C/4) X_k terms carry the volume part s C/24 N_k of g_k.
                // The factor 1/12 is applied when the sums are written; node
                // 0 takes -(g_1 + g_2 + g_3), summed as integers.
                V W0[3], Ar[3][3], Xr[3][3];
                const V Cq = F::quarter(F::add(F::add(cs[cn.v[0]], cs[cn.v[1]]), F::add(cs[cn.v[2]], cs[cn.v[3]])));
#pragma unroll
                for (int d = 0; d < 3; d++) {
                    W0[d] = F::add(F::add(ws[ee.e[0] * 3 + d], ws[ee.e[1] * 3 + d]), ws[ee.e[2] * 3 + d]);
                    Xr[0][d] = a[d]; Xr[1][d] = b[d]; Xr[2][d] = c[d];
                    Ar[0][d] = F::sub(F::add(ws[ee.e[3] * 3 + d], ws[ee.e[4] * 3 + d]), F::add(W0[d], F::mul(Cq, a[d])));
                    Ar[1][d] = F::sub(ws[ee.e[5] * 3 + d], F::add(W0[d], F::mul(Cq, b[d])));
                    Ar[2][d] = F::sgn(F::add(W0[d], F::mul(Cq, c[d])), -1.f);
                }
                int vr0 = cn.v[1], vr1 = cn.v[2], vr2 = cn.v[3];
                Lq g0[3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
#pragma unroll 1
                for (int k = 0; k < 3; k++) {
#pragma unroll
                    for (int d = 0; d < 3; d++) {
                        const int d1 = (d + 1) % 3, d2 = (d + 2) % 3;
                        const V g = F::sub(F::det2(Ar[1][d1], Xr[2][d2], Ar[1][d2], Xr[2][d1]),
                                           F::det2(Ar[2][d1], Xr[1][d2], Ar[2][d2], Xr[1][d1]));
                        const Lq q = FX::q(F::sgn(g, -s), sg_g);
                        acc_add<NL>(acc_g, sgs, vr0 * 3 + d, q);
                        lq_sub(g0[d], q);
                    }
                    // rotate: position 0 takes the next k
#pragma unroll
                    for (int d = 0; d < 3; d++) {
                        V t0 = Ar[0][d]; Ar[0][d] = Ar[1][d]; Ar[1][d] = Ar[2][d]; Ar[2][d] = t0;
                        V t1 = Xr[0][d]; Xr[0][d] = Xr[1][d]; Xr[1][d] = Xr[2][d]; Xr[2][d] = t1;
                    }
                    const int tv = vr0; vr0 = vr1; vr1 = vr2; vr2 = tv;
                }
#pragma unroll
                for (int d = 0; d < 3; d++) acc_add<NL>(acc_g, sgs, cn.v[0] * 3 + d, g0[d]);
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
                V n1[2] = {F::sgn(b[1], -s), F::sgn(b[0], s)};
                V n2[2] = {F::sgn(a[1], s), F::sgn(a[0], -s)};
#pragma unroll
                for (int d = 0; d < 2; d++) {
                    const Lq q1 = FX::q(n1[d], sg_e);
                    const Lq q0 = lq_neg_sum(q1, FX::q(n2[d], sg_e), Lq{0, 0, 0});
                    acc_add<NL>(acc_e, se, ee.e[0] * 2 + d, q0);
                    acc_add<NL>(acc_e, se, ee.e[1] * 2 + d, q0);
                    acc_add<NL>(acc_e, se, ee.e[2] * 2 + d, q1);
                }
                const Lq qv = FX::q(F::sgn(det, s), sg_v);
#pragma unroll
                for (int r = 0; r < 3; r++) acc_add<NL>(acc_v, sv, cn.v[r], qv);
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
                const V gax = F::add(F::sgn(F::mul(A2[1], f3), -s), F::mul(h, b[1]));
                const V gay = F::add(F::sgn(F::mul(A2[0], f3), s), F::sgn(F::mul(h, b[0]), -1.f));
                const V gbx = F::add(F::sgn(F::mul(A1[1], f3), s), F::sgn(F::mul(h, a[1]), -1.f));
                const V gby = F::add(F::sgn(F::mul(A1[0], f3), -s), F::mul(h, a[0]));
                const Lq qax = FX::q(gax, sg_g), qay = FX::q(gay, sg_g), qbx = FX::q(gbx, sg_g), qby = FX::q(gby, sg_g);
                acc_add<NL>(acc_g, sgs, cn.v[1] * 2, qax);
                acc_add<NL>(acc_g, sgs, cn.v[1] * 2 + 1, qay);
                acc_add<NL>(acc_g, sgs, cn.v[2] * 2, qbx);
                acc_add<NL>(acc_g, sgs, cn.v[2] * 2 + 1, qby);
                acc_add<NL>(acc_g, sgs, cn.v[0] * 2, lq_neg_sum(qax, qbx, Lq{0, 0, 0}));
                acc_add<NL>(acc_g, sgs, cn.v[0] * 2 + 1, lq_neg_sum(qay, qby, Lq{0, 0, 0}));
            }
        }
    }

    // ---- boundary faces ------------------------------------------------------
    // global boundary-node index of local boundary node lb (for bw)
    auto gbn = [&](int lb) { return lb < ti.n_bo ? int64_t(ti.bnode0) + lb : int64_t(hbo[lb - ti.n_bo]); };
    for (int j = tid; j < ti.n_bf; j += NTH) {
        const SFace f = sbf[j];
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
                    for (int k = 0; k < 3; k++) acc_add<NL>(acc_e, se, f.e[k] * 3 + d, qe);
#pragma unroll
                    for (int k = 0; k < 3; k++) acc_add<NL>(acc_b, sb, f.b[k] * 3 + d, qb);
                }
            }
            if (WHAT & DO_ADJ) {
                V WB[3];
#pragma unroll
                for (int d = 0; d < 3; d++)
                    WB[d] = F::add(F::add(ws[f.e[0] * 3 + d], ws[f.e[1] * 3 + d]), ws[f.e[2] * 3 + d]);
                // 12 x the gradient, like the element terms: 1/2 (t x W_B) and
                // 1/2 (W_B x u) from the edges' n_B/12, and with boundary-normal
                // weights K = 1/3 sum of bw at the face's nodes, 12 (1/2) (t x K)
                // = t x K6, K6 = 6 K = 2 sum bw
                V K6[3];
                const bool hasK = A.bwa.bw != nullptr;
                if (hasK) {
                    double Kd[3] = {0.0, 0.0, 0.0};
#pragma unroll
                    for (int k = 0; k < 3; k++) {
                        const int64_t bi = gbn(f.b[k]);
#pragma unroll
                        for (int d = 0; d < 3; d++) Kd[d] += A.bwa.bw[3 * bi + d];
                    }
#pragma unroll
                    for (int d = 0; d < 3; d++) K6[d] = F::from_double(2.0 * Kd[d]);
                    if (!(isfinite(Kd[0]) && isfinite(Kd[1]) && isfinite(Kd[2]))) atomicOr(red + 11, 1u);
                }
#pragma unroll
                for (int d = 0; d < 3; d++) {
                    const int d1 = (d + 1) % 3, d2 = (d + 2) % 3;
                    V gq = F::half(F::det2(tt[d1], WB[d2], tt[d2], WB[d1]));
                    V gr = F::half(F::det2(WB[d1], u[d2], WB[d2], u[d1]));
                    if (hasK) {
                        gq = F::add(gq, F::det2(tt[d1], K6[d2], tt[d2], K6[d1]));
                        gr = F::add(gr, F::det2(K6[d1], u[d2], K6[d2], u[d1]));
                    }
                    acc_add<NL>(acc_g, sgs, f.v[1] * 3 + d, FX::q(gq, sg_g));
                    acc_add<NL>(acc_g, sgs, f.v[2] * 3 + d, FX::q(gr, sg_g));
                    acc_add<NL>(acc_g, sgs, f.v[0] * 3 + d, FX::q(F::sgn(F::add(gq, gr), -1.f), sg_g));
                }
            }
        } else {
            if (WHAT & DO_FWD) {
                V nB[2] = {F::diff(xs[f.v[0] * 2 + 1], xs[f.v[1] * 2 + 1]), F::diff(xs[f.v[1] * 2 + 0], xs[f.v[0] * 2 + 0])};
#pragma unroll
                for (int d = 0; d < 2; d++) {
                    acc_add<NL>(acc_e, se, f.e[0] * 2 + d, FX::q(F::half(nB[d]), sg_e));
                    const Lq qb = FX::q(nB[d], sg_b);
#pragma unroll
                    for (int k = 0; k < 2; k++) acc_add<NL>(acc_b, sb, f.b[k] * 2 + d, qb);
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
                        const int64_t bi = gbn(f.b[k]);
                        Kd[0] += A.bwa.bw[2 * bi];
                        Kd[1] += A.bwa.bw[2 * bi + 1];
                    }
                    gx = F::add(gx, F::from_double(0.5 * Kd[1]));
                    gy = F::add(gy, F::from_double(-0.5 * Kd[0]));
                    if (!(isfinite(Kd[0]) && isfinite(Kd[1]))) atomicOr(red + 11, 1u);
                }
                acc_add<NL>(acc_g, sgs, f.v[1] * 2, FX::q(gx, sg_g));
                acc_add<NL>(acc_g, sgs, f.v[1] * 2 + 1, FX::q(gy, sg_g));
                acc_add<NL>(acc_g, sgs, f.v[0] * 2, FX::q(F::sgn(gx, -1.f), sg_g));
                acc_add<NL>(acc_g, sgs, f.v[0] * 2 + 1, FX::q(F::sgn(gy, -1.f), sg_g));
            }
        }
    }
    __syncthreads();

    // ---- non-finite inputs (rare; tile-uniform branch) -----------------------
    // Every target to which an element or boundary face with a non-finite
    // input contributes is NaN: forward outputs (n, V, bnormal) from the
    // coordinates, gradients from the coordinates, w, c and the boundary-normal
    // weights.  Such contributions went into the integer sums as arbitrary
    // values (the scales above bound the finite ones only); their targets are
    // marked with a first-limb value no sum can reach (|limb sums| < 2^31 by
    // the headroom argument above) and written as NaN (records too, so the
    // merge carries the NaN to the owner's output).
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
#pragma unroll
                    for (int d = 0; d < DIM; d++) acc_e[ee.e[l] * DIM + d] = MARK;
#pragma unroll
                for (int r = 0; r <= DIM; r++) acc_v[cn.v[r]] = MARK;
            }
            if ((WHAT & DO_ADJ) && pa) {
#pragma unroll
                for (int r = 0; r <= DIM; r++)
#pragma unroll
                    for (int d = 0; d < DIM; d++) acc_g[cn.v[r] * DIM + d] = MARK;
            }
        }
        for (int j = tid; j < ti.n_bf; j += NTH) {
            const SFace f = sbf[j];
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
                        const int64_t bi = gbn(f.b[k]);
#pragma unroll
                        for (int d = 0; d < DIM; d++) pa |= !isfinite(A.bwa.bw[DIM * bi + d]);
                    }
                }
            }
            pa |= px;
            if ((WHAT & DO_FWD) && px) {
#pragma unroll
                for (int k = 0; k < FE; k++)
#pragma unroll
                    for (int d = 0; d < DIM; d++) acc_e[f.e[k] * DIM + d] = MARK;
#pragma unroll
                for (int k = 0; k < DIM; k++)
#pragma unroll
                    for (int d = 0; d < DIM; d++) acc_b[f.b[k] * DIM + d] = MARK;
            }
            if ((WHAT & DO_ADJ) && pa) {
#pragma unroll
                for (int k = 0; k < DIM; k++)
#pragma unroll
                    for (int d = 0; d < DIM; d++) acc_g[f.v[k] * DIM + d] = MARK;
            }
        }
        __syncthreads();
    }

    // ---- outputs: owned targets, records of halo targets ---------------------
    const double esc = DIM == 3 ? 1.0 / 12.0 : 1.0 / 3.0;
    const double vsc = DIM == 3 ? 1.0 / 24.0 : 1.0 / 6.0;
    const double bsc = DIM == 3 ? 1.0 / 3.0 : 1.0 / 2.0;
    // out(p, q): entry q of the planes p at scale sg, NaN where marked
    auto outv = [&](const int* p, int stride, int q, int sg, double sc) {
        if (range_bad || (poison && p[q] == MARK)) return qnan_d();
        return FX::out(acc_load<NL>(p, stride, q), sg, sc);
    };
    // Every output loop takes U entries per thread at a time, so that U
    // independent conversions are in flight.  Owned entries go to the outputs,
    // halo entries to this tile's contiguous block of records (packed:
    // edges and boundary nodes DIM doubles, nodes V then DIM gradient doubles
    // in separate arrays).
    constexpr int U = 4;
    auto emit = [&](int N, const int* p, int stride, int sg, double sc, int n_own_q, double* own, double* rec) {
        for (int q0 = tid; q0 < N; q0 += U * NTH) {
            double v[U];
#pragma unroll
            for (int u = 0; u < U; u++) {
                const int q = q0 + u * NTH;
                v[u] = q < N ? outv(p, stride, q, sg, sc) : 0.0;
            }
#pragma unroll
            for (int u = 0; u < U; u++) {
                const int q = q0 + u * NTH;
                if (q < n_own_q) own[q] = v[u];
                else if (q < N) rec[q - n_own_q] = v[u];
            }
        }
    };
    if (WHAT & DO_FWD) {
        emit(nedges * DIM, acc_e, se, sg_e, esc, ti.n_eo * DIM, A.n_out + int64_t(ti.edge0) * DIM,
             A.rec_e + int64_t(ti.hedge_off) * DIM);
        emit(nbn * DIM, acc_b, sb, sg_b, bsc, ti.n_bo * DIM, A.bnormal + int64_t(ti.bnode0) * DIM,
             A.rec_b + int64_t(ti.hbo_off) * DIM);
        emit(nnodes, acc_v, sv, sg_v, vsc, ti.n_own, A.vol + ti.node0, A.rec_v + ti.halo_off);
    }
    if (WHAT & DO_ADJ)
        emit(nnodes * DIM, acc_g, sgs, sg_g, DIM == 3 ? 1.0 / 12.0 : 1.0, ti.n_own * DIM,
             A.grad + int64_t(ti.node0) * DIM, A.rec_g + int64_t(ti.halo_off) * DIM);
}

// ---- merge: records into the owners' outputs ---------------------------------
// Targets with records, in order: edges [0, n_me), nodes [n_me, n_me + n_mn),
// boundary nodes after them.  Each thread takes whole targets and adds their
// records in ascending record order (fixed, so the sums are reproducible).
struct MergeArgs {
    const void* plan;
    double* n_out;
    double* vol;
    double* bnormal;
    double* grad;
    const double* rec_e;
    const double* rec_v;
    const double* rec_g;
    const double* rec_b;
};

template <int DIM, int WHAT>
__device__ __forceinline__ void merge_targets(const MergeArgs& M, int64_t first, int64_t stride) {
    const PlanHeader* H = static_cast<const PlanHeader*>(M.plan);
    const int64_t ne = (WHAT & DO_FWD) ? H->n_me : 0, nn = H->n_mn, nb = (WHAT & DO_FWD) ? H->n_mb : 0;
    const int32_t* me_id = plan_at<int32_t>(M.plan, H->off_me_id);
    const int32_t* me_ptr = plan_at<int32_t>(M.plan, H->off_me_ptr);
    const int32_t* me_rec = plan_at<int32_t>(M.plan, H->off_me_rec);
    const int32_t* mn_id = plan_at<int32_t>(M.plan, H->off_mn_id);
    const int32_t* mn_ptr = plan_at<int32_t>(M.plan, H->off_mn_ptr);
    const int32_t* mn_rec = plan_at<int32_t>(M.plan, H->off_mn_rec);
    const int32_t* mb_id = plan_at<int32_t>(M.plan, H->off_mb_id);
    const int32_t* mb_ptr = plan_at<int32_t>(M.plan, H->off_mb_ptr);
    const int32_t* mb_rec = plan_at<int32_t>(M.plan, H->off_mb_rec);
    for (int64_t k = first; k < ne + nn + nb; k += stride) {
        if (k < ne) {
            const int64_t e = me_id[k];
            double v[DIM];
#pragma unroll
            for (int d = 0; d < DIM; d++) v[d] = M.n_out[e * DIM + d];
            for (int r = me_ptr[k]; r < me_ptr[k + 1]; r++) {
                const double* p = M.rec_e + int64_t(me_rec[r]) * DIM;
#pragma unroll
                for (int d = 0; d < DIM; d++) v[d] = __dadd_rn(v[d], p[d]);
            }
#pragma unroll
            for (int d = 0; d < DIM; d++) M.n_out[e * DIM + d] = v[d];
        } else if (k < ne + nn) {
            const int64_t j = k - ne, i = mn_id[j];
            double v = 0.0, g[DIM];
            if (WHAT & DO_FWD) v = M.vol[i];
            if (WHAT & DO_ADJ)
#pragma unroll
                for (int d = 0; d < DIM; d++) g[d] = M.grad[i * DIM + d];
            for (int r = mn_ptr[j]; r < mn_ptr[j + 1]; r++) {
                const int64_t rr = mn_rec[r];
                if (WHAT & DO_FWD) v = __dadd_rn(v, M.rec_v[rr]);
                if (WHAT & DO_ADJ)
#pragma unroll
                    for (int d = 0; d < DIM; d++) g[d] = __dadd_rn(g[d], M.rec_g[rr * DIM + d]);
            }
            if (WHAT & DO_FWD) M.vol[i] = v;
            if (WHAT & DO_ADJ)
#pragma unroll
                for (int d = 0; d < DIM; d++) M.grad[i * DIM + d] = g[d];
        } else {
            const int64_t j = k - ne - nn, b = mb_id[j];
            double v[DIM];
#pragma unroll
            for (int d = 0; d < DIM; d++) v[d] = M.bnormal[b * DIM + d];
            for (int r = mb_ptr[j]; r < mb_ptr[j + 1]; r++) {
                const double* p = M.rec_b + int64_t(mb_rec[r]) * DIM;
#pragma unroll
                for (int d = 0; d < DIM; d++) v[d] = __dadd_rn(v[d], p[d]);
            }
#pragma unroll
            for (int d = 0; d < DIM; d++) M.bnormal[b * DIM + d] = v[d];
        }
    }
}

template <int DIM, int WHAT>
__global__ void __launch_bounds__(NT) k_merge(MergeArgs M) {
    merge_targets<DIM, WHAT>(M, blockIdx.x * int64_t(NT) + threadIdx.x, int64_t(gridDim.x) * NT);
}

// resident CTAs per SM the register allocation must allow: the forward alone
// and the FP32 form need little shared memory and fit three CTAs, the other
// adjoint-carrying forms fit two
template <int PREC, int WHAT>
constexpr int scatter_min_ctas() { return (PREC == EM_PREC_MIXED || WHAT == DO_FWD) ? 3 : 2; }

// NTH = 2 NT for tiles so large that one CTA fills an SM's shared memory:
// the register file then still holds 16 warps per SM
template <int DIM, int PREC, int WHAT, int NTH>
__global__ void __launch_bounds__(NTH, NTH == NT ? scatter_min_ctas<PREC, WHAT>() : 1) k_stile(SArgs A) {
    extern __shared__ __align__(16) char smem[];
    const int t = (int)(A.tile_base + blockIdx.x);
    auto pf = [&](int lane) {
        if (A.ahead > 0) prefetch_stile_l2<DIM, (WHAT & DO_ADJ) != 0>(A, t + A.ahead, lane);
    };
    run_stile<DIM, PREC, WHAT, NTH>(A, t, smem, pf);
}

inline int check_valence(int val_e, int val_v) {
    // A limb plane entry holds the sum of fewer than 1024 limbs of magnitude
    // <= 2^21.  Per element an edge entry receives up to 3 of them (the
    // integer sum -(q1 + q2 + q3) at the edges of node 0) and a boundary face
    // one; a node's gradient entry receives up to 3 per element (node 0) and
    // one per boundary face, of which a node has at most 3 per element.
    if (val_e > 340 || val_v > 170)
        return fail(EM_ERR_ARG, "tiled path: an edge with more than 340 elements or a node with more than 170 "
                                "elements exceeds its fixed-point headroom; use the gather path");
    return EM_OK;
}

template <int DIM, int PREC, int WHAT>
int launch_stiles(const em_mesh* m, SArgs& A, cudaStream_t s) {
    const SmemS L = s_layout<DIM, PREC, WHAT>(A.D);
    static size_t configured = 0;
    EM_TRY(check_valence(A.val_e, A.val_v));
    if (L.total > 227 * 1024)
        return fail(EM_ERR_ARG, "tile needs " + std::to_string(L.total) +
                                    " bytes of shared memory (> 227 KB): rebuild the plan with a smaller tile_nodes");
    if (L.total > 48 * 1024 && L.total > configured) {
        EM_CUDA_TRY(cudaFuncSetAttribute(k_stile<DIM, PREC, WHAT, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         227 * 1024));
        if constexpr (DIM == 3)
            EM_CUDA_TRY(cudaFuncSetAttribute(k_stile<DIM, PREC, WHAT, 2 * NT>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
        configured = 227 * 1024;
    }
    // one resident CTA of NT threads per SM leaves half the register file
    // idle: such tiles run with 2 NT threads (3D; the results do not depend
    // on the thread count)
    bool wide = false;
    int per_sm = 0;
    EM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_stile<DIM, PREC, WHAT, NT>, NT, L.total));
    if constexpr (DIM == 3) {
        if (per_sm < 2) {
            wide = true;
            EM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_stile<DIM, PREC, WHAT, 2 * NT>,
                                                                      2 * NT, L.total));
        }
    }
    // with one CTA per SM nothing hides a tile's staging latency: tile t
    // prefetches the tile that starts after it (tiles resident at once ahead)
    A.ahead = per_sm == 1 ? num_sms() : 0;
    const int64_t n_tiles = A.n_tiles;
    const int64_t chunk = 1 << 30;
    for (int64_t base = 0; base < n_tiles; base += chunk) {
        A.tile_base = base;
        const int64_t nb = n_tiles - base < chunk ? n_tiles - base : chunk;
        if constexpr (DIM == 3) {
            if (wide)
                k_stile<DIM, PREC, WHAT, 2 * NT><<<(unsigned)nb, 2 * NT, L.total, s>>>(A);
            else
                k_stile<DIM, PREC, WHAT, NT><<<(unsigned)nb, NT, L.total, s>>>(A);
        } else {
            k_stile<DIM, PREC, WHAT, NT><<<(unsigned)nb, NT, L.total, s>>>(A);
        }
        note_launches(1);
    }
    // merge the records (none on a grid that fits one tile)
    const int64_t nmerge = m->plan_info[EM_PLAN_INFO_REC_EDGES] + m->plan_info[EM_PLAN_INFO_REC_NODES] +
                           m->plan_info[EM_PLAN_INFO_REC_BNODES];
    if (nmerge > 0) {
        MergeArgs M{A.plan, A.n_out, A.vol, A.bnormal, A.grad, A.rec_e, A.rec_v, A.rec_g, A.rec_b};
        k_merge<DIM, WHAT><<<grid_for(nmerge, NT), NT, 0, s>>>(M);
        note_launches(1);
    }
    EM_CUDA_TRY(cudaGetLastError());
    return EM_OK;
}

template <int DIM, int PREC>
int dispatch_s(const em_mesh* m, int what, SArgs& A, cudaStream_t s) {
    if (what == GATHER_FWD) return launch_stiles<DIM, PREC, DO_FWD>(m, A, s);
    if (what == GATHER_ADJ) return launch_stiles<DIM, PREC, DO_ADJ>(m, A, s);
    return launch_stiles<DIM, PREC, DO_FWD | DO_ADJ>(m, A, s);
}

// records of one grid in a buffer of scatter_rec_bytes(plan_info) bytes (an
// upper bound for both dimensions: 4 doubles per record), packed as
// [edge records][DIM], [node records] (V), [node records][DIM] (grad),
// [boundary-node records][DIM]
inline size_t scatter_rec_bytes(const int64_t* pi) {
    return sizeof(double) * REC_DOUBLES *
           (size_t)(pi[EM_PLAN_INFO_REC_EDGES] + pi[EM_PLAN_INFO_REC_NODES] + pi[EM_PLAN_INFO_REC_BNODES]);
}

__host__ __device__ inline void rec_pointers(const int64_t* pi, int dim, void* base, double** re, double** rv,
                                             double** rg, double** rb) {
    double* p = static_cast<double*>(base);
    *re = p;
    p += dim * pi[EM_PLAN_INFO_REC_EDGES];
    *rv = p;
    p += pi[EM_PLAN_INFO_REC_NODES];
    *rg = p;
    p += dim * pi[EM_PLAN_INFO_REC_NODES];
    *rb = p;
}

// ---- batched: the tiles of many grids in one launch --------------------------
// Work item = (grid, tile), numbered through the grids' tile prefix sums.  Two
// launch shapes run each item through the same scatter tile, and one merge
// launch covers every grid's records, so both give the results of the
// single-grid tiled path bit for bit:
//   item grid (default): one CTA per item, dispatched by the hardware in item
//     order;
//   persistent: a fixed set of CTAs claims items through one atomic counter.
__device__ __forceinline__ void args_from_item(const em_batch_item& it, SArgs& A) {
    A.plan = it.mesh.plan;
    A.x = it.x; A.w = it.w; A.c = it.c;
    A.n_out = it.n_edge; A.vol = it.vol; A.bnormal = it.bnormal; A.grad = it.grad_x;
    rec_pointers(it.mesh.plan_info, it.mesh.dim, it.rec, &A.rec_e, &A.rec_v, &A.rec_g, &A.rec_b);
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
    SArgs B;
    args_from_item(items[g], B);
    prefetch_stile_l2<DIM, true>(B, (int)(nx - pre[g]), lane);
}

// one CTA per work item; `ahead` > 0: prefetch item wk + ahead into L2
template <int DIM, int PREC, int NTH>
__global__ void __launch_bounds__(NTH, (NTH == NT ? scatter_min_ctas<PREC, DO_FWD | DO_ADJ>() : 1))
    k_sbatched_items(const em_batch_item* __restrict__ items, const int64_t* __restrict__ prefix, int n_meshes,
                     SDims D, int32_t* status, int ahead) {
    extern __shared__ __align__(16) char smem[];
    __shared__ SArgs sA;     // the item's arguments, read by every thread
    const int64_t wk = blockIdx.x;
    const int64_t total = prefix[n_meshes];
    if (wk >= total) return;
    const int g = item_grid(prefix, n_meshes, wk);
    const em_batch_item& it = items[g];
    if (it.mesh.dim != DIM) {   // block-uniform
        if (threadIdx.x == 0) atomicExch(status, EM_ERR_ARG);
        return;
    }
    if (threadIdx.x == 0) {
        args_from_item(it, sA);
        sA.D = D;
    }
    __syncthreads();
    auto pf = [&](int lane) {
        if (ahead > 0 && wk + ahead < total) prefetch_item_l2<DIM>(items, prefix, n_meshes, wk + ahead, lane);
    };
    run_stile<DIM, PREC, DO_FWD | DO_ADJ, NTH>(sA, (int)(wk - prefix[g]), smem, pf);
}

// persistent CTAs draining the work list; `prefetch`: prefetch the item
// claimed next into L2
template <int DIM, int PREC, int NTH>
__global__ void __launch_bounds__(NTH, (NTH == NT ? scatter_min_ctas<PREC, DO_FWD | DO_ADJ>() : 1))
    k_sbatched(const em_batch_item* __restrict__ items, const int64_t* __restrict__ prefix, int n_meshes, SDims D,
               unsigned long long* counter, int32_t* status, int prefetch) {
    extern __shared__ __align__(16) char smem[];
    __shared__ long long s_next;
    __shared__ SArgs sA;
    // the tile prefix sums live in shared memory behind the tile's layout
    const SmemS L = s_layout<DIM, PREC, DO_FWD | DO_ADJ>(D);
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
            args_from_item(it, sA);
            sA.D = D;
        }
        __syncthreads();
        // s_next (written before the tile's first barrier) is this block's
        // next item
        auto pf = [&](int lane) {
            const long long nx = s_next;
            if (prefetch && nx < total) prefetch_item_l2<DIM>(items, spre, n_meshes, nx, lane);
        };
        run_stile<DIM, PREC, DO_FWD | DO_ADJ, NTH>(sA, (int)(wk - spre[g]), smem, pf);
        __syncthreads();
    }
}

// the records of every grid: blockIdx.y = grid
template <int DIM>
__global__ void __launch_bounds__(NT) k_sbatched_merge(const em_batch_item* __restrict__ items) {
    const em_batch_item& it = items[blockIdx.y];
    if (it.mesh.dim != DIM) return;
    MergeArgs M;
    M.plan = it.mesh.plan;
    M.n_out = it.n_edge; M.vol = it.vol; M.bnormal = it.bnormal; M.grad = it.grad_x;
    double *re, *rv, *rg, *rb;
    rec_pointers(it.mesh.plan_info, DIM, it.rec, &re, &rv, &rg, &rb);
    M.rec_e = re; M.rec_v = rv; M.rec_g = rg; M.rec_b = rb;
    merge_targets<DIM, DO_FWD | DO_ADJ>(M, blockIdx.x * int64_t(NT) + threadIdx.x, int64_t(gridDim.x) * NT);
}

template <int DIM, int PREC, int NTH>
int launch_sbatched_as(int n_meshes, const em_batch_item* items, const int64_t* prefix, int64_t n_items,
                       const SDims& D, int blocks, int per_sm, size_t bytes, unsigned long long* counter,
                       int32_t* status, cudaStream_t s) {
    if (blocks == 0) {
        // one CTA per item; with one CTA per SM, item wk prefetches the item
        // that starts after it
        const int ahead = per_sm == 1 ? num_sms() : 0;
        EM_CUDA_TRY(cudaFuncSetAttribute(k_sbatched_items<DIM, PREC, NTH>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
        k_sbatched_items<DIM, PREC, NTH><<<(unsigned)n_items, NTH, bytes, s>>>(items, prefix, n_meshes, D, status,
                                                                                ahead);
    } else {
        if (blocks < 0) blocks = num_sms() * (per_sm > 0 ? per_sm : 1);
        EM_CUDA_TRY(cudaFuncSetAttribute(k_sbatched<DIM, PREC, NTH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(bytes + sizeof(int64_t) * (size_t)(n_meshes + 1))));
        k_sbatched<DIM, PREC, NTH><<<blocks, NTH, bytes + sizeof(int64_t) * (size_t)(n_meshes + 1), s>>>(
            items, prefix, n_meshes, D, counter, status, per_sm == 1 ? 1 : 0);
    }
    note_launches(1);
    // every grid's merge in one launch (about 4 CTAs per SM in all)
    const unsigned gx = (unsigned)std::max<int64_t>(1, (4ll * num_sms() + n_meshes - 1) / n_meshes);
    k_sbatched_merge<DIM><<<dim3(gx, (unsigned)n_meshes), NT, 0, s>>>(items);
    note_launches(1);
    EM_CUDA_TRY(cudaGetLastError());
    return EM_OK;
}

template <int DIM, int PREC>
int launch_sbatched(int n_meshes, const em_batch_item* items, const int64_t* prefix, int64_t n_items, const SDims& D,
                    int blocks, unsigned long long* counter, int32_t* status, cudaStream_t s) {
    const SmemS L = s_layout<DIM, PREC, DO_FWD | DO_ADJ>(D);
    const size_t bytes = L.total;
    const size_t need = L.total + (blocks != 0 ? sizeof(int64_t) * (size_t)(n_meshes + 1) : 0);
    if (need > 227 * 1024)
        return fail(EM_ERR_ARG, "batched tiles need " + std::to_string(need) +
                                    " bytes of shared memory (> 227 KB): use a smaller tile_nodes or fewer grids");
    // as for one grid: tiles that fill an SM run with 2 NT threads (3D) and
    // prefetch their next item (the results depend on neither)
    int per_sm = 0;
    EM_CUDA_TRY(cudaFuncSetAttribute(k_sbatched_items<DIM, PREC, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)need));
    EM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sbatched_items<DIM, PREC, NT>, NT, need));
    if constexpr (DIM == 3) {
        if (per_sm < 2) {
            EM_CUDA_TRY(cudaFuncSetAttribute(k_sbatched_items<DIM, PREC, 2 * NT>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need));
            EM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sbatched_items<DIM, PREC, 2 * NT>,
                                                                      2 * NT, need));
            return launch_sbatched_as<DIM, PREC, 2 * NT>(n_meshes, items, prefix, n_items, D, blocks, per_sm, bytes,
                                                         counter, status, s);
        }
    }
    return launch_sbatched_as<DIM, PREC, NT>(n_meshes, items, prefix, n_items, D, blocks, per_sm, bytes, counter,
                                             status, s);
}

}  // namespace

size_t scatter_ws_bytes(const em_mesh* m) { return (scatter_rec_bytes(m->plan_info) + 255) & ~size_t(255); }

int scatter_run(const em_mesh* m, int prec, int what, const double* x, const double* w, const double* c, double* n,
                double* vol, double* bnormal, double* g, void* ws, cudaStream_t s, const BwAux* bw) {
    const int64_t* pi = m->plan_info;
    if (pi[EM_PLAN_INFO_S_MAX_NODES] <= 0 || pi[EM_PLAN_INFO_S_MAX_EDGES] <= 0)
        return fail(EM_ERR_ARG, "mesh->plan_info has no scatter tiles (plan from an older library version?)");
    if (scatter_rec_bytes(pi) && !ws) return fail(EM_ERR_WORKSPACE, "tiled path needs its workspace for records");
    SArgs A;
    A.plan = m->plan;
    A.x = x; A.w = w; A.c = c;
    A.n_out = n; A.vol = vol; A.bnormal = bnormal; A.grad = g;
    rec_pointers(pi, m->dim, ws, &A.rec_e, &A.rec_v, &A.rec_g, &A.rec_b);
    A.D.max_nodes = (int)pi[EM_PLAN_INFO_S_MAX_NODES];
    A.D.max_edges = (int)pi[EM_PLAN_INFO_S_MAX_EDGES];
    A.D.max_bnodes = (int)std::max<int64_t>(pi[EM_PLAN_INFO_S_MAX_BNODES], 1);
    A.n_tiles = (int)pi[EM_PLAN_INFO_TILES];
    A.val_e = (int)(pi[EM_PLAN_INFO_MAX_EDGE_VALENCE] > 0 ? pi[EM_PLAN_INFO_MAX_EDGE_VALENCE] : 64);
    A.val_v = (int)(pi[EM_PLAN_INFO_MAX_NODE_VALENCE] > 0 ? pi[EM_PLAN_INFO_MAX_NODE_VALENCE] : 64);
    A.tile_base = 0;
    A.ahead = 0;
    A.bwa = bw ? *bw : BwAux{nullptr, nullptr, nullptr};
    if (m->dim == 3) {
        if (prec == EM_PREC_FP64) return dispatch_s<3, EM_PREC_FP64>(m, what, A, s);
        if (prec == EM_PREC_DW) return dispatch_s<3, EM_PREC_DW>(m, what, A, s);
        return dispatch_s<3, EM_PREC_MIXED>(m, what, A, s);
    }
    if (prec == EM_PREC_FP64) return dispatch_s<2, EM_PREC_FP64>(m, what, A, s);
    if (prec == EM_PREC_DW) return dispatch_s<2, EM_PREC_DW>(m, what, A, s);
    return dispatch_s<2, EM_PREC_MIXED>(m, what, A, s);
}

int batched_impl(int n_meshes, const em_batch_item* items, const int64_t* tile_prefix, int64_t n_items,
                 const int64_t* max_info, int dim, int precision, int blocks, int32_t* status, void* ws,
                 size_t* ws_bytes, cudaStream_t s) {
    bool query;
    EM_TRY(check_ws(ws, ws_bytes, 256, &query));
    if (query) return EM_OK;
    if (n_meshes <= 0 || n_meshes > 65535 || !items || !tile_prefix || !max_info || !status)
        return fail(EM_ERR_ARG, "batched call needs 1..65535 grids, items, tile_prefix, max_info and status");
    if (n_items <= 0 || n_items > 0x7fffffffLL) return fail(EM_ERR_ARG, "n_items must be in [1, 2^31)");
    if (blocks < EM_BATCH_PERSISTENT) return fail(EM_ERR_ARG, "blocks must be >= EM_BATCH_PERSISTENT (-1)");
    if (dim != 2 && dim != 3) return fail(EM_ERR_ARG, "dim must be 2 or 3");
    if (precision != EM_PREC_FP64 && precision != EM_PREC_DW && precision != EM_PREC_MIXED)
        return fail(EM_ERR_ARG, "batched pass supports FP64, DW and MIXED");
    SDims D;
    D.max_nodes = (int)max_info[EM_PLAN_INFO_S_MAX_NODES];
    D.max_edges = (int)max_info[EM_PLAN_INFO_S_MAX_EDGES];
    D.max_bnodes = (int)std::max<int64_t>(max_info[EM_PLAN_INFO_S_MAX_BNODES], 1);
    if (D.max_nodes <= 0 || D.max_edges <= 0) return fail(EM_ERR_ARG, "max_info has no scatter tiles");
    // each grid's tiles accumulate in exact fixed point
    EM_TRY(check_valence((int)std::min<int64_t>(max_info[EM_PLAN_INFO_MAX_EDGE_VALENCE], 1 << 30),
                         (int)std::min<int64_t>(max_info[EM_PLAN_INFO_MAX_NODE_VALENCE], 1 << 30)));
    unsigned long long* counter = static_cast<unsigned long long*>(ws);
    EM_CUDA_TRY(cudaMemsetAsync(counter, 0, sizeof(unsigned long long), s));
    EM_CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(int32_t), s));
    if (dim == 3) {
        if (precision == EM_PREC_FP64) return launch_sbatched<3, EM_PREC_FP64>(n_meshes, items, tile_prefix, n_items, D, blocks, counter, status, s);
        if (precision == EM_PREC_DW) return launch_sbatched<3, EM_PREC_DW>(n_meshes, items, tile_prefix, n_items, D, blocks, counter, status, s);
        return launch_sbatched<3, EM_PREC_MIXED>(n_meshes, items, tile_prefix, n_items, D, blocks, counter, status, s);
    }
    if (precision == EM_PREC_FP64) return launch_sbatched<2, EM_PREC_FP64>(n_meshes, items, tile_prefix, n_items, D, blocks, counter, status, s);
    if (precision == EM_PREC_DW) return launch_sbatched<2, EM_PREC_DW>(n_meshes, items, tile_prefix, n_items, D, blocks, counter, status, s);
    return launch_sbatched<2, EM_PREC_MIXED>(n_meshes, items, tile_prefix, n_items, D, blocks, counter, status, s);
}

}  // namespace em

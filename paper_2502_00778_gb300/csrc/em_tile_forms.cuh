// Arithmetic shared by the tiled kernels (em_tiled.cu: ordered gather,
// em_scatter.cu: scatter tiles): the three precision forms, the exact
// fixed-point accumulation of the scatter tiles, non-finite helpers and L2
// prefetch hints.
#pragma once
#include "em_common.cuh"
#include "em_dw.cuh"

namespace em {

namespace {

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
    static __device__ __forceinline__ V quarter(V a) { return __dmul_rn(0.25, a); }
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
    static __device__ __forceinline__ V quarter(V a) { return {__fmul_rn(0.25f, a.h), __fmul_rn(0.25f, a.l)}; }
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
    static __device__ __forceinline__ V quarter(V a) { return 0.25f * a; }
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
__device__ __forceinline__ double tile_origin_component(const double* x, int node0, int n_own, int d) {
    double o = x[int64_t(node0) * DIM + d];
    for (int k = 1; !isfinite(o) && k < n_own; k++) o = x[(int64_t(node0) + k) * DIM + d];
    return isfinite(o) ? o : 0.0;
}
template <int DIM>
__device__ __forceinline__ void tile_origin(const double* x, int node0, int n_own, double* org) {
#pragma unroll
    for (int d = 0; d < DIM; d++) org[d] = tile_origin_component<DIM>(x, node0, n_own, d);
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

// round(t*s) for a power of two s (|t*s| < 2^22), as an int, and the exact
// remainder t*s - round(t*s): t*s is exact, so fma(t, s, MAGIC) rounds it as
// t*s + MAGIC would, and fma(t, s, -round) is exact (the scaling costs no
// separate multiply)
__device__ __forceinline__ int fx_round_s(float t, float s, float& rem) {
    const float y = __fmaf_rn(t, s, FX_MAGIC);
    rem = __fmaf_rn(t, s, -__fsub_rn(y, FX_MAGIC));
    return __float_as_int(y) - 0x4B400000;
}
__device__ __forceinline__ int fx_round_last(float t, float s) {   // remainder not needed
    return __float_as_int(__fmaf_rn(t, s, FX_MAGIC)) - 0x4B400000;
}

// -(a + b + c) and x -= q, limb by limb: exact integer sums of quantised
// values (each limb stays within 3 x 2^21)
__device__ __forceinline__ Lq lq_neg_sum(const Lq& a, const Lq& b, const Lq& c) {
    return {-(a.a + b.a + c.a), -(a.b + b.b + c.b), -(a.c + b.c + c.c)};
}
__device__ __forceinline__ void lq_sub(Lq& x, const Lq& q) {
    x.a -= q.a;
    x.b -= q.b;
    x.c -= q.c;
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

// q * 2^-sg as a double, rounded to nearest even, with integer instructions
// only (the int64 -> double conversion instruction runs on the FP64 pipe,
// which the output pass of a tile would otherwise saturate).  |q| < 2^62 and
// sg within the forms' [LO, HI] ranges keep the result a normal double.
// |q| is shifted so that its leading one is bit 63; its upper 53 bits are
// the mantissa, rounded on the 11 bits below; a carry out of the rounding
// (mantissa 2^53) moves into the exponent field through the addition.
__device__ __forceinline__ double fx_to_double(long long q, int sg) {
    if (q == 0) return 0.0;
    const unsigned long long sign = (unsigned long long)q & 0x8000000000000000ull;
    unsigned long long a = q < 0 ? 0ull - (unsigned long long)q : (unsigned long long)q;
    const int lz = __clzll((long long)a);
    a <<= lz;
    unsigned long long m = a >> 11;
    const unsigned rem = (unsigned)(a & 0x7ffull);
    m += (rem > 0x400u || (rem == 0x400u && (m & 1ull))) ? 1ull : 0ull;
    const long long field = 1023 + 63 - lz - sg;   // biased exponent of 2^(63 - lz - sg)
    return __longlong_as_double((long long)((((unsigned long long)(field - 1)) << 52) + m + sign));
}

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

// ---- upper bounds for the fixed-point scales --------------------------------
// A bound m 2^e with a float mantissa m in [1, 2) and an integer exponent, so
// that it covers any double range.  A key gives the bound of the double whose
// upper word follows it (20 mantissa bits, exact in a float); products and
// sums round up.  Taking the exponent of a whole product gives away less than
// one bit, where rounding each factor to a power of two gave away up to one
// bit per factor.  Integer and FP32 instructions only.
struct Ub {
    float m;
    int e;
};

// m >= 1 (a normal float) to [1, 2), adjusting e; exact
__device__ __forceinline__ Ub ub_norm(float m, int e) {
    const unsigned b = __float_as_uint(m);
    const int k = (int)((b >> 23) & 0xffu) - 127;
    return {__uint_as_float(b - ((unsigned)k << 23)), e + k};
}

// above every value whose key is k (k below the key of infinity)
__device__ __forceinline__ Ub ub_key(unsigned k) {
    const unsigned n = k + 1u;
    const int ex = (int)(n >> 20);
    if (ex == 0) return {1.0f, -1022};   // every subnormal double is below 2^-1022
    return {__uint_as_float(0x3f800000u | ((n & 0xfffffu) << 3)), ex - 1023};
}

// a * c for a float c >= 1 (a small integer or 1 + 2^-k: exact)
__device__ __forceinline__ Ub ub_scale(Ub a, float c) { return ub_norm(__fmul_ru(a.m, c), a.e); }
__device__ __forceinline__ Ub ub_mul(Ub a, Ub b) { return ub_norm(__fmul_ru(a.m, b.m), a.e + b.e); }
__device__ __forceinline__ Ub ub_add(Ub a, Ub b) {
    if (a.e < b.e) {
        const Ub t = a;
        a = b;
        b = t;
    }
    const int d = a.e - b.e;
    // b.m 2^-d (exact for d <= 60; 2^-60 bounds it beyond)
    const float bs = d > 60 ? 0x1p-60f : __fmul_ru(b.m, __uint_as_float((unsigned)(127 - d) << 23));
    return ub_norm(__fadd_ru(a.m, bs), a.e);
}
// the least e' with m 2^e < 2^e'
__device__ __forceinline__ int ub_exp(Ub a) { return a.e + 1; }
// the least k with m < 2^k, for a normal float m >= 1
__device__ __forceinline__ int ub_bits(float m) { return (int)((__float_as_uint(m) >> 23) & 0xffu) - 126; }


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
        return sc == 1.0 ? fx_to_double(q, sg) : __dmul_rn(fx_to_double(q, sg), sc);
    }
};

template <>
struct Fix<EM_PREC_DW> {
    // LO, HI: the float powers of two 2^(sg - 42) and 2^(sg - 21) below stay normal
    static constexpr int NL = 3, TOP = 62, LO = -80, HI = 148;
    static __device__ __forceinline__ Lq q(dw v, int sg) {
        float r;
        const int a = fx_round_s(v.h, pow2f(sg - 42), r);
        const int b = fx_round_s(r, 2097152.0f, r);
        const int c = fx_round_last(r, 2097152.0f);
        const int b2 = fx_round_s(v.l, pow2f(sg - 21), r);
        const int c2 = fx_round_last(r, 2097152.0f);
        return {a, b + b2, c + c2};
    }
    static __device__ __forceinline__ unsigned mag(dw v) {
        return mkey(f_to_double((fabsf(v.h) + fabsf(v.l)) * 1.000001f));
    }
    // once per output: the conversion runs on the integer pipe, one DMUL
    // applies the output factor
    static __device__ __forceinline__ double out(long long q, int sg, double sc) {
        return sc == 1.0 ? fx_to_double(q, sg) : __dmul_rn(fx_to_double(q, sg), sc);
    }
};

template <>
struct Fix<EM_PREC_MIXED> {
    static constexpr int NL = 2, TOP = 41, LO = -80, HI = 148;
    static __device__ __forceinline__ Lq q(float v, int sg) {
        float r;
        const int a = fx_round_s(v, pow2f(sg - 21), r);
        return {a, fx_round_last(r, 2097152.0f), 0};
    }
    static __device__ __forceinline__ unsigned mag(float v) { return mkey(f_to_double(v)); }
    static __device__ __forceinline__ double out(long long q, int sg, double sc) {
        return sc == 1.0 ? fx_to_double(q, sg) : __dmul_rn(fx_to_double(q, sg), sc);
    }
};

// block-wide maxima without a cleared slot: each warp writes its maximum to
// its own entry of slot s (16 entries per slot), and readers take the max of
// the entries after a barrier, lane w reading warp w's entry (whole warps
// only: every lane of the warp calls red_max)
constexpr int RED_WARPS = 16;
__device__ __forceinline__ void block_max(unsigned* wred, int s, unsigned v) {
    v = __reduce_max_sync(0xffffffffu, v);
    if ((threadIdx.x & 31) == 0) wred[s * RED_WARPS + (threadIdx.x >> 5)] = v;
}
__device__ __forceinline__ unsigned red_max(const unsigned* wred, int s, int nwarps) {
    const int lane = (int)(threadIdx.x & 31);
    return __reduce_max_sync(0xffffffffu, lane < nwarps ? wred[s * RED_WARPS + lane] : 0u);
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

}  // namespace

}  // namespace em

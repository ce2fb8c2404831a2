// Device primitives: stable LSD radix sort of (u64 key, u32 value) pairs and
// multi-block exclusive scans.  Used by edge_build (64-bit (min,max) edge keys,
// face keys) and by the gather-plan builder.
#include "em_common.cuh"

namespace em {

namespace {

constexpr int SORT_THREADS = 256;
constexpr int SORT_ROUNDS = 16;
constexpr int SORT_TILE = SORT_THREADS * SORT_ROUNDS;  // 4096 pairs per block
constexpr unsigned FULL = 0xffffffffu;

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// block-wide exclusive scan of one value per thread; *total gets the sum
template <typename T>
__device__ T block_exclusive_scan(T v, T* sm, T* total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sm[wid] = x;
    __syncthreads();
    if (wid == 0) {
        T s = lane < nw ? sm[lane] : T(0);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(FULL, s, o);
            if (lane >= o) s += y;
        }
        if (lane < nw) sm[lane] = s;
    }
    __syncthreads();
    T excl = (wid ? sm[wid - 1] : T(0)) + x - v;
    *total = sm[nw - 1];
    __syncthreads();
    return excl;
}

template <typename Tin, typename Tout>
__global__ void k_scan_block_sums(const Tin* __restrict__ in, int64_t n, Tout* __restrict__ bsum) {
    __shared__ Tout sm[32];
    int64_t base = int64_t(blockIdx.x) * SCAN_TILE + threadIdx.x * SCAN_ITEMS;
    Tout s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; i++)
        if (base + i < n) s += Tout(in[base + i]);
    Tout tot;
    block_exclusive_scan<Tout>(s, sm, &tot);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

// single block: exclusive scan of nb block sums in place, total in bsum[nb]
template <typename Tout>
__global__ void k_scan_top(Tout* bsum, int64_t nb) {
    __shared__ Tout sm[32];
    Tout carry = 0;
    for (int64_t off = 0; off < nb; off += SCAN_THREADS) {
        int64_t i = off + threadIdx.x;
        Tout v = i < nb ? bsum[i] : Tout(0);
        Tout tot;
        Tout ex = block_exclusive_scan<Tout>(v, sm, &tot);
        if (i < nb) bsum[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) bsum[nb] = carry;
}

template <typename Tin, typename Tout>
__global__ void k_scan_apply(const Tin* __restrict__ in, int64_t n, const Tout* __restrict__ bsum,
                             Tout* __restrict__ out, int64_t nb) {
    __shared__ Tout sm[32];
    int64_t base = int64_t(blockIdx.x) * SCAN_TILE + threadIdx.x * SCAN_ITEMS;
    Tout v[SCAN_ITEMS];
    Tout s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; i++) {
        v[i] = (base + i < n) ? Tout(in[base + i]) : Tout(0);
        s += v[i];
    }
    Tout tot;
    Tout ex = block_exclusive_scan<Tout>(s, sm, &tot) + bsum[blockIdx.x];
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; i++) {
        if (base + i < n) out[base + i] = ex;
        ex += v[i];
    }
    if (blockIdx.x == nb - 1 && threadIdx.x == 0) out[n] = bsum[nb];
}

template <typename Tin, typename Tout>
int scan_impl(const Tin* in, Tout* out, int64_t n, void* ws, cudaStream_t s) {
    if (n <= 0) {
        EM_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(Tout), s));
        return EM_OK;
    }
    int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    Tout* bsum = static_cast<Tout*>(ws);
    k_scan_block_sums<Tin, Tout><<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, n, bsum);
    k_scan_top<Tout><<<1, SCAN_THREADS, 0, s>>>(bsum, nb);
    k_scan_apply<Tin, Tout><<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, n, bsum, out, nb);
    EM_CUDA_TRY(cudaGetLastError());
    return EM_OK;
}

// ---- radix sort ----------------------------------------------------------

__global__ void k_radix_hist(const uint64_t* __restrict__ keys, int64_t n, int shift, unsigned mask,
                             uint32_t* __restrict__ hist, int64_t ntiles) {
    __shared__ uint32_t h[256];
    for (int d = threadIdx.x; d < 256; d += blockDim.x) h[d] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    int64_t t0 = int64_t(blockIdx.x) * SORT_TILE;
    for (int r = 0; r < SORT_ROUNDS; r++) {
        int64_t i = t0 + r * SORT_THREADS + threadIdx.x;
        unsigned d = i < n ? unsigned((keys[i] >> shift) & mask) : 0xffffffffu;
        unsigned peers = __match_any_sync(FULL, d);
        if (d != 0xffffffffu && lane == __ffs(peers) - 1) atomicAdd(&h[d], (uint32_t)__popc(peers));
    }
    __syncthreads();
    for (int d = threadIdx.x; d < 256; d += blockDim.x) hist[int64_t(d) * ntiles + blockIdx.x] = h[d];
}

__global__ void k_radix_scatter(const uint64_t* __restrict__ kin, const uint32_t* __restrict__ vin,
                                uint64_t* __restrict__ kout, uint32_t* __restrict__ vout, int64_t n, int shift,
                                unsigned mask, const uint32_t* __restrict__ offs, int64_t ntiles) {
    __shared__ uint32_t cnt[SORT_THREADS / 32][256];
    __shared__ uint32_t run[256];
    __shared__ uint32_t base[256];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int d = threadIdx.x; d < 256; d += blockDim.x) {
        run[d] = 0;
        base[d] = offs[int64_t(d) * ntiles + blockIdx.x];
    }
    int64_t t0 = int64_t(blockIdx.x) * SORT_TILE;
    const unsigned lt = lanemask_lt();
    for (int r = 0; r < SORT_ROUNDS; r++) {
        uint32_t* cf = &cnt[0][0];
        for (int k = threadIdx.x; k < (SORT_THREADS / 32) * 256; k += blockDim.x) cf[k] = 0;
        __syncthreads();
        int64_t i = t0 + r * SORT_THREADS + threadIdx.x;
        bool valid = i < n;
        uint64_t key = valid ? kin[i] : 0;
        uint32_t val = valid ? vin[i] : 0;
        unsigned d = valid ? unsigned((key >> shift) & mask) : 0xffffffffu;
        unsigned peers = __match_any_sync(FULL, d);
        unsigned rank = __popc(peers & lt);
        if (valid && rank == 0) cnt[w][d] = __popc(peers);
        __syncthreads();
        if (valid) {
            uint32_t pre = run[d];
            for (int q = 0; q < w; q++) pre += cnt[q][d];
            uint32_t dst = base[d] + pre + rank;
            kout[dst] = key;
            vout[dst] = val;
        }
        __syncthreads();
        for (int dd = threadIdx.x; dd < 256; dd += blockDim.x) {
            uint32_t s = 0;
#pragma unroll
            for (int q = 0; q < SORT_THREADS / 32; q++) s += cnt[q][dd];
            run[dd] += s;
        }
        __syncthreads();
    }
}

}  // namespace

size_t scan_ws_bytes(int64_t n) {
    int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    return size_t(nb + 1) * sizeof(int64_t) + 256;
}

int exclusive_scan_i32_to_i64(const int32_t* in, int64_t* out, int64_t n, void* ws, cudaStream_t s) {
    return scan_impl<int32_t, int64_t>(in, out, n, ws, s);
}

size_t radix_sort_ws_bytes(int64_t n) {
    int64_t ntiles = (n + SORT_TILE - 1) / SORT_TILE;
    WsLayout L(nullptr);
    L.take<uint32_t>(size_t(ntiles) * 256 + 1);          // histograms
    L.take<uint32_t>(size_t(ntiles) * 256 + 1);          // offsets
    L.take<char>(scan_ws_bytes(ntiles * 256));           // scan scratch
    return L.bytes();
}

int radix_sort_pairs(uint64_t* keys, uint32_t* vals, uint64_t* kt, uint32_t* vt, int64_t n, int nbits,
                     void* ws, cudaStream_t s) {
    if (n <= 1 || nbits <= 0) return EM_OK;
    int64_t ntiles = (n + SORT_TILE - 1) / SORT_TILE;
    WsLayout L(ws);
    uint32_t* hist = L.take<uint32_t>(size_t(ntiles) * 256 + 1);
    uint32_t* offs = L.take<uint32_t>(size_t(ntiles) * 256 + 1);
    void* sws = L.take<char>(scan_ws_bytes(ntiles * 256));
    uint64_t *ka = keys, *kb = kt;
    uint32_t *va = vals, *vb = vt;
    int passes = 0;
    for (int shift = 0; shift < nbits; shift += 8) {
        int bits = nbits - shift < 8 ? nbits - shift : 8;
        unsigned mask = (1u << bits) - 1;
        k_radix_hist<<<(unsigned)ntiles, SORT_THREADS, 0, s>>>(ka, n, shift, mask, hist, ntiles);
        EM_TRY((scan_impl<uint32_t, uint32_t>(hist, offs, ntiles * 256, sws, s)));
        k_radix_scatter<<<(unsigned)ntiles, SORT_THREADS, 0, s>>>(ka, va, kb, vb, n, shift, mask, offs, ntiles);
        EM_CUDA_TRY(cudaGetLastError());
        uint64_t* tk = ka; ka = kb; kb = tk;
        uint32_t* tv = va; va = vb; vb = tv;
        passes++;
    }
    if (passes & 1) {
        EM_CUDA_TRY(cudaMemcpyAsync(keys, ka, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, s));
        EM_CUDA_TRY(cudaMemcpyAsync(vals, va, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, s));
    }
    return EM_OK;
}

}  // namespace em

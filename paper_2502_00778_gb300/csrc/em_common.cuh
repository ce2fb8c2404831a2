// Shared host/device helpers of the edge-metrics library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>
#include <string>

#include "../../include/edgemetrics.h"

// ---------------------------------------------------------------------------
// host-side error state (thread-local, reported by em_last_error)
// ---------------------------------------------------------------------------
namespace em {

void set_error(int code, const std::string& msg);
int fail(int code, const std::string& msg);          // set_error + return code

#define EM_CUDA_TRY(expr)                                                                   \
    do {                                                                                    \
        cudaError_t _e = (expr);                                                            \
        if (_e != cudaSuccess)                                                              \
            return ::em::fail(EM_ERR_CUDA, std::string(#expr " failed: ") + cudaGetErrorString(_e)); \
    } while (0)

#define EM_TRY(expr)                 \
    do {                             \
        int _s = (expr);             \
        if (_s != EM_OK) return _s;  \
    } while (0)

// launch bookkeeping for em_kernel_launches()
void note_launches(int k);

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// Carves 256-byte-aligned sub-buffers out of one caller workspace.  With a
// null base it only measures.
struct WsLayout {
    char* base;
    size_t off;
    explicit WsLayout(void* b) : base(static_cast<char*>(b)), off(0) {}
    template <typename T>
    T* take(size_t count) {
        off = (off + 255) & ~size_t(255);
        T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
        off += count * sizeof(T);
        return p;
    }
    size_t bytes() const { return (off + 255) & ~size_t(255); }
};

// Workspace protocol shared by all entry points: size query with ws == NULL.
inline int check_ws(void* ws, size_t* ws_bytes, size_t need, bool* query) {
    if (!ws_bytes) return fail(EM_ERR_ARG, "ws_bytes must not be NULL");
    if (!ws) { *ws_bytes = need; *query = true; return EM_OK; }
    *query = false;
    if (*ws_bytes < need)
        return fail(EM_ERR_WORKSPACE, "workspace too small: need " + std::to_string(need) + " bytes, got " +
                                          std::to_string(*ws_bytes));
    if (reinterpret_cast<uintptr_t>(ws) & 255) return fail(EM_ERR_WORKSPACE, "workspace must be 256-byte aligned");
    return EM_OK;
}

inline unsigned grid_for(int64_t n, int threads, int64_t cap = 152 * 64) {
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return (unsigned)b;
}

inline int num_sms() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 152;
    }
    return sms;
}

// ---------------------------------------------------------------------------
// primitives (em_sort.cu)
// ---------------------------------------------------------------------------

// Stable LSD radix sort of (key, value) pairs on the low `nbits` key bits.
// keys/vals are sorted in place; kt/vt are scratch buffers of the same size.
size_t radix_sort_ws_bytes(int64_t n);
int radix_sort_pairs(uint64_t* keys, uint32_t* vals, uint64_t* kt, uint32_t* vt, int64_t n, int nbits,
                     void* ws, cudaStream_t s);

// Exclusive prefix sum of int32 counts into int64 offsets; out[n] = total.
size_t scan_ws_bytes(int64_t n);
int exclusive_scan_i32_to_i64(const int32_t* in, int64_t* out, int64_t n, void* ws, cudaStream_t s);

inline int bits_for(int64_t maxval) {  // bits needed to represent values 0..maxval
    int b = 1;
    while (b < 63 && (int64_t(1) << b) <= maxval) b++;
    return b;
}

}  // namespace em

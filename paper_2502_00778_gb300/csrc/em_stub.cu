// Placeholders for entry points not yet built.
#include "em_common.cuh"
#include "em_kernels.cuh"
namespace em {
size_t csr_fwd_ws_bytes(const em_mesh*) { return 0; }
int csr_fwd(const em_mesh*, const double*, double*, double*, double*, void*, cudaStream_t) {
    return fail(EM_ERR_ARG, "CSR path not available");
}
int batched_impl(int, const em_batch_item*, const int64_t*, int, int, int32_t*, void*, size_t*, cudaStream_t) {
    return fail(EM_ERR_ARG, "batched path not available");
}
}  // namespace em

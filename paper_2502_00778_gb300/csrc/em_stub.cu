// Placeholders for entry points not yet built.
#include "em_common.cuh"
#include "em_kernels.cuh"
namespace em {
int batched_impl(int, const em_batch_item*, const int64_t*, int, int, int32_t*, void*, size_t*, cudaStream_t) {
    return fail(EM_ERR_ARG, "batched path not available");
}
}  // namespace em

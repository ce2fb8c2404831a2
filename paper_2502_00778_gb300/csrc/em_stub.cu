// Placeholders for entry points not yet built.
#include "em_common.cuh"
#include "em_kernels.cuh"
namespace em {
}  // namespace em

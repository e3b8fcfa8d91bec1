// kernels_batch_d9.cu -- batched-job kernels for d = 9, 10 (see batch_impl.cuh).
#include "batch_impl.cuh"

namespace hdmd {
HDMD_BATCH_INSTANTIATE(9)
HDMD_BATCH_INSTANTIATE(10)
}  // namespace hdmd

// kernels_batch_d4.cu -- batched-job kernels for d = 4, 5 (see batch_impl.cuh).
#include "batch_impl.cuh"

namespace hdmd {
HDMD_BATCH_INSTANTIATE(4)
HDMD_BATCH_INSTANTIATE(5)
}  // namespace hdmd

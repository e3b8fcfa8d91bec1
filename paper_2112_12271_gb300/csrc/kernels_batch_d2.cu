// kernels_batch_d2.cu -- batched-job kernels for d = 2, 3 (see batch_impl.cuh).
#include "batch_impl.cuh"

namespace hdmd {
HDMD_BATCH_INSTANTIATE(2)
HDMD_BATCH_INSTANTIATE(3)
}  // namespace hdmd

// kernels_batch_lo.cu -- batched-job kernels for d = 2..5 (see batch_impl.cuh).
#include "batch_impl.cuh"

namespace hdmd {
HDMD_BATCH_INSTANTIATE(2)
HDMD_BATCH_INSTANTIATE(3)
HDMD_BATCH_INSTANTIATE(4)
HDMD_BATCH_INSTANTIATE(5)
}  // namespace hdmd

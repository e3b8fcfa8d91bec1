// kernels_batch_d6.cu -- batched-job kernels for d = 6..7 (see batch_impl.cuh).
#include "batch_impl.cuh"

namespace hdmd {
HDMD_BATCH_INSTANTIATE(6)
HDMD_BATCH_INSTANTIATE(7)
}  // namespace hdmd

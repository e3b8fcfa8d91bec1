// kernels_batch_d8.cu -- batched-job kernels for d = 8 (see batch_impl.cuh).
#include "batch_impl.cuh"

namespace hdmd {
HDMD_BATCH_INSTANTIATE(8)
}  // namespace hdmd

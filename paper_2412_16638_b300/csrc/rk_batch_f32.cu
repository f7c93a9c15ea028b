// Batched-step kernels for f32 storage (one translation unit per storage type
// so the kernel instantiations compile in parallel).
#define RK_BATCH_INSTANTIATE
#include "rk_batch.cuh"

namespace rk {
template rk_status batch_group_run<float>(rk_problem**, int, double, int, cudaStream_t, int, BatchTotals*);
}  // namespace rk

// Batched-step kernels for f32 storage (one translation unit per storage type
// so the large kernel instantiations compile in parallel).
#define RK_BATCH_INSTANTIATE
#include "rk_batch.cuh"

namespace rk {
template int batch_grid_s<float>(int, const LaunchCfg&, int, int);
template void batch_launch_s<float>(int, const LaunchCfg&, int, BatchItem*, const int*, int, double, int*, cudaStream_t);
}  // namespace rk

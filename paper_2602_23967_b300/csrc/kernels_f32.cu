// kernels_f32.cu — setup and solve kernels with float matrix values and float vectors.
#include "kernels_impl.cuh"

namespace pdhcg {
PDHCG_INSTANTIATE(float, float)
template cudaError_t launch_sell_fill<float>(int, const int32_t*, const int64_t*, const int32_t*,
                                               const float*, float*, cudaStream_t);
template cudaError_t launch_sell_fill_batch<float>(const FillDesc*, int, cudaStream_t);
}  // namespace pdhcg

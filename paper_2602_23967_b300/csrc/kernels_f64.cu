// kernels_f64.cu — setup and solve kernels with double matrix values and double vectors.
#include "kernels_impl.cuh"

namespace pdhcg {
PDHCG_INSTANTIATE(double, double)
template cudaError_t launch_sell_fill<double>(int, const int32_t*, const int64_t*, const int32_t*,
                                               const double*, double*, cudaStream_t);
template cudaError_t launch_sell_fill_batch<double>(const FillDesc*, int, cudaStream_t);
}  // namespace pdhcg

// kernels_f64.cu — setup and solve kernels with double matrix values and double vectors.
#include "kernels_impl.cuh"

namespace pdhcg {
PDHCG_INSTANTIATE(double, double)
}  // namespace pdhcg

// kernels_mixed.cu — setup and solve kernels with float matrix values and double vectors.
#include "kernels_impl.cuh"

namespace pdhcg {
PDHCG_INSTANTIATE(float, double)
}  // namespace pdhcg

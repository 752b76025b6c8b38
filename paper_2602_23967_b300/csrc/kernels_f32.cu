// kernels_f32.cu — setup and solve kernels with float matrix values and float vectors.
#include "kernels_impl.cuh"

namespace pdhcg {
PDHCG_INSTANTIATE(float, float)
}  // namespace pdhcg

// kernels_dfloat.cu — setup and solve kernels with float matrix values and
// double-float vectors.
#include "kernels_impl.cuh"

namespace pdhcg {
PDHCG_INSTANTIATE(float, dfloat)
}  // namespace pdhcg

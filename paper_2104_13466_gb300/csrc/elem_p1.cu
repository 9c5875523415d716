// Element kernels instantiated for polynomial order P = 1.
#include "elem_adjoint.cuh"

namespace sdme {
SDME_INSTANTIATE_ORDER(1)
SDME_INSTANTIATE_ADJOINT(1)
}  // namespace sdme

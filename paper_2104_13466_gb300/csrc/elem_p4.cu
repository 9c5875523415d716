// Element kernels instantiated for polynomial order P = 4.
#include "elem_adjoint.cuh"

namespace sdme {
SDME_INSTANTIATE_ORDER(4)
SDME_INSTANTIATE_ADJOINT(4)
}  // namespace sdme

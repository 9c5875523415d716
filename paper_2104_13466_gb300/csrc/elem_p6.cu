// Element kernels instantiated for polynomial order P = 6.
#include "batch_elem.cuh"
#include "cond_columns.cuh"
#include "elem_adjoint.cuh"
#include "quad_launch.cuh"

namespace sdme {
SDME_INSTANTIATE_ORDER(6)
SDME_INSTANTIATE_ADJOINT(6)
SDME_INSTANTIATE_BATCH(6)
SDME_INSTANTIATE_COND(6)
}  // namespace sdme

// Element kernels instantiated for polynomial order P = 3.
#include "batch_elem.cuh"
#include "cond_columns.cuh"
#include "elem_adjoint.cuh"
#include "quad_launch.cuh"

namespace sdme {
SDME_INSTANTIATE_ORDER(3)
SDME_INSTANTIATE_ADJOINT(3)
SDME_INSTANTIATE_BATCH(3)
SDME_INSTANTIATE_COND(3)
}  // namespace sdme

// Element kernels instantiated for polynomial order P = 2.
#include "batch_elem.cuh"
#include "cond_columns.cuh"
#include "elem_adjoint.cuh"
#include "quad_launch.cuh"

namespace sdme {
SDME_INSTANTIATE_ORDER(2)
SDME_INSTANTIATE_ADJOINT(2)
SDME_INSTANTIATE_BATCH(2)
SDME_INSTANTIATE_COND(2)
}  // namespace sdme

// Element kernels instantiated for polynomial order P = 1.
#include "batch_elem.cuh"
#include "cond_columns.cuh"
#include "elem_adjoint.cuh"
#include "quad_launch.cuh"

namespace sdme {
SDME_INSTANTIATE_ORDER(1)
SDME_INSTANTIATE_ADJOINT(1)
SDME_INSTANTIATE_BATCH(1)
SDME_INSTANTIATE_COND(1)
}  // namespace sdme

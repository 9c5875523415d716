// Element kernels instantiated for polynomial order P = 5.
#include "batch_elem.cuh"
#include "cond_columns.cuh"
#include "elem_adjoint.cuh"
#include "quad_launch.cuh"

namespace sdme {
SDME_INSTANTIATE_ORDER(5)
SDME_INSTANTIATE_ADJOINT(5)
SDME_INSTANTIATE_BATCH(5)
SDME_INSTANTIATE_COND(5)
}  // namespace sdme

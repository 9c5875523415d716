// Element kernels instantiated for polynomial order P = 7.
#include "batch_elem.cuh"
#include "cond_columns.cuh"
#include "elem_adjoint.cuh"
#include "quad_launch.cuh"

namespace sdme {
SDME_INSTANTIATE_ORDER(7)
SDME_INSTANTIATE_ADJOINT(7)
SDME_INSTANTIATE_BATCH(7)
SDME_INSTANTIATE_COND(7)
}  // namespace sdme

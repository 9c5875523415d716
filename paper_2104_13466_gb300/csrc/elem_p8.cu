// Element kernels instantiated for polynomial order P = 8.
#include "batch_elem.cuh"
#include "cond_columns.cuh"
#include "elem_adjoint.cuh"
#include "quad_launch.cuh"

namespace sdme {
SDME_INSTANTIATE_ORDER(8)
SDME_INSTANTIATE_ADJOINT(8)
SDME_INSTANTIATE_BATCH(8)
SDME_INSTANTIATE_COND(8)
}  // namespace sdme

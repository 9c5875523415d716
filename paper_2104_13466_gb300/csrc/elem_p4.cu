// Element kernels instantiated for polynomial order P = 4.
#include "batch_elem.cuh"
#include "cond_columns.cuh"
#include "elem_adjoint.cuh"
#include "quad_launch.cuh"

namespace sdme {
SDME_INSTANTIATE_ORDER(4)
SDME_INSTANTIATE_ADJOINT(4)
SDME_INSTANTIATE_BATCH(4)
SDME_INSTANTIATE_COND(4)
}  // namespace sdme

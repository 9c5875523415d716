// Element kernels instantiated for polynomial order P = 1.
#include "elem_launch.cuh"

namespace sdme {
SDME_INSTANTIATE_ORDER(1)
}  // namespace sdme

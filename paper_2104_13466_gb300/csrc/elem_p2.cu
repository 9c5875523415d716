// Element kernels instantiated for polynomial order P = 2.
#include "elem_launch.cuh"

namespace sdme {
SDME_INSTANTIATE_ORDER(2)
}  // namespace sdme

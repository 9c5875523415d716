// Element kernels instantiated for polynomial order P = 3.
#include "elem_launch.cuh"

namespace sdme {
SDME_INSTANTIATE_ORDER(3)
}  // namespace sdme

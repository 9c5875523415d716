// Element kernels instantiated for polynomial order P = 7.
#include "elem_launch.cuh"

namespace sdme {
SDME_INSTANTIATE_ORDER(7)
}  // namespace sdme

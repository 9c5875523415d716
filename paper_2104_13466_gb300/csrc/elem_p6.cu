// Element kernels instantiated for polynomial order P = 6.
#include "elem_launch.cuh"

namespace sdme {
SDME_INSTANTIATE_ORDER(6)
}  // namespace sdme

// Element kernels instantiated for polynomial order P = 8.
#include "elem_launch.cuh"

namespace sdme {
SDME_INSTANTIATE_ORDER(8)
}  // namespace sdme

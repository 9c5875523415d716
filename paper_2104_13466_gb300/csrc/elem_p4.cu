// Element kernels instantiated for polynomial order P = 4.
#include "elem_launch.cuh"

namespace sdme {
SDME_INSTANTIATE_ORDER(4)
}  // namespace sdme

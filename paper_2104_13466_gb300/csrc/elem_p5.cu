// Element kernels instantiated for polynomial order P = 5.
#include "elem_launch.cuh"

namespace sdme {
SDME_INSTANTIATE_ORDER(5)
}  // namespace sdme

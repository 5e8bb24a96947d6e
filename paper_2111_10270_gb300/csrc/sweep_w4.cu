// Sweep kernel instantiations for BDDs of layer width <= 4.
#include "sweep.cuh"

namespace fdog {
FDOG_DEFINE_SWEEP_WIDTH(4, true)
}  // namespace fdog

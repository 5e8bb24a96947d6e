// Sweep kernel instantiations for BDDs of layer width <= 8.
#include "sweep.cuh"

namespace fdog {
FDOG_DEFINE_SWEEP_WIDTH(8, false)
}  // namespace fdog

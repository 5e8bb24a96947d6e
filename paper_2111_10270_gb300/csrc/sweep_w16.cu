// Sweep kernel instantiations for BDDs of layer width <= 16.
#include "sweep.cuh"

namespace fdog {
FDOG_DEFINE_SWEEP_WIDTH(16, false)
}  // namespace fdog

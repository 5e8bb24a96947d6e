// Sweep kernel instantiations for BDDs of layer width <= 2.
#include "sweep.cuh"

namespace fdog {
FDOG_DEFINE_SWEEP_WIDTH(2, true)
}  // namespace fdog

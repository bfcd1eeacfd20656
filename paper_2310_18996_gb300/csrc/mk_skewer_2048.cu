// The fused skewer kernel and the statistics kernel for FFT length 2048.
#include "mk_skewer_unit.cuh"

namespace mk {
template struct SkewerUnit<2048>;
}  // namespace mk

// The fused skewer kernel and the statistics kernel for FFT length 512.
#include "mk_skewer_unit.cuh"

namespace mk {
template struct SkewerUnit<512>;
}  // namespace mk

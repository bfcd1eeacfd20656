// The fused skewer kernel and the statistics kernel for FFT length 256.
#include "mk_skewer_unit.cuh"

namespace mk {
template struct SkewerUnit<256>;
}  // namespace mk

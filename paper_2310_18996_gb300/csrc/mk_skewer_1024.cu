// The fused skewer kernel and the statistics kernel for FFT length 1024.
#include "mk_skewer_unit.cuh"

namespace mk {
template struct SkewerUnit<1024>;
}  // namespace mk

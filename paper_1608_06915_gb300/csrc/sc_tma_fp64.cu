// TMA stream-collide instantiated for double storage (own translation unit for build parallelism).
#include "sc_tma.cuh"

namespace lbmk {
LBM_SC_DEFINE(fp64, double, double)
}  // namespace lbmk

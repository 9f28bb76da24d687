// TMA stream-collide instantiated for float storage (own translation unit for build parallelism).
#include "sc_tma.cuh"

namespace lbmk {
LBM_SC_DEFINE(fp32, float, float)
}  // namespace lbmk

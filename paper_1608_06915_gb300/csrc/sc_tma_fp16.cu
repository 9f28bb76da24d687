// TMA stream-collide instantiated for __half storage (own translation unit for build parallelism).
#include "sc_tma.cuh"

namespace lbmk {
LBM_SC_DEFINE(fp16, __half, float)
}  // namespace lbmk

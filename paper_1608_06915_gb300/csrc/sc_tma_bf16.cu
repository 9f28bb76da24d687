// TMA stream-collide instantiated for __nv_bfloat16 storage (own translation unit for build parallelism).
#include "sc_tma.cuh"

namespace lbmk {
LBM_SC_DEFINE(bf16, __nv_bfloat16, float)
}  // namespace lbmk

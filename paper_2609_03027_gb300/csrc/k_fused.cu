// Fused FP32 path (placeholder until the fused kernel lands).
#include "epic_internal.h"

namespace epic {
epic_status fused_setup(epic_plan_s* p)
{
    p->last_error = "fused FP32 path not built yet";
    return EPIC_ERR_UNSUPPORTED;
}
epic_status fused_run(epic_plan_s*, const uint8_t*, int, cudaStream_t, float*, bool) { return EPIC_ERR_UNSUPPORTED; }
}  // namespace epic

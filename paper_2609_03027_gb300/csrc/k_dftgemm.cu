// Tensor-core DFT-as-GEMM path (placeholder until the tcgen05 kernel lands).
#include "epic_internal.h"

namespace epic {
epic_status dftgemm_setup(epic_plan_s* p)
{
    p->last_error = "DFT-GEMM path not built yet";
    return EPIC_ERR_UNSUPPORTED;
}
epic_status dftgemm_run(epic_plan_s*, const uint8_t*, int, cudaStream_t, float*, bool) { return EPIC_ERR_UNSUPPORTED; }
}  // namespace epic

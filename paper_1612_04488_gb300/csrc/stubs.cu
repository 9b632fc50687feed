// Placeholder for the tensor-core operator until fsm_tc.cu provides it.
#include "lbe_internal.h"
#include "sweep.h"

namespace lbe {
lbe_status tc_apply_L(Ctx* c, DevTables*, int, const double*, const float*, float*, float*, cudaStream_t) {
    c->last_error = "BF16 tensor-core operator not built";
    return LBE_UNSUPPORTED;
}
}  // namespace lbe

// Temporary entry points for the tensor-core path, the refinement driver and the service.
#include "lbe_internal.h"
#include "sweep.h"

namespace lbe {
lbe_status tc_apply_L(Ctx* c, DevTables*, int, const double*, const float*, float*, float*, cudaStream_t) {
    c->last_error = "BF16 tensor-core operator not built";
    return LBE_UNSUPPORTED;
}
void stop_service(Ctx*) {}
}  // namespace lbe

extern "C" {
lbe_status lbe_submit(lbe_ctx*, const lbe_problem*, uint64_t*) { return LBE_UNSUPPORTED; }
lbe_status lbe_poll(lbe_ctx*, uint64_t, lbe_result*, int*) { return LBE_UNSUPPORTED; }
lbe_status lbe_set_max_active(lbe_ctx*, int) { return LBE_UNSUPPORTED; }
}

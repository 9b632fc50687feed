// The fast-spectral operator (fsm_cc_kernels.cuh) instantiated in FP32 arithmetic.
#include "fsm_cc_kernels.cuh"

namespace lbe {

void init_twiddles_f32() { upload_twiddles(); }

template lbe_status fsm_cc_apply<float>(const DevTables&, int, const double*, const float*, float*, float*, void*, int,
                                     cudaStream_t, int);

}  // namespace lbe

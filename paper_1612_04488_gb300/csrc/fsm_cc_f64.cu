// The fast-spectral operator (fsm_cc_kernels.cuh) instantiated in FP64 arithmetic.
#include "fsm_cc_kernels.cuh"

namespace lbe {

void init_twiddles_f64() { upload_twiddles(); }

template lbe_status fsm_cc_apply<double>(const DevTables&, int, const double*, const double*, double*, double*, void*, int,
                                     cudaStream_t, int);

}  // namespace lbe

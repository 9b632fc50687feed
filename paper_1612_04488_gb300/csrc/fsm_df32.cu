// The double-float fast-spectral operator (fsm_cc_kernels.cuh) for the 32-point grid.
#include "fsm_cc_kernels.cuh"

namespace lbe {

void init_twiddles_df32() { upload_twiddles(); }

template void run_fsm_df<32>(const DevTables&, int, const double*, const double*, dfloat*, dfloat*, dfloat2*,
                             dfloat2*, int, int, cudaStream_t);

}  // namespace lbe

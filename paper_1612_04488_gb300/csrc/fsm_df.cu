// The fast-spectral operator (fsm_cc_kernels.cuh) in double-float arithmetic on double data
// (LBE_DF32), grids 8, 16 and 24; the 32-point grid is instantiated in fsm_df32.cu.
#include "fsm_cc_kernels.cuh"

namespace lbe {

void init_twiddles_df() { upload_twiddles(); }

template void run_fsm_df<8>(const DevTables&, int, const double*, const double*, dfloat*, dfloat*, dfloat2*,
                            dfloat2*, int, int, cudaStream_t);
template void run_fsm_df<16>(const DevTables&, int, const double*, const double*, dfloat*, dfloat*, dfloat2*,
                             dfloat2*, int, int, cudaStream_t);
template void run_fsm_df<24>(const DevTables&, int, const double*, const double*, dfloat*, dfloat*, dfloat2*,
                             dfloat2*, int, int, cudaStream_t);

namespace {
// in place: the 8 bytes of a double-float become the double hi + lo
__global__ void k_df_to_double(double* __restrict__ x, long n) {
    for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < n; k += (long)gridDim.x * blockDim.x) {
        const dfloat v = reinterpret_cast<const dfloat*>(x)[k];
        x[k] = (double)v;
    }
}
}  // namespace

// The operator in double-float arithmetic on double data: h is read as double and rounded to
// a double-float on load; Lplus and Lout (double arrays) first receive double-floats, which
// a last pass widens in place.  Scratch as for the double path (8-byte elements).
lbe_status fsm_df_apply(const DevTables& t, int cells, const double* delta, const double* h, double* Lplus,
                        double* Lout, void* scratch, int chunk, cudaStream_t s, int mode) {
    const long n3 = (long)t.nv * t.nv * t.nv;
    if (mode == 2 && t.sym_reps2 == 0) mode = t.sym_reps1 ? 1 : 0;
    if (mode == 1 && t.sym_reps1 == 0) mode = 0;
    if (mode != 0 && (!Lplus || !Lout)) return LBE_INTERNAL;
    if (!t.mult_x) return LBE_INTERNAL;
    auto* Hbuf = (dfloat2*)scratch;
    dfloat2* Ybuf = Hbuf + n3 * cells;
    auto* lp = reinterpret_cast<dfloat*>(Lplus);
    auto* lo = reinterpret_cast<dfloat*>(Lout);
    switch (t.nv) {
        case 8: run_fsm_df<8>(t, cells, delta, h, lp, lo, Hbuf, Ybuf, chunk, mode, s); break;
        case 16: run_fsm_df<16>(t, cells, delta, h, lp, lo, Hbuf, Ybuf, chunk, mode, s); break;
        case 24: run_fsm_df<24>(t, cells, delta, h, lp, lo, Hbuf, Ybuf, chunk, mode, s); break;
        case 32: run_fsm_df<32>(t, cells, delta, h, lp, lo, Hbuf, Ybuf, chunk, mode, s); break;
        default: return LBE_UNSUPPORTED;
    }
    const long n = (long)cells * n3;
    if (Lplus) k_df_to_double<<<4 * sm_count(), 256, 0, s>>>(Lplus, n);
    if (Lout) k_df_to_double<<<4 * sm_count(), 256, 0, s>>>(Lout, n);
    g_launches += (Lplus ? 1 : 0) + (Lout ? 1 : 0);
    return LBE_OK;
}

}  // namespace lbe

// Host side of the fast-spectral operator shared by its arithmetic instances: twiddle set-up,
// scratch sizing and the L-moments kernel (A4).  The transform kernels are in
// fsm_cc_kernels.cuh; fsm_cc_f64.cu, fsm_cc_f32.cu, fsm_df.cu and fsm_df32.cu instantiate them.
#include "fsm_cc_kernels.cuh"

namespace lbe {

void init_twiddles_cc() {
    init_twiddles_f64();
    init_twiddles_f32();
    init_twiddles_df();
    init_twiddles_df32();
}

// Scratch needed by fsm_cc_apply for `cells` cells: H (cells) and Y (chunk * (M+1)) volumes.
size_t fsm_cc_scratch_bytes(const DevTables& t, int cells, int elem_bytes, int* chunk_out) {
    const long n3 = (long)t.nv * t.nv * t.nv;
    const long vol = n3 * 2 * elem_bytes;
    // keep one chunk's inverse transforms (chunk * (M+1) volumes) within ~96 MB of L2
    long fit = (96L << 20) / (vol * (t.M + 1));
    if (fit < 1) fit = 1;
    if (fit > 64) fit = 64;
    int chunk = cells < fit ? cells : (int)fit;
    if (chunk < 1) chunk = 1;
    if (chunk_out) *chunk_out = chunk;
    return (size_t)vol * cells + (size_t)vol * chunk * (t.M + 1);
}

template <typename T>
void lmoments(const DevTables& t, int cells, const T* Lh, const T* h, const double* nd, double* G,
              cudaStream_t s) {
    if (cells <= 0) return;
    g_launches += 1;
    const T* vel = sizeof(T) == 8 ? (const T*)t.vel_d : (const T*)t.vel_f;
    k_lmoments<T><<<cells, 8 * t.nv, 0, s>>>(Lh, h, nd, vel, t.nv, t.dv * t.dv * t.dv, G);
}


template void lmoments<double>(const DevTables&, int, const double*, const double*, const double*,
                               double*, cudaStream_t);
template void lmoments<float>(const DevTables&, int, const float*, const float*, const double*,
                              double*, cudaStream_t);

}  // namespace lbe

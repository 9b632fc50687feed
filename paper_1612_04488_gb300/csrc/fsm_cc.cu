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

// The L-moments of a plate cell in the orbit layout (one value per orbit {1, R2, R3, R2 R3},
// at (i1 H + j2) H + j3): v1 v3 (L h + nd h) is even under R2 and R3, so G_1 is four times the
// quarter's sum; v2 v3 (L h + nd h) is odd under R2, so G_2 = 0.  One thread per (j2, j3).
template <typename T>
__global__ void __launch_bounds__(256) k_lmoments_q(const T* __restrict__ Lh, const T* __restrict__ h,
                                                    const double* __restrict__ nd, const T* __restrict__ vel,
                                                    int nv, double dv3, double* __restrict__ G) {
    __shared__ double red[32 * 2];
    const int H = nv / 2;
    const long cell = blockIdx.x;
    const long n3 = (long)nv * nv * nv;
    const T ndc = (T)nd[cell];
    const int p = threadIdx.x;
    Acc<T> a0;
    if (p < H * H) {
        const T v3 = vel[p % H];
        for (int i1 = 0; i1 < nv; ++i1) {
            const long idx = cell * n3 + (long)i1 * H * H + p;
            const T t = (Lh[idx] + ndc * h[idx]) * v3;
            a0.add(vel[i1] * t);
        }
    }
    double sm[2] = {a0.value(), 0.0};
    block_reduce<2>(sm, red);
    if (threadIdx.x == 0) {
        G[2 * cell + 0] = 8.0 * sm[0] * dv3;
        G[2 * cell + 1] = 0.0;
    }
}

// The L-moments of a duct cell in the orbit layout (one value per orbit {1, R3}, at
// (i1 nv + i2) nv / 2 + j3): v_j v3 (L h + nd h) is even under R3, so G_j is twice the half's
// sum.  One thread per (i2, j3).
template <typename T>
__global__ void __launch_bounds__(512) k_lmoments_h(const T* __restrict__ Lh, const T* __restrict__ h,
                                                    const double* __restrict__ nd, const T* __restrict__ vel,
                                                    int nv, double dv3, double* __restrict__ G) {
    __shared__ double red[32 * 2];
    const int H = nv / 2;
    const long cell = blockIdx.x;
    const long n3 = (long)nv * nv * nv;
    const T ndc = (T)nd[cell];
    const int p = threadIdx.x;  // < nv H
    const T v2 = vel[p / H], v3 = vel[p % H];
    Acc<T> a0, a1;
    for (int i1 = 0; i1 < nv; ++i1) {
        const long idx = cell * n3 + (long)i1 * nv * H + p;
        const T t = (Lh[idx] + ndc * h[idx]) * v3;
        a0.add(vel[i1] * t);
        a1.add(v2 * t);
    }
    double sm[2] = {a0.value(), a1.value()};
    block_reduce<2>(sm, red);
    if (threadIdx.x == 0) {
        G[2 * cell + 0] = 4.0 * sm[0] * dv3;
        G[2 * cell + 1] = 4.0 * sm[1] * dv3;
    }
}

// quarter: 1 plates in the orbit layout, 2 ducts in the orbit layout
template <typename T>
void lmoments(const DevTables& t, int cells, const T* Lh, const T* h, const double* nd, double* G,
              cudaStream_t s, int quarter) {
    if (cells <= 0) return;
    g_launches += 1;
    const T* vel = sizeof(T) == 8 ? (const T*)t.vel_d : (const T*)t.vel_f;
    if (quarter == 2) {
        k_lmoments_h<T><<<cells, t.nv * (t.nv / 2), 0, s>>>(Lh, h, nd, vel, t.nv, t.dv * t.dv * t.dv, G);
        return;
    }
    if (quarter) {
        const int H = t.nv / 2, threads = (H * H + 31) / 32 * 32;
        k_lmoments_q<T><<<cells, threads, 0, s>>>(Lh, h, nd, vel, t.nv, t.dv * t.dv * t.dv, G);
        return;
    }
    k_lmoments<T><<<cells, 8 * t.nv, 0, s>>>(Lh, h, nd, vel, t.nv, t.dv * t.dv * t.dv, G);
}


template void lmoments<double>(const DevTables&, int, const double*, const double*, const double*,
                               double*, cudaStream_t, int);
template void lmoments<float>(const DevTables&, int, const float*, const float*, const double*,
                              double*, cudaStream_t, int);

}  // namespace lbe

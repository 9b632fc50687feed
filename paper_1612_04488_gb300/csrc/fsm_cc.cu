// Fast-spectral hard-sphere collision operator on CUDA cores (FP64 and FP32 paths).
//
// Steps (per cell, batched over cells):
//   A1  H = F h                          forward 3D DFT, three in-place axis passes
//   A2  c_p = F^-1[(psi_p + i phi_p) H]  one packed complex inverse DFT per direction p;
//       gain = sum_p w'_p (A_p Re c_p + B_p Im c_p)
//   A3  loss = F^-1[G H];  L+ h = delta (gain - f_eq loss),  L h = L+ h - delta nu_eq h
//   A4  G_j = 2 sum_v v_j v3 (L h + N delta h) dv^3   (lmoments kernel)
// (Sec. 2, Eq. LBE_collision; the operator's reading is stated in lbe.h.)
//
// Layout: h, L+ h, L h are [cell][i1][i2][i3]; H is [cell][k1][k2][k3] complex; the
// inverse transforms of a chunk of cells live in Y[cell][p][...] (p = 0..M, p = M is the
// loss), transformed in place along i3, then i2, and the last pass (along i1, coalesced
// across threads) accumulates the gain over p in registers and writes the outputs.
// Every thread owns one 1D line and keeps it in registers (dft_line in common.cuh).
#include <cmath>

#include "common.cuh"
#include "lbe_internal.h"

namespace lbe {

void init_twiddles_cc() {
    double2 hd[4][32];
    float2 hf[4][32];
    const int ns[4] = {8, 16, 24, 32};
    for (int s = 0; s < 4; ++s)
        for (int m = 0; m < 32; ++m) {
            double a = -2.0 * M_PI * (m % ns[s]) / ns[s];
            hd[s][m] = make_double2(std::cos(a), std::sin(a));
            hf[s][m] = make_float2((float)std::cos(a), (float)std::sin(a));
        }
    cudaMemcpyToSymbol(c_tw_d, hd, sizeof(hd));
    cudaMemcpyToSymbol(c_tw_f, hf, sizeof(hf));
}

namespace {

template <typename T> __device__ __forceinline__ cplx_t<T> mk(T a, T b);
template <> __device__ __forceinline__ double2 mk<double>(double a, double b) { return make_double2(a, b); }
template <> __device__ __forceinline__ float2 mk<float>(float a, float b) { return make_float2(a, b); }

// Line L of a batch of volumes along AXIS: first element offset and stride.
template <int N, int AXIS>
__device__ __forceinline__ void line_of(long L, long& base, int& stride) {
    const long vol = L / (N * N);
    const int r = (int)(L % (N * N));
    if (AXIS == 0) {          // r = i2 * N + i3
        base = vol * N * N * N + r;
        stride = N * N;
    } else if (AXIS == 1) {   // r = i1 * N + i3
        base = vol * N * N * N + (long)(r / N) * N * N + (r % N);
        stride = N;
    } else {                  // r = i1 * N + i2
        base = vol * N * N * N + (long)r * N;
        stride = 1;
    }
}

template <typename T, int N, int AXIS, bool REAL_IN>
__global__ void __launch_bounds__(128) k_fwd(const T* __restrict__ hin, cplx_t<T>* __restrict__ H,
                                             long nlines) {
    const long L = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (L >= nlines) return;
    long base;
    int st;
    line_of<N, AXIS>(L, base, st);
    T re[N], im[N];
#pragma unroll
    for (int j = 0; j < N; ++j) {
        if (REAL_IN) {
            re[j] = hin[base + (long)j * st];
            im[j] = T(0);
        } else {
            const cplx_t<T> z = H[base + (long)j * st];
            re[j] = z.x;
            im[j] = z.y;
        }
    }
    dft_line<T, N, false>(re, im);
#pragma unroll
    for (int j = 0; j < N; ++j) H[base + (long)j * st] = mk<T>(re[j], im[j]);
}

// Y[cell][p] = F^-1_3 (mult_p * H[cell]) for p = 0..M (first inverse pass, along i3).
template <typename T, int N>
__global__ void __launch_bounds__(128) k_inv_first(const cplx_t<T>* __restrict__ H,
                                                   const cplx_t<T>* __restrict__ mult,
                                                   cplx_t<T>* __restrict__ Y, int ncell, int P) {
    const long L = blockIdx.x * (long)blockDim.x + threadIdx.x;
    const long nl = (long)ncell * P * N * N;
    if (L >= nl) return;
    const long cp = L / (N * N);
    const int r = (int)(L % (N * N));
    const long cell = cp / P;
    const int p = (int)(cp % P);
    const cplx_t<T>* hl = H + cell * N * N * N + (long)r * N;
    const cplx_t<T>* ml = mult + (long)p * N * N * N + (long)r * N;
    T re[N], im[N];
#pragma unroll
    for (int j = 0; j < N; ++j) {
        const cplx_t<T> z = hl[j], m = ml[j];
        re[j] = m.x * z.x - m.y * z.y;
        im[j] = m.x * z.y + m.y * z.x;
    }
    dft_line<T, N, true>(re, im);
    cplx_t<T>* yl = Y + cp * N * N * N + (long)r * N;
#pragma unroll
    for (int j = 0; j < N; ++j) yl[j] = mk<T>(re[j], im[j]);
}

template <typename T, int N>
__global__ void __launch_bounds__(128) k_inv_mid(cplx_t<T>* __restrict__ Y, long nlines) {
    const long L = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (L >= nlines) return;
    long base;
    int st;
    line_of<N, 1>(L, base, st);
    T re[N], im[N];
#pragma unroll
    for (int j = 0; j < N; ++j) {
        const cplx_t<T> z = Y[base + (long)j * st];
        re[j] = z.x;
        im[j] = z.y;
    }
    dft_line<T, N, true>(re, im);
#pragma unroll
    for (int j = 0; j < N; ++j) Y[base + (long)j * st] = mk<T>(re[j], im[j]);
}

// Last inverse pass along i1 with the angular sum and the operator assembly.
template <typename T, int N>
__global__ void __launch_bounds__(128) k_inv_last(const cplx_t<T>* __restrict__ Y,
                                                  const cplx_t<T>* __restrict__ ab,
                                                  const T* __restrict__ feq, const T* __restrict__ nu1,
                                                  const T* __restrict__ h, const double* __restrict__ delta,
                                                  T* __restrict__ Lplus, T* __restrict__ Lout, int ncell,
                                                  int M) {
    constexpr int N2 = N * N, N3 = N * N * N;
    const long L = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (L >= (long)ncell * N2) return;
    const long cell = L / N2;
    const int r = (int)(L % N2);
    T acc[N];
    {
        const cplx_t<T>* yl = Y + (cell * (M + 1) + M) * N3 + r;
        T re[N], im[N];
#pragma unroll
        for (int j = 0; j < N; ++j) {
            const cplx_t<T> z = yl[(long)j * N2];
            re[j] = z.x;
            im[j] = z.y;
        }
        dft_line<T, N, true>(re, im);
#pragma unroll
        for (int j = 0; j < N; ++j) acc[j] = -feq[j * N2 + r] * re[j];
    }
    for (int p = 0; p < M; ++p) {
        const cplx_t<T>* yl = Y + (cell * (M + 1) + p) * N3 + r;
        const cplx_t<T>* al = ab + (long)p * N3 + r;
        T re[N], im[N];
#pragma unroll
        for (int j = 0; j < N; ++j) {
            const cplx_t<T> z = yl[(long)j * N2];
            re[j] = z.x;
            im[j] = z.y;
        }
        dft_line<T, N, true>(re, im);
#pragma unroll
        for (int j = 0; j < N; ++j) {
            const cplx_t<T> w = al[j * N2];
            acc[j] += w.x * re[j] + w.y * im[j];
        }
    }
    const T d = (T)delta[cell];
#pragma unroll
    for (int j = 0; j < N; ++j) {
        const long idx = cell * N3 + (long)j * N2 + r;
        const T lp = d * acc[j];
        if (Lplus) Lplus[idx] = lp;
        if (Lout) Lout[idx] = lp - d * nu1[j * N2 + r] * h[idx];
    }
}

// G_j = 2 sum_v v_j v3 (L h + nd h) dv^3, one block per cell, fixed reduction order.
template <typename T>
__global__ void __launch_bounds__(256) k_lmoments(const T* __restrict__ Lh, const T* __restrict__ h,
                                                  const double* __restrict__ nd,
                                                  const double* __restrict__ vel, int nv, double dv3,
                                                  double* __restrict__ G) {
    __shared__ double red[32 * 2];
    const long cell = blockIdx.x;
    const int n3 = nv * nv * nv;
    const double ndc = nd[cell];
    double s[2] = {0.0, 0.0};
    for (int i = threadIdx.x; i < n3; i += blockDim.x) {
        const int i1 = i / (nv * nv), i2 = (i / nv) % nv, i3 = i % nv;
        const double t = (double)Lh[cell * n3 + i] + ndc * (double)h[cell * n3 + i];
        const double v3t = vel[i3] * t;
        s[0] += vel[i1] * v3t;
        s[1] += vel[i2] * v3t;
    }
    block_reduce<2>(s, red);
    if (threadIdx.x == 0) {
        G[2 * cell + 0] = 2.0 * s[0] * dv3;
        G[2 * cell + 1] = 2.0 * s[1] * dv3;
    }
}

inline unsigned nblk(long n, int b) { return (unsigned)((n + b - 1) / b); }

template <typename T, int N>
void run_fsm(const DevTables& t, int cells, const double* delta, const T* h, T* Lplus, T* Lout,
             cplx_t<T>* Hbuf, cplx_t<T>* Ybuf, int chunk, cudaStream_t s) {
    constexpr int B = 128;
    const long nl = (long)cells * N * N;
    k_fwd<T, N, 0, true><<<nblk(nl, B), B, 0, s>>>(h, Hbuf, nl);
    k_fwd<T, N, 1, false><<<nblk(nl, B), B, 0, s>>>(nullptr, Hbuf, nl);
    k_fwd<T, N, 2, false><<<nblk(nl, B), B, 0, s>>>(nullptr, Hbuf, nl);
    const cplx_t<T>* mult;
    const cplx_t<T>* ab;
    const T* feq;
    const T* nu1;
    if constexpr (sizeof(T) == 8) {
        mult = (const cplx_t<T>*)t.mult_d;
        ab = (const cplx_t<T>*)t.ab_d;
        feq = (const T*)t.feq_d;
        nu1 = (const T*)t.nu1_d;
    } else {
        mult = (const cplx_t<T>*)t.mult_f;
        ab = (const cplx_t<T>*)t.ab_f;
        feq = (const T*)t.feq_f;
        nu1 = (const T*)t.nu1_f;
    }
    const int P = t.M + 1;
    const long N3 = (long)N * N * N;
    g_launches += 3;
    g_levals += cells;
    for (int c0 = 0; c0 < cells; c0 += chunk) {
        g_launches += 3;
        const int cc = (cells - c0 < chunk) ? cells - c0 : chunk;
        const long nf = (long)cc * P * N * N;
        k_inv_first<T, N><<<nblk(nf, B), B, 0, s>>>(Hbuf + c0 * N3, mult, Ybuf, cc, P);
        k_inv_mid<T, N><<<nblk(nf, B), B, 0, s>>>(Ybuf, nf);
        const long nlast = (long)cc * N * N;
        k_inv_last<T, N><<<nblk(nlast, B), B, 0, s>>>(Ybuf, ab, feq, nu1, h + c0 * N3, delta + c0,
                                                      Lplus ? Lplus + c0 * N3 : nullptr,
                                                      Lout ? Lout + c0 * N3 : nullptr, cc, t.M);
    }
}

}  // namespace

// Scratch needed by fsm_cc_apply for `cells` cells: H (cells) and Y (chunk * (M+1)) volumes.
size_t fsm_cc_scratch_bytes(const DevTables& t, int cells, int elem_bytes, int* chunk_out) {
    const long n3 = (long)t.nv * t.nv * t.nv;
    const long vol = n3 * 2 * elem_bytes;
    int chunk = cells < 64 ? cells : 64;
    if (chunk < 1) chunk = 1;
    if (chunk_out) *chunk_out = chunk;
    return (size_t)vol * cells + (size_t)vol * chunk * (t.M + 1);
}

template <typename T>
lbe_status fsm_cc_apply(const DevTables& t, int cells, const double* delta, const T* h, T* Lplus,
                        T* Lout, void* scratch, int chunk, cudaStream_t s) {
    const long n3 = (long)t.nv * t.nv * t.nv;
    cplx_t<T>* Hbuf = (cplx_t<T>*)scratch;
    cplx_t<T>* Ybuf = Hbuf + n3 * cells;
    switch (t.nv) {
        case 8: run_fsm<T, 8>(t, cells, delta, h, Lplus, Lout, Hbuf, Ybuf, chunk, s); break;
        case 16: run_fsm<T, 16>(t, cells, delta, h, Lplus, Lout, Hbuf, Ybuf, chunk, s); break;
        case 24: run_fsm<T, 24>(t, cells, delta, h, Lplus, Lout, Hbuf, Ybuf, chunk, s); break;
        case 32: run_fsm<T, 32>(t, cells, delta, h, Lplus, Lout, Hbuf, Ybuf, chunk, s); break;
        default: return LBE_UNSUPPORTED;
    }
    return LBE_OK;
}

template <typename T>
void lmoments(const DevTables& t, int cells, const T* Lh, const T* h, const double* nd, double* G,
              cudaStream_t s) {
    if (cells <= 0) return;
    g_launches += 1;
    k_lmoments<T><<<cells, 256, 0, s>>>(Lh, h, nd, t.vel_d, t.nv, t.dv * t.dv * t.dv, G);
}

template lbe_status fsm_cc_apply<double>(const DevTables&, int, const double*, const double*,
                                         double*, double*, void*, int, cudaStream_t);
template lbe_status fsm_cc_apply<float>(const DevTables&, int, const double*, const float*, float*,
                                        float*, void*, int, cudaStream_t);
template void lmoments<double>(const DevTables&, int, const double*, const double*, const double*,
                               double*, cudaStream_t);
template void lmoments<float>(const DevTables&, int, const float*, const float*, const double*,
                              double*, cudaStream_t);

}  // namespace lbe

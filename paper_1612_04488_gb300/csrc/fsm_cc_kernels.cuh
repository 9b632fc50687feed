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
// Layout: h, L+ h, L h are [cell][i1][i2][i3]; H is [cell][k1][k2][k3] complex.  The
// forward transform does the i3 and i2 axes per k1-plane in shared memory (k_slab2d), then
// i1 in place (k_fwd).  The inverse transforms of a chunk of cells, sized so that they stay
// in L2, live in Y[cell][p][...] (p = 0..M, p = M is the loss): k_slab2d applies the
// multiplier and the i3, i2 axes per plane; k_inv_last4 transforms along i1 (coalesced
// across lanes), sums the directions over four warps and writes the outputs.  Every lane
// owns one 1D line in registers (dft_line in common.cuh).
//
// This header holds the kernels and the per-chunk driver; the translation units
// fsm_cc_f64.cu, fsm_cc_f32.cu, fsm_df.cu and fsm_df32.cu instantiate them per
// arithmetic (and grid), so that they compile in parallel.  Each unit keeps its own copy
// of the twiddle tables, filled by init_twiddles_cc().
#pragma once

#include <algorithm>
#include <cmath>
#include <type_traits>

#include "common.cuh"
#include "lbe_internal.h"
#include "sweep.h"

namespace lbe {

namespace {

template <typename T> __device__ __forceinline__ cplx_t<T> mk(T a, T b);
template <> __device__ __forceinline__ double2 mk<double>(double a, double b) { return make_double2(a, b); }
template <> __device__ __forceinline__ float2 mk<float>(float a, float b) { return make_float2(a, b); }
template <> __device__ __forceinline__ dfloat2 mk<dfloat>(dfloat a, dfloat b) { return dfloat2{a, b}; }

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

// 2D transform of one k1-plane ("slab", N x N complex) along i3 then i2, staged in shared
// memory so that global loads and stores are coalesced rows.  One warp per slab.
//   REAL_IN:  forward transform of a real plane of h (A1, first two axes)
//   MULT:     inverse transform of mult_p * H (A2, first two axes of direction p's inverse)
template <typename T, int N, bool INV, bool REAL_IN, bool MULT, int WPB, typename TIN = T>
__global__ void __launch_bounds__(32 * WPB) k_slab2d(const TIN* __restrict__ hin, const cplx_t<T>* __restrict__ Hin,
                                                     const cplx_t<T>* __restrict__ mult,
                                                     cplx_t<T>* __restrict__ out, long nslabs, int P,
                                                     int loss_slot) {
    constexpr int LD = N + 1, N2 = N * N;
    __shared__ cplx_t<T> sm[WPB][N][LD];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long sid = (long)blockIdx.x * WPB + w;
    if (sid >= nslabs) return;
    const long vol = sid / N;                 // MULT: cell * P + p; otherwise the volume
    const int k1 = (int)(sid % N);
    long ibase, mbase = 0;
    if (MULT) {
        const long cell = vol / P;
        const int p = (int)(vol % P);
        const int pm = (p == P - 1) ? loss_slot : p;  // last slot: the loss multiplier
        ibase = cell * N * N2 + (long)k1 * N2;
        mbase = (long)pm * N * N2 + (long)k1 * N2;
    } else {
        ibase = vol * N * N2 + (long)k1 * N2;
    }
    const long obase = vol * N * N2 + (long)k1 * N2;
    for (int idx = lane; idx < N2; idx += 32) {
        cplx_t<T> z;
        if (REAL_IN) {
            z.x = T(hin[ibase + idx]);
            z.y = T(0);
        } else {
            z = Hin[ibase + idx];
            if (MULT) {
                const cplx_t<T> m = mult[mbase + idx];
                const T xr = m.x * z.x - m.y * z.y, xi = m.x * z.y + m.y * z.x;
                z.x = xr;
                z.y = xi;
            }
        }
        sm[w][idx / N][idx % N] = z;
    }
    __syncwarp();
    // along i3 (lane owns row k2 = lane), then along i2 (lane owns column i3 = lane): one loop,
    // so the unrolled line transform is emitted once (the kernel's code stays small enough for
    // the instruction cache)
#pragma unroll 1
    for (int pass = 0; pass < 2; ++pass) {
        if (lane < N) {
            cplx_t<T>* p0 = pass == 0 ? &sm[w][lane][0] : &sm[w][0][lane];
            const int st = pass == 0 ? 1 : LD;
            T re[N], im[N];
#pragma unroll
            for (int j = 0; j < N; ++j) {
                re[j] = p0[j * st].x;
                im[j] = p0[j * st].y;
            }
            dft_line<T, N, INV>(re, im);
#pragma unroll
            for (int j = 0; j < N; ++j) p0[j * st] = mk<T>(re[j], im[j]);
        }
        __syncwarp();
    }
    for (int idx = lane; idx < N2; idx += 32) out[obase + idx] = sm[w][idx / N][idx % N];
}

// Last inverse pass (along i1) with the angular sum split over the four warps of a block:
// the 32 lanes hold 32 consecutive (i2, i3) lines of one cell, warp w sums directions
// p = w, w+4, ...; the partial sums meet in shared memory in a fixed order (A2-A3).
// With RAW, the representatives' gain goes to Lplus and the loss convolution to Lout
// unassembled, for k_sym to complete.  Y holds M directions and the loss in slot M.
template <typename T, int N, bool RAW, typename TIN = T>
__global__ void __launch_bounds__(128) k_inv_last4(const cplx_t<T>* __restrict__ Y,
                                                   const cplx_t<T>* __restrict__ ab,
                                                   const T* __restrict__ feq, const T* __restrict__ nu1,
                                                   const TIN* __restrict__ h, const double* __restrict__ delta,
                                                   T* __restrict__ Lplus, T* __restrict__ Lout, int ncell,
                                                   int M) {
    constexpr int N2 = N * N, N3 = N * N * N, TILES = N2 / 32;
    __shared__ T red[4][N][32];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long cell = blockIdx.x / TILES;
    const int r = (blockIdx.x % TILES) * 32 + lane;
    if (cell >= ncell) return;
    T acc[N];
#pragma unroll
    for (int j = 0; j < N; ++j) acc[j] = T(0);
    // slots p = w, w + 4, .. of the M directions and the loss (p = M), one line transform in
    // the loop body (emitted once)
    for (int p = w; p <= M; p += 4) {
        const cplx_t<T>* yl = Y + (cell * (M + 1) + p) * N3 + r;
        T re[N], im[N];
#pragma unroll
        for (int j = 0; j < N; ++j) {
            const cplx_t<T> z = yl[(long)j * N2];
            re[j] = z.x;
            im[j] = z.y;
        }
        dft_line<T, N, true>(re, im);
        if (p == M) {  // the loss convolution
            if (RAW) {
#pragma unroll
                for (int j = 0; j < N; ++j) Lout[cell * N3 + (long)j * N2 + r] = re[j];
            } else {
#pragma unroll
                for (int j = 0; j < N; ++j) acc[j] += -feq[j * N2 + r] * re[j];
            }
            continue;
        }
        const cplx_t<T>* al = ab + (long)p * N3 + r;
#pragma unroll
        for (int j = 0; j < N; ++j) {
            const cplx_t<T> a = al[j * N2];
            acc[j] += a.x * re[j] + a.y * im[j];
        }
    }
#pragma unroll
    for (int j = 0; j < N; ++j) red[w][j][lane] = acc[j];
    __syncthreads();
    const T d = (T)delta[cell];
    for (int j = w; j < N; j += 4) {
        const T sum = ((red[0][j][lane] + red[1][j][lane]) + red[2][j][lane]) + red[3][j][lane];
        const long idx = cell * N3 + (long)j * N2 + r;
        if (RAW) {
            Lplus[idx] = sum;
            continue;
        }
        const T lp = d * sum;
        if (Lplus) Lplus[idx] = lp;
        if (Lout) Lout[idx] = lp - d * nu1[j * N2 + r] * T(h[idx]);
    }
}

// Completes the symmetry-reduced operator.  For h with parities s2 (v2 -> -v2) and
// s3 = -1 (v3 -> -v3), the operator commutes with the reflections and the direction set is
// closed under them, so the sum over all directions equals the sum over one representative
// per orbit, G, symmetrised: gain(v) = sum_g s_g G(g v) over g in {1, R3} (MODE 1) or
// {1, R2, R3, R2R3} (MODE 2, s2 = +1).  One thread per orbit of velocity points.
template <typename T, int N, int MODE, typename TIN = T>
__global__ void __launch_bounds__(128) k_sym(T* __restrict__ Lplus, T* __restrict__ Lout,
                                             const T* __restrict__ feq, const T* __restrict__ nu1,
                                             const TIN* __restrict__ h, const double* __restrict__ delta,
                                             int ncell, bool want_lplus, bool want_l) {
    constexpr int N2 = N * N, N3 = N2 * N, H = N / 2;
    constexpr int per_cell = MODE == 2 ? N * H * H : N * N * H;
    const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (t >= (long)ncell * per_cell) return;
    const long cell = t / per_cell;
    const int q = (int)(t % per_cell);
    int i1, i2, i3;
    if (MODE == 2) {
        i1 = q / (H * H);
        i2 = (q / H) % H;
        i3 = q % H;
    } else {
        i1 = q / (N * H);
        i2 = (q / H) % N;
        i3 = q % H;
    }
    const int j2 = N - 1 - i2, j3 = N - 1 - i3;
    const long base = cell * N3 + (long)i1 * N2;
    const T d = (T)delta[cell];
    long idx[4];
    T sgn[4];
    int nptr;
    T gs;
    if (MODE == 2) {
        idx[0] = base + i2 * N + i3;   // v
        idx[1] = base + j2 * N + i3;   // R2 v   (s2 = +1)
        idx[2] = base + i2 * N + j3;   // R3 v   (s3 = -1)
        idx[3] = base + j2 * N + j3;   // R2R3 v (s2 s3 = -1)
        sgn[0] = T(1); sgn[1] = T(1); sgn[2] = T(-1); sgn[3] = T(-1);
        nptr = 4;
        gs = (Lplus[idx[0]] + Lplus[idx[1]]) - (Lplus[idx[2]] + Lplus[idx[3]]);
    } else {
        idx[0] = base + i2 * N + i3;
        idx[1] = base + i2 * N + j3;   // R3 v
        sgn[0] = T(1); sgn[1] = T(-1);
        nptr = 2;
        gs = Lplus[idx[0]] - Lplus[idx[1]];
    }
    for (int k = 0; k < nptr; ++k) {
        const long g = idx[k];
        const int v = (int)(g - cell * N3);
        const T lp = d * (sgn[k] * gs - feq[v] * Lout[g]);
        const T hv = T(h[g]);
        if (want_lplus) Lplus[g] = lp;
        if (want_l) Lout[g] = lp - d * nu1[v] * hv;
    }
}

template <typename T> struct Acc;
template <> struct Acc<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double x) { s += x; }
    __device__ __forceinline__ double value() const { return s; }
};
template <> struct Acc<float> {  // compensated float sum
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float x) {
        const float y = x - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

// G_j = 2 sum_v v_j v3 (L h + nd h) dv^3, one block of 8 nv threads per cell (thread t owns
// i3 = t % nv and rows i2 = t/nv + 8k), fixed reduction order.
template <typename T>
__global__ void __launch_bounds__(256) k_lmoments(const T* __restrict__ Lh, const T* __restrict__ h,
                                                  const double* __restrict__ nd,
                                                  const T* __restrict__ vel, int nv, double dv3,
                                                  double* __restrict__ G) {
    __shared__ double red[32 * 2];
    const long cell = blockIdx.x;
    const long n3 = (long)nv * nv * nv;
    const T ndc = (T)nd[cell];
    const int i3 = threadIdx.x % nv, r0 = threadIdx.x / nv;
    const T v3 = vel[i3];
    Acc<T> a0, a1;
    for (int i1 = 0; i1 < nv; ++i1) {
        const T v1 = vel[i1];
        for (int i2 = r0; i2 < nv; i2 += 8) {
            const long idx = cell * n3 + ((long)i1 * nv + i2) * nv + i3;
            const T t = (Lh[idx] + ndc * h[idx]) * v3;
            a0.add(v1 * t);
            a1.add(vel[i2] * t);
        }
    }
    double s[2] = {a0.value(), a1.value()};
    block_reduce<2>(s, red);
    if (threadIdx.x == 0) {
        G[2 * cell + 0] = 2.0 * s[0] * dv3;
        G[2 * cell + 1] = 2.0 * s[1] * dv3;
    }
}

inline unsigned nblk(long n, int b) { return (unsigned)((n + b - 1) / b); }

template <typename T, int N, typename TH = T>
void run_fsm(const DevTables& t, int cells, const double* delta, const TH* h, T* Lplus, T* Lout,
             cplx_t<T>* Hbuf, cplx_t<T>* Ybuf, int chunk, int mode, cudaStream_t s) {
    constexpr int B = 128;
    constexpr int WPB = (sizeof(T) == 8 && N == 32) ? 2 : 4;
    const long nl = (long)cells * N * N;
    const long ns = (long)cells * N;
    k_slab2d<T, N, false, true, false, WPB, TH><<<nblk(ns, WPB), 32 * WPB, 0, s>>>(h, nullptr, nullptr, Hbuf, ns, 1,
                                                                                 0);
    k_fwd<T, N, 0, false><<<nblk(nl, B), B, 0, s>>>(nullptr, Hbuf, nl);
    const cplx_t<T>* mult;
    const cplx_t<T>* ab;
    const T* feq;
    const T* nu1;
    if constexpr (std::is_same<T, double>::value) {
        mult = (const cplx_t<T>*)t.mult_d;
        ab = (const cplx_t<T>*)t.ab_d;
        feq = (const T*)t.feq_d;
        nu1 = (const T*)t.nu1_d;
    } else if constexpr (std::is_same<T, dfloat>::value) {
        mult = (const cplx_t<T>*)t.mult_x;
        ab = (const cplx_t<T>*)t.ab_x;
        feq = (const T*)t.feq_x;
        nu1 = (const T*)t.nu1_x;
    } else {
        mult = (const cplx_t<T>*)t.mult_f;
        ab = (const cplx_t<T>*)t.ab_f;
        feq = (const T*)t.feq_f;
        nu1 = (const T*)t.nu1_f;
    }
    const int Muse = mode == 2 ? t.sym_reps2 : (mode == 1 ? t.sym_reps1 : t.M);
    const int P = Muse + 1;
    const long N3 = (long)N * N * N;
    g_launches += 2;
    g_levals += cells;
    // the scratch holds chunk * (M + 1) inverse-transform volumes; the parity-reduced forms
    // use P of them per cell, so the same scratch (and L2 footprint) takes more cells per chunk
    chunk = std::min(cells, std::max(chunk, chunk * (t.M + 1) / P));
    for (int c0 = 0; c0 < cells; c0 += chunk) {
        g_launches += 2;
        const int cc = (cells - c0 < chunk) ? cells - c0 : chunk;
        const long nsl = (long)cc * P * N;
        k_slab2d<T, N, true, false, true, WPB, T><<<nblk(nsl, WPB), 32 * WPB, 0, s>>>(nullptr, Hbuf + c0 * N3, mult,
                                                                                  Ybuf, nsl, P, t.M);
        const long blocks = (long)cc * (N * N / 32);
        if (mode == 0) {
            k_inv_last4<T, N, false, TH><<<(unsigned)blocks, 128, 0, s>>>(Ybuf, ab, feq, nu1, h + c0 * N3, delta + c0,
                                                                    Lplus ? Lplus + c0 * N3 : nullptr,
                                                                    Lout ? Lout + c0 * N3 : nullptr, cc, Muse);
        } else {
            // raw gain of the representatives and the loss convolution, then symmetrise
            k_inv_last4<T, N, true, TH><<<(unsigned)blocks, 128, 0, s>>>(Ybuf, ab, feq, nu1, h + c0 * N3, delta + c0,
                                                                   Lplus + c0 * N3, Lout + c0 * N3, cc, Muse);
            g_launches += 1;
            const long nt = (long)cc * (mode == 2 ? N * (N / 2) * (N / 2) : N * N * (N / 2));
            if (mode == 2)
                k_sym<T, N, 2, TH><<<nblk(nt, 128), 128, 0, s>>>(Lplus + c0 * N3, Lout + c0 * N3, feq, nu1, h + c0 * N3,
                                                             delta + c0, cc, true, true);
            else
                k_sym<T, N, 1, TH><<<nblk(nt, 128), 128, 0, s>>>(Lplus + c0 * N3, Lout + c0 * N3, feq, nu1, h + c0 * N3,
                                                             delta + c0, cc, true, true);
        }
    }
}


// Fills this translation unit's copy of the twiddle tables (common.cuh) on the current device.
inline void upload_twiddles() {
    double2 hd[4][32];
    float2 hf[4][32];
    dfloat2 hx[4][32];
    const int ns[4] = {8, 16, 24, 32};
    for (int s = 0; s < 4; ++s)
        for (int m = 0; m < 32; ++m) {
            const double a = -2.0 * M_PI * (m % ns[s]) / ns[s];
            hd[s][m] = make_double2(std::cos(a), std::sin(a));
            hf[s][m] = make_float2((float)std::cos(a), (float)std::sin(a));
            hx[s][m] = dfloat2{dfloat(std::cos(a)), dfloat(std::sin(a))};
        }
    cudaMemcpyToSymbol(c_tw_d, hd, sizeof(hd));
    cudaMemcpyToSymbol(c_tw_f, hf, sizeof(hf));
    cudaMemcpyToSymbol(c_tw_df, hx, sizeof(hx));
}

}  // namespace

template <typename T>
lbe_status fsm_cc_apply(const DevTables& t, int cells, const double* delta, const T* h, T* Lplus,
                        T* Lout, void* scratch, int chunk, cudaStream_t s, int mode) {
    const long n3 = (long)t.nv * t.nv * t.nv;
    if (mode == 2 && t.sym_reps2 == 0) mode = t.sym_reps1 ? 1 : 0;
    if (mode == 1 && t.sym_reps1 == 0) mode = 0;
    if (mode != 0 && (!Lplus || !Lout)) return LBE_INTERNAL;  // the symmetrised path needs both outputs
    cplx_t<T>* Hbuf = (cplx_t<T>*)scratch;
    cplx_t<T>* Ybuf = Hbuf + n3 * cells;
    switch (t.nv) {
        case 8: run_fsm<T, 8>(t, cells, delta, h, Lplus, Lout, Hbuf, Ybuf, chunk, mode, s); break;
        case 16: run_fsm<T, 16>(t, cells, delta, h, Lplus, Lout, Hbuf, Ybuf, chunk, mode, s); break;
        case 24: run_fsm<T, 24>(t, cells, delta, h, Lplus, Lout, Hbuf, Ybuf, chunk, mode, s); break;
        case 32: run_fsm<T, 32>(t, cells, delta, h, Lplus, Lout, Hbuf, Ybuf, chunk, mode, s); break;
        default: return LBE_UNSUPPORTED;
    }
    return LBE_OK;
}

// The double-float operator for one grid size (instantiated in fsm_df.cu / fsm_df32.cu).
template <int N>
void run_fsm_df(const DevTables& t, int cells, const double* delta, const double* h, dfloat* lp, dfloat* lo,
                dfloat2* Hbuf, dfloat2* Ybuf, int chunk, int mode, cudaStream_t s) {
    run_fsm<dfloat, N, double>(t, cells, delta, h, lp, lo, Hbuf, Ybuf, chunk, mode, s);
}

// Twiddle uploads of the instantiating units.
void init_twiddles_f64();
void init_twiddles_f32();
void init_twiddles_df();
void init_twiddles_df32();

}  // namespace lbe

// Device helpers shared by the library's kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace lbe {

// Double-float: the unevaluated sum hi + lo of two floats with |lo| <= ulp(hi) / 2, about
// 2^-44 relative per operation -- FP64-class accuracy from the FP32 pipes, which on this GPU
// issue many times the FP64 rate.  Built from the error-free transformations TwoSum (Knuth),
// Fast2Sum (Dekker; |a| >= |b|) and the FMA form of TwoProduct; every step is an explicitly
// rounded intrinsic so that no contraction or reassociation can remove an error term.
// Addition is the cheap variant (error relative to |a| + |b|), which suits transforms and
// sums whose error is measured against the size of their inputs.
struct dfloat {
    float hi, lo;
    dfloat() = default;
    __host__ __device__ constexpr dfloat(float h, float l) : hi(h), lo(l) {}
    __host__ __device__ dfloat(double x) : hi((float)x), lo((float)(x - (double)(float)x)) {}
    __host__ __device__ constexpr dfloat(int x) : hi((float)x), lo(0.f) {}
    __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};
struct dfloat2 {
    dfloat x, y;
};

__device__ __forceinline__ dfloat df_fast2sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return dfloat(s, __fsub_rn(b, __fsub_rn(s, a)));
}
__device__ __forceinline__ dfloat df_twosum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return dfloat(s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb)));
}
// The results of + and * are left unnormalised (|lo| may reach a few ulps of hi), which saves
// the renormalising Fast2Sum.  TwoSum / TwoProduct of the hi parts stay exact whatever the
// split, but the lo terms are rounded together, so the per-operation error bound grows with
// |lo| / ulp(hi) beyond the ~2^-44 of normalised pairs; the agreement of the transforms with
// FP64 (about 1e-13 of the scale) is measured by the parity tests, not implied by this bound.
// Widening to double adds the parts exactly.
__device__ __forceinline__ dfloat operator+(dfloat a, dfloat b) {
    const dfloat s = df_twosum(a.hi, b.hi);
    return dfloat(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ dfloat operator-(dfloat a) { return dfloat(-a.hi, -a.lo); }
__device__ __forceinline__ dfloat operator-(dfloat a, dfloat b) { return a + (-b); }
__device__ __forceinline__ dfloat operator*(dfloat a, dfloat b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return dfloat(p, e);
}
__device__ __forceinline__ dfloat& operator+=(dfloat& a, dfloat b) { return a = a + b; }

template <typename T> struct Cplx;
template <> struct Cplx<double> { using type = double2; };
template <> struct Cplx<float> { using type = float2; };
template <> struct Cplx<dfloat> { using type = dfloat2; };
template <typename T> using cplx_t = typename Cplx<T>::type;

// Twiddles W^m = exp(-2 pi i m / N) for N in {8, 16, 24, 32}, slot = index of N.
// Each translation unit that uses them fills its own copy once per device
// (see init_twiddles in fsm_cc.cu).
static __constant__ double2 c_tw_d[4][32];
static __constant__ float2 c_tw_f[4][32];
static __constant__ dfloat2 c_tw_df[4][32];

template <int N> struct TwSlot;
template <> struct TwSlot<8> { static constexpr int v = 0; };
template <> struct TwSlot<16> { static constexpr int v = 1; };
template <> struct TwSlot<24> { static constexpr int v = 2; };
template <> struct TwSlot<32> { static constexpr int v = 3; };

template <typename T, int N> __device__ __forceinline__ cplx_t<T> tw(int m);
template <> __device__ __forceinline__ double2 tw<double, 8>(int m) { return c_tw_d[0][m]; }
template <> __device__ __forceinline__ double2 tw<double, 16>(int m) { return c_tw_d[1][m]; }
template <> __device__ __forceinline__ double2 tw<double, 24>(int m) { return c_tw_d[2][m]; }
template <> __device__ __forceinline__ double2 tw<double, 32>(int m) { return c_tw_d[3][m]; }
template <> __device__ __forceinline__ float2 tw<float, 8>(int m) { return c_tw_f[0][m]; }
template <> __device__ __forceinline__ float2 tw<float, 16>(int m) { return c_tw_f[1][m]; }
template <> __device__ __forceinline__ float2 tw<float, 24>(int m) { return c_tw_f[2][m]; }
template <> __device__ __forceinline__ float2 tw<float, 32>(int m) { return c_tw_f[3][m]; }
template <> __device__ __forceinline__ dfloat2 tw<dfloat, 8>(int m) { return c_tw_df[0][m]; }
template <> __device__ __forceinline__ dfloat2 tw<dfloat, 16>(int m) { return c_tw_df[1][m]; }
template <> __device__ __forceinline__ dfloat2 tw<dfloat, 24>(int m) { return c_tw_df[2][m]; }
template <> __device__ __forceinline__ dfloat2 tw<dfloat, 32>(int m) { return c_tw_df[3][m]; }

__host__ __device__ constexpr bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }
__host__ __device__ constexpr int ilog2(int n) { return n <= 1 ? 0 : 1 + ilog2(n / 2); }
__host__ __device__ constexpr int bitrev(int i, int bits) {
    int r = 0;
    for (int b = 0; b < bits; ++b) r |= ((i >> b) & 1) << (bits - 1 - b);
    return r;
}

template <typename T, int N, bool INV>
__device__ __forceinline__ void dft_line(T (&re)[N], T (&im)[N]);

// Length N = 3 * 2^k by one mixed-radix step (Cooley-Tukey): the three interleaved
// subsequences x[3j + r] are transformed with length N/3, then for every k1 < N/3
//     X[k1 + (N/3) k2] = sum_r W_3^(r k2) (W_N^(r k1) Y_r[k1]),   k2 = 0, 1, 2,
// a twiddle product and one 3-point DFT.  With d = z1 - z2 and m = z0 - (z1 + z2)/2 the
// 3-point DFT is Z0 = z0 + z1 + z2, Z1 = m -+ i (sqrt(3)/2) d, Z2 = m +- i (sqrt(3)/2) d
// (upper signs forward).  W_N^(N/3) = -1/2 - i sqrt(3)/2 supplies both constants.
template <typename T, int N, bool INV>
__device__ __forceinline__ void dft_line_radix3(T (&re)[N], T (&im)[N]) {
    constexpr int K = N / 3;
    T sr[3][K], si[3][K];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int j = 0; j < K; ++j) {
            sr[r][j] = re[3 * j + r];
            si[r][j] = im[3 * j + r];
        }
#pragma unroll
    for (int r = 0; r < 3; ++r) dft_line<T, K, INV>(sr[r], si[r]);
    const auto w3 = tw<T, N>(K);
    const T half = w3.x;                  // -1/2
    const T c = INV ? w3.y : -w3.y;       // +-sqrt(3)/2: the sign of the forward form
#pragma unroll
    for (int k1 = 0; k1 < K; ++k1) {
        T zr[3], zi[3];
        zr[0] = sr[0][k1];
        zi[0] = si[0][k1];
#pragma unroll
        for (int r = 1; r < 3; ++r) {
            if (k1 == 0) {
                zr[r] = sr[r][k1];
                zi[r] = si[r][k1];
            } else {
                const auto w = tw<T, N>(r * k1);
                const T wr = w.x, wi = INV ? -w.y : w.y;
                zr[r] = sr[r][k1] * wr - si[r][k1] * wi;
                zi[r] = sr[r][k1] * wi + si[r][k1] * wr;
            }
        }
        const T tr = zr[1] + zr[2], ti = zi[1] + zi[2];
        const T dr = zr[1] - zr[2], di = zi[1] - zi[2];
        const T mr = zr[0] + tr * half, mi = zi[0] + ti * half;
        re[k1] = zr[0] + tr;
        im[k1] = zi[0] + ti;
        // forward: Z1 = m - i c d = (mr + c di, mi - c dr); Z2 = (mr - c di, mi + c dr)
        re[k1 + K] = mr + c * di;
        im[k1 + K] = mi - c * dr;
        re[k1 + 2 * K] = mr - c * di;
        im[k1 + 2 * K] = mi + c * dr;
    }
}

// In-register 1D DFT of length N (forward: exp(-2 pi i jk/N); INV: exp(+...)), unscaled.
// Radix-2 decimation in time for powers of two, one radix-3 step for 3 * 2^k, direct
// summation otherwise; every index is a compile-time constant after unrolling, so the line
// stays in registers.
template <typename T, int N, bool INV>
__device__ __forceinline__ void dft_line(T (&re)[N], T (&im)[N]) {
    if constexpr (N % 3 == 0 && is_pow2(N / 3) && N >= 12) {
        dft_line_radix3<T, N, INV>(re, im);
    } else if constexpr (is_pow2(N)) {
        constexpr int B = ilog2(N);
#pragma unroll
        for (int i = 0; i < N; ++i) {
            const int j = bitrev(i, B);
            if (j > i) {
                T t = re[i]; re[i] = re[j]; re[j] = t;
                t = im[i]; im[i] = im[j]; im[j] = t;
            }
        }
#pragma unroll
        for (int stage = 0; stage < B; ++stage) {
            const int len = 2 << stage;
#pragma unroll
            for (int i = 0; i < N; i += len) {
#pragma unroll
                for (int j = 0; j < len / 2; ++j) {
                    // m is a compile-time constant after unrolling: W^0 = 1, W^(N/4) = -i
                    // (+i inverse) are exact swaps, W^(N/8) and W^(3N/8) = (+-1 - i) sqrt(1/2)
                    // take two real products; the rest is the general complex product
                    const int m = j * (N / len);
                    const int a = i + j, b = i + j + len / 2;
                    T xr, xi;
                    if (m == 0) {
                        xr = re[b];
                        xi = im[b];
                    } else if (4 * m == N) {
                        if (INV) {
                            xr = -im[b];
                            xi = re[b];
                        } else {
                            xr = im[b];
                            xi = -re[b];
                        }
                    } else if (8 * m == N || 8 * m == 3 * N) {
                        const T c = tw<T, N>(N / 8).x;  // sqrt(1/2)
                        const T s = re[b] + im[b], d = im[b] - re[b];
                        if (8 * m == N) {  // forward (1 - i) c, inverse (1 + i) c
                            xr = INV ? -(c * d) : c * s;
                            xi = INV ? c * s : c * d;
                        } else {           // forward (-1 - i) c, inverse (-1 + i) c
                            xr = INV ? -(c * s) : c * d;
                            xi = INV ? -(c * d) : -(c * s);
                        }
                    } else {
                        const auto w = tw<T, N>(m);
                        const T wr = w.x, wi = INV ? -w.y : w.y;
                        xr = re[b] * wr - im[b] * wi;
                        xi = re[b] * wi + im[b] * wr;
                    }
                    re[b] = re[a] - xr;
                    im[b] = im[a] - xi;
                    re[a] = re[a] + xr;
                    im[a] = im[a] + xi;
                }
            }
        }
    } else {
        T orr[N], oi[N];
#pragma unroll
        for (int k = 0; k < N; ++k) {
            T ar = 0, ai = 0;
#pragma unroll
            for (int j = 0; j < N; ++j) {
                const auto w = tw<T, N>((j * k) % N);
                const T wr = w.x, wi = INV ? -w.y : w.y;
                ar += re[j] * wr - im[j] * wi;
                ai += re[j] * wi + im[j] * wr;
            }
            orr[k] = ar;
            oi[k] = ai;
        }
#pragma unroll
        for (int k = 0; k < N; ++k) {
            re[k] = orr[k];
            im[k] = oi[k];
        }
    }
}

// Deterministic block reduction of NV doubles (fixed tree for a fixed blockDim).
template <int NV>
__device__ __forceinline__ void block_reduce(double (&v)[NV], double* smem /*[32*NV]*/) {
#pragma unroll
    for (int k = 0; k < NV; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) smem[warp * NV + k] = v[k];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double s = (lane < nw) ? smem[lane * NV + k] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
            v[k] = s;
        }
    }
    __syncthreads();
}

// The same fixed-tree block reduction in double-float arithmetic: FP64-class sums that stay
// on the FP32 pipes (for kernels whose data are float).
template <int NV>
__device__ __forceinline__ void block_reduce_df(dfloat (&v)[NV], dfloat* smem /*[32*NV]*/) {
#pragma unroll
    for (int k = 0; k < NV; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const dfloat w(__shfl_down_sync(0xffffffffu, v[k].hi, o), __shfl_down_sync(0xffffffffu, v[k].lo, o));
            v[k] = v[k] + w;
        }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) smem[warp * NV + k] = v[k];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            dfloat s = (lane < nw) ? smem[lane * NV + k] : dfloat(0);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const dfloat w(__shfl_down_sync(0xffffffffu, s.hi, o), __shfl_down_sync(0xffffffffu, s.lo, o));
                s = s + w;
            }
            v[k] = s;
        }
    }
    __syncthreads();
}

}  // namespace lbe

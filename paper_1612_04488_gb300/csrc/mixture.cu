// Binary hard-sphere mixture (Sec. 4): the four linearized collision operators of a mixture
// as one dense matrix, built on the device from the Carleman form for unequal masses and
// applied as a GEMM (FP64, double-float on the FP32 pipes, or tcgen05 BF16 hi / lo through
// fsm_dense.cu), and the SIS of Eqs. LBE2_true1 / LBE2_true2 for Poiseuille flow between plates
// and through rectangular ducts, with defect correction for the mixed-precision solves.
//
// Operator (include/lbe.h has the full statement).  For species a colliding with b,
// mu_b = m_b / (m_a + m_b), c = mu_b - mu_a, and x ⊥ y: v* = v + x + y, v' = v + 2 mu_b x,
// v*' = v + c x + y; hard spheres give the constant kernel d_ab^2 = 4 b_ab, so in Fourier
// space (f_j = sum_l f^_l w^(l j), f^ = DFT / N^3)
//   F(Q+_ab(f, g))_k = sum_{l + m = k mod N} beta_ab(l, m) f^_l g^_m,
//   beta_ab(l, m) = sum_p 2 b_ab w_p phi((2 mu_b xi_l + c xi_m).e_p) psi_p(m),
// with the single-species phi, psi, hemisphere rule and truncation R; Nyquist l is zeroed
// in phi and Nyquist m in psi.  The linearized operator restricted to h_b, as a spectral
// matrix on h^ (row k, column m, l = k - m mod N):
//   K_ab[k, m] = f^_a(l) (beta_ab(l, m) - G_ab(m)) + [a = b] sum_c beta_ac(m, l) f^_c(l),
//   G_ab = sum_p 2 b_ab w_p phi_p psi_p (the loss, mass independent).
// The velocity-space matrix is F^-1 K F; separable passes along each velocity axis carry the
// columns to the unknown's basis (the full grid, or one value per orbit of the plate parity,
// even in v2 and odd in v3, or of the duct parity, odd in v3) and the rows to its
// representatives.  L+_a = sum_b K_ab h_b and
// L_a = L+_a - nu_a h_a with nu_a = sum_b F^-1(G_ab F f_b,eq).
//
// delta: b_AA = delta mu1 sqrt(2 / m) / 4 (units m_A = kT = d_A = 1, m = chi_A + chi_B m_B),
// mu1 the first Chapman-Enskog approximation of the mixture viscosity, b_ab = b_AA d_ab^2.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"
#include "lbe_internal.h"
#include "sweep.h"

namespace lbe {

struct MixOp {
    int nv = 0, M = 0, layout = 0;  // layout 0: full velocity grid, 1: plate orbit layout, 2: duct orbit layout
    double vmax = 0, R = 0;
    double r[2] = {1, 1}, d[2] = {1, 1}, chi[2] = {0.5, 0.5}, mbar = 1;
    int nr = 0;               // rows (= columns) of one species block
    double b0 = 0, mu1 = 0;   // b_AA at delta = 1, first-approximation viscosity
    double Nal[2] = {0, 0};   // N_a of Sec. 4 (independent of delta)
    double cU[2] = {0, 0};    // (2 r_a / chi_a) sum v3^2 f_a,eq dv^3 (discrete)
    double cq[2] = {0, 0};    // 2 r_a sum (r_a |v|^2 - 5/2) v3^2 f_a,eq dv^3
    double* L = nullptr;      // [2 nr][2 nr] row-major, delta = 1
    double* nu = nullptr;     // [2][n3] nu_a at delta = 1
    double* feq = nullptr;    // [2][n3]
    double* vel = nullptr;    // [nv]
    std::vector<double> nu_h; // host copy of nu
    size_t bytes = 0;
    DevTables tab[2];         // per species: the transport sweep's tables (vel, f_a,eq, nu_a)
    float2* Ldf = nullptr;    // L as double-float (hi, lo) pairs, built at first use
    float2* Xdf = nullptr;    // the cell operand as double-float pairs (grow-only)
    size_t xdf_bytes = 0;
    double* part = nullptr;   // split-K partial sums of the GEMM (grow-only)
    size_t part_bytes = 0;
    MixTc* tc = nullptr;      // the same operator in BF16 hi / lo on the tensor cores (first use)
    double* zero = nullptr;   // [n3] zeros: the source-free sweep's f_eq
    DevTables tab0[2];        // tab with a zero source (the correction equation's sweep)
    float* ftab = nullptr;    // float copies for the low-precision sweeps: f_eq [2][n3], nu [2][n3],
                              // zeros [n3], vel [nv]
};

namespace {

// First Chapman-Enskog approximation of the viscosity of a binary hard-sphere mixture in
// units m_A = kT = d_A = 1 (rigid spheres: every reduced collision integral is 1).
double viscosity1(double mB, double dB, double xA) {
    const double m1 = 1.0, m2 = mB, x1 = xA, x2 = 1.0 - xA, s12 = 0.5 * (1.0 + dB);
    const double e1 = 5.0 / 16.0 * std::sqrt(m1 / M_PI);
    const double e2 = 5.0 / 16.0 * std::sqrt(m2 / M_PI) / (dB * dB);
    const double e12 = 5.0 / 16.0 * std::sqrt(2.0 * m1 * m2 / (M_PI * (m1 + m2))) / (s12 * s12);
    const double q = (m1 + m2) * (m1 + m2) / (4.0 * m1 * m2);
    const double X = x1 * x1 / e1 + 2.0 * x1 * x2 / e12 + x2 * x2 / e2;
    const double Y = 0.6 * (x1 * x1 / e1 * (m1 / m2) + 2.0 * x1 * x2 / e12 * q * e12 * e12 / (e1 * e2) +
                            x2 * x2 / e2 * (m2 / m1));
    const double Z = 0.6 * (x1 * x1 * m1 / m2 + 2.0 * x1 * x2 * (q * (e12 / e1 + e12 / e2) - 1.0) +
                            x2 * x2 * m2 / m1);
    return (1.0 + Z) / (X + Y);
}

// T[p n3 + m] = (sin, cos)(f s_p(m))
__global__ void k_mix_trig(double2* __restrict__ T, const double* __restrict__ s, long total, double f) {
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
        double sn, cs;
        sincos(f * s[t], &sn, &cs);
        T[t] = make_double2(sn, cs);
    }
}

// beta[l n3 + m] = keep(l) sum_p wp[p] phi(x) psi_p(m), x = R (2 mu s_p(l) + c s_p(m)):
// phi = 2 R^2 [sin x / x - 2 sin^2(x/2) / x^2] = 4 R^2 sin(x/2) [cos(x/2) - sin(x/2) / x] / x,
// with sin and cos of x/2 = R mu s_p(l) + (R c / 2) s_p(m) by angle addition from the tables
// TL = (sin, cos)(R mu s_p(l)) and TM = (sin, cos)(R c s_p(m) / 2).
__global__ void __launch_bounds__(256) k_mix_beta(double* __restrict__ B, const double* __restrict__ s,
                                                  const double2* __restrict__ TL, const double2* __restrict__ TM,
                                                  const double* __restrict__ psi, const unsigned char* __restrict__ keep,
                                                  const double* __restrict__ wp, int M, long n3, double twomu,
                                                  double c, double R) {
    const long total = n3 * n3;
    const double R2 = R * R;
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
        const long l = t / n3, m = t - l * n3;
        double acc = 0.0;
        if (keep[l])
            for (int p = 0; p < M; ++p) {
                const long pl = p * n3 + l, pm = p * n3 + m;
                const double x = R * (twomu * s[pl] + c * s[pm]);
                double ph;
                if (fabs(x) < 1e-3) {
                    ph = R2 * (1.0 - x * x / 4.0 + x * x * x * x / 72.0);
                } else {
                    const double2 a = TL[pl], b = TM[pm];
                    const double sh = a.x * b.y + a.y * b.x, ch = a.y * b.y - a.x * b.x, inv = 1.0 / x;
                    ph = 4.0 * R2 * sh * inv * (ch - sh * inv);
                }
                acc += wp[p] * ph * psi[pm];
            }
        B[t] = acc;
    }
}

// spectral matrix of block (a, b) (file header): K[k n3 + m]
__global__ void __launch_bounds__(256) k_mix_fourier(double2* __restrict__ K, const double* __restrict__ Bab,
                                                     const double* __restrict__ Ba0, const double* __restrict__ Ba1,
                                                     const double2* __restrict__ fa, const double2* __restrict__ f0,
                                                     const double2* __restrict__ f1, const double* __restrict__ Gab,
                                                     int N, int diag) {
    const long n3 = (long)N * N * N, total = n3 * n3;
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
        const long k = t / n3, m = t - k * n3;
        const int k1 = (int)(k / (N * N)), k2 = (int)(k / N % N), k3 = (int)(k % N);
        const int m1 = (int)(m / (N * N)), m2 = (int)(m / N % N), m3 = (int)(m % N);
        const long l = ((long)((k1 - m1 + N) % N) * N + (k2 - m2 + N) % N) * N + (k3 - m3 + N) % N;
        const double g = Bab[l * n3 + m] - Gab[m];
        double re = fa[l].x * g, im = fa[l].y * g;
        if (diag) {
            const double b0 = Ba0[m * n3 + l], b1 = Ba1[m * n3 + l];
            re += b0 * f0[l].x + b1 * f1[l].x;
            im += b0 * f0[l].y + b1 * f1[l].y;
        }
        K[t] = make_double2(re, im);
    }
}

// Y[(o Nout + j) inner + i] = sum_a C[j Nin + a] X[(o Nin + a) inner + i]   (complex)
__global__ void __launch_bounds__(256) k_axis_pass(const double2* __restrict__ X, double2* __restrict__ Y,
                                                   const double2* __restrict__ C, long outer, int Nin, long inner,
                                                   int Nout) {
    const long total = outer * Nout * inner;
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
        const long i = t % inner, rr = t / inner;
        const int j = (int)(rr % Nout);
        const long o = rr / Nout;
        const double2* x = X + o * Nin * inner + i;
        const double2* cj = C + (long)j * Nin;
        double re = 0.0, im = 0.0;
        for (int a = 0; a < Nin; ++a) {
            const double2 cc = cj[a], xv = x[a * inner];
            re += cc.x * xv.x - cc.y * xv.y;
            im += cc.x * xv.y + cc.y * xv.x;
        }
        Y[t] = make_double2(re, im);
    }
}

__global__ void k_mix_store(double* __restrict__ L, const double2* __restrict__ Y, long nr, long ld, long row0,
                            long col0) {
    const long total = nr * nr;
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
        const long r = t / nr, c = t - r * nr;
        L[(row0 + r) * ld + col0 + c] = Y[t].x;
    }
}

// FP64 GEMM of the mixture operator: for species a and cell n,
//   y_a[n cs + j] = scale sum_{b, c} L[(a nr + j) 2nr + b nr + c] h_b[n cs + c].
// 64 x 64 output tile per block, 4 x 4 per thread, K in slices of 16.  With a cell list `map`
// (may be null) GEMM column n is cell map[n], in h and in y (the porous cell's fluid cells).
constexpr int kMT = 64, kNT = 64, kKT = 16;
// With a K split (gridDim.z > 1) slice z covers k in [z kc, (z+1) kc) and writes its unscaled
// partial sums to part[(z cells + cell) rows + row]; k_mix_reduce adds the slices in order.
__global__ void __launch_bounds__(256) k_mix_gemm(const double* __restrict__ L, int nr, const double* __restrict__ hA,
                                                  const double* __restrict__ hB, long cs, int cells, double scale,
                                                  double* __restrict__ yA, double* __restrict__ yB, int kc,
                                                  double* __restrict__ part, const int* __restrict__ map) {
    __shared__ double As[kKT][kMT + 1];
    __shared__ double Bs[kKT][kNT + 1];
    const int rows = 2 * nr, K = 2 * nr;
    const int row0 = blockIdx.x * kMT, cell0 = blockIdx.y * kNT;
    const int kb = blockIdx.z * kc, ke = min(K, kb + kc);
    const int t = threadIdx.x, ty = t / 16, tx = t % 16;
    double acc[4][4] = {};
    for (int k0 = kb; k0 < ke; k0 += kKT) {
        // A: 64 rows x 16 k, each thread 4 consecutive k of one row
        {
            const int r = t / 4, kq = (t % 4) * 4;
            const int gr = row0 + r;
            for (int q = 0; q < 4; ++q) {
                const int gk = k0 + kq + q;
                As[kq + q][r] = (gr < rows && gk < ke) ? L[(long)gr * K + gk] : 0.0;
            }
        }
        // B: 16 k x 64 cells, each thread 4 consecutive k of one cell
        {
            const int cc = t / 4, kq = (t % 4) * 4;
            const int gc = cell0 + cc;
            for (int q = 0; q < 4; ++q) {
                const int gk = k0 + kq + q;
                double v = 0.0;
                if (gc < cells && gk < ke) {
                    const long src = map ? map[gc] : gc;
                    v = gk < nr ? hA[src * cs + gk] : hB[src * cs + gk - nr];
                }
                Bs[kq + q][cc] = v;
            }
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kKT; ++k) {
            double a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[k][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[k][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
    if (part) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int gr = row0 + ty * 4 + i;
            if (gr >= rows) continue;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int gc = cell0 + tx * 4 + q;
                if (gc < cells) part[((long)blockIdx.z * cells + gc) * rows + gr] = acc[i][q];
            }
        }
        return;
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int gr = row0 + ty * 4 + i;
        if (gr >= rows) continue;
        double* y = gr < nr ? yA : yB;
        const int j = gr < nr ? gr : gr - nr;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int gc = cell0 + tx * 4 + q;
            if (gc < cells) y[(long)(map ? map[gc] : gc) * cs + j] = scale * acc[i][q];
        }
    }
}

// The same GEMM in double-float arithmetic on the FP32 pipes: L and the cell operand as (hi, lo)
// float pairs, each product formed exactly by FMA (TwoProduct, cross terms added) and
// accumulated by TwoSum; the pairs are renormalised after every K slice of the tile and widened
// to double at the end (about 1e-13 of the scale, against the FP64 kernel's rounding).
// X[cell][k] = both species' h of a cell as double-float pairs (once per GEMM, so the tiles read
// float pairs and the GEMM does no FP64 arithmetic)
__global__ void k_mix_h_to_df(const double* __restrict__ hA, const double* __restrict__ hB, long cs, int nr,
                              int cells, float2* __restrict__ X, const int* __restrict__ map) {
    const long K = 2L * nr, total = K * cells;
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
        const long n = t / K, k = t - n * K, c = map ? map[n] : n;
        const dfloat d(k < nr ? hA[c * cs + k] : hB[c * cs + k - nr]);
        X[t] = make_float2(d.hi, d.lo);
    }
}

__global__ void __launch_bounds__(256) k_mix_gemm_df(const float2* __restrict__ L, int nr,
                                                     const float2* __restrict__ X, long cs, int cells, double scale,
                                                     double* __restrict__ yA, double* __restrict__ yB, int kc,
                                                     double* __restrict__ part, const int* __restrict__ map) {
    __shared__ float2 As[kKT][kMT + 1];
    __shared__ float2 Bs[kKT][kNT + 1];
    const int rows = 2 * nr, K = 2 * nr;
    const int row0 = blockIdx.x * kMT, cell0 = blockIdx.y * kNT;
    const int kb = blockIdx.z * kc, ke = min(K, kb + kc);
    const int t = threadIdx.x, ty = t / 16, tx = t % 16;
    dfloat acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = dfloat(0.f, 0.f);
    for (int k0 = kb; k0 < ke; k0 += kKT) {
        {
            const int r = t / 4, kq = (t % 4) * 4;
            const int gr = row0 + r;
            for (int q = 0; q < 4; ++q) {
                const int gk = k0 + kq + q;
                As[kq + q][r] = (gr < rows && gk < ke) ? L[(long)gr * K + gk] : make_float2(0.f, 0.f);
            }
        }
        {
            const int cc = t / 4, kq = (t % 4) * 4;
            const int gc = cell0 + cc;
            for (int q = 0; q < 4; ++q) {
                const int gk = k0 + kq + q;
                Bs[kq + q][cc] = (gc < cells && gk < ke) ? X[(long)gc * K + gk] : make_float2(0.f, 0.f);
            }
        }
        __syncthreads();
#pragma unroll 4
        for (int k = 0; k < kKT; ++k) {
            dfloat a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = dfloat(As[k][ty * 4 + i].x, As[k][ty * 4 + i].y);
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = dfloat(Bs[k][tx * 4 + j].x, Bs[k][tx * 4 + j].y);
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * b[j];
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = df_fast2sum(acc[i][j].hi, acc[i][j].lo);
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int gr = row0 + ty * 4 + i;
        if (gr >= rows) continue;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int gc = cell0 + tx * 4 + q;
            if (gc >= cells) continue;
            const double v = (double)acc[i][q];
            if (part)
                part[((long)blockIdx.z * cells + gc) * rows + gr] = v;
            else
                (gr < nr ? yA : yB)[(long)(map ? map[gc] : gc) * cs + (gr < nr ? gr : gr - nr)] = scale * v;
        }
    }
}

__global__ void k_mix_to_df(const double* __restrict__ L, long n, float2* __restrict__ out) {
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < n; t += (long)gridDim.x * blockDim.x) {
        const dfloat d(L[t]);
        out[t] = make_float2(d.hi, d.lo);
    }
}

// y = scale * sum_z part[z] in slice order (deterministic)
__global__ void k_mix_reduce(const double* __restrict__ part, int nsplit, int nr, int cells, long cs, double scale,
                             double* __restrict__ yA, double* __restrict__ yB, const int* __restrict__ map) {
    const long rows = 2L * nr, total = rows * cells;
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
        const long gc = t / rows, gr = t - gc * rows;
        double v = 0.0;
        for (int z = 0; z < nsplit; ++z) v += part[((long)z * cells + gc) * rows + gr];
        (gr < nr ? yA : yB)[(map ? map[gc] : gc) * cs + (gr < nr ? gr : gr - nr)] = scale * v;
    }
}

// L_a = L+_a - delta nu_a h_a over cells x n3 (full layout)
__global__ void k_mix_loss(const double* __restrict__ lp, const double* __restrict__ h, const double* __restrict__ nu,
                           double delta, long n3, long total, double* __restrict__ L) {
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x)
        L[t] = lp[t] - delta * nu[t % n3] * h[t];
}

// ---- SIS kernels.  Orbit layouts, cell stride nv^3: plates keep the nq = nv^3 / 4 values at
// (i1 H + j2) H + j3 with j2, j3 < H = nv / 2; ducts the nv^3 / 2 values at (i1 nv + i2) H + j3 --
struct MixSisDev {
    double r[2], chi[2], Nd[2], delta, dv3, sqm;
    double cU[2], cq[2];
    int nv, cells, sis;
    int src;     // 1: the problem's own iteration; 0: the source-free one of the correction equation
    int layout;  // 1 plates (one value per orbit of {1, R2, R3, R2 R3}), 2 ducts ({1, R3})
};
constexpr int kMom = 9;  // per cell: U, q, W1, P13, G1, W2, X12, P23, G2

// the representative q of the orbit layout -> (i1, i2, i3) and the orbit size
__device__ __forceinline__ void orbit_point(int q, int N, int layout, int* i1, int* i2, int* i3) {
    const int H = N / 2, E2 = layout == 1 ? H : N;
    *i1 = q / (E2 * H);
    *i2 = q / H % E2;
    *i3 = q % H;
}

// per (cell, species): mom[(a cells + n) kMom + .] = {U, q, W1, P13, G1, W2, X12, P23, G2}: U, q,
// W1 = F201/4, P13, W2 = F021/4, X12 = F111/4, P23 of h^(k+1/2) and G_j of L h^(k), h^(k); sums
// over the orbit representatives times the orbit size (4 plates, 2 ducts).  A thread takes whole
// rows (i1, i2) of the layout: it sums v3 x, v3^3 x (x = h^(k+1/2)) and the G integrand along
// i3, then applies the row's (v1, v2) weights once.
template <typename T>
__global__ void __launch_bounds__(256) k_mix_moments(MixSisDev P, const T* __restrict__ hh,
                                                     const double* __restrict__ h, const T* __restrict__ lp,
                                                     const double* __restrict__ nu, const double* __restrict__ vel,
                                                     double* __restrict__ mom) {
    const int n = blockIdx.x, a = blockIdx.y, N = P.nv, H = N / 2;
    const int E2 = P.layout == 1 ? H : N, rows = N * E2;
    const long n3 = (long)N * N * N, off = ((long)a * P.cells + n) * n3;
    const double r = P.r[a], Nd = P.Nd[a], dl = P.delta;
    const double* __restrict__ nua = nu + a * n3;
    double s[kMom] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int row = threadIdx.x; row < rows; row += blockDim.x) {
        const int i1 = row / E2, i2 = row - i1 * E2;
        const long o = off + (long)row * H, vf = ((long)i1 * N + i2) * N;
        double A0 = 0.0, A1 = 0.0, B0 = 0.0;
        for (int i3 = 0; i3 < H; ++i3) {
            const double v3 = vel[i3];
            const double x = (double)hh[o + i3] * v3;
            A0 += x;
            A1 += v3 * v3 * x;
            if (P.sis) B0 += ((double)lp[o + i3] + (Nd - dl * nua[vf + i3]) * h[o + i3]) * v3;
        }
        const double v1 = vel[i1], v2 = vel[i2];
        s[0] += A0;
        s[1] += (r * (v1 * v1 + v2 * v2) - 2.5) * A0 + r * A1;
        s[2] += (2.0 * v1 * v1 - 1.0) * A0;
        s[3] += v1 * A0;
        s[5] += (2.0 * v2 * v2 - 1.0) * A0;
        s[6] += v1 * v2 * A0;
        s[7] += v2 * A0;
        s[4] += v1 * B0;
        s[8] += v2 * B0;
    }
    __shared__ double red[kMom][8];
    for (int k = 0; k < kMom; ++k) {
        double v = s[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) red[k][threadIdx.x >> 5] = v;
    }
    __syncthreads();
    if (threadIdx.x < kMom) {
        const int k = threadIdx.x;
        double v = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[k][w];
        const double wq = (P.layout == 1 ? 4.0 : 2.0) * P.dv3;
        const double scl = k == 0 ? wq / P.chi[a] : (k == 3 || k == 7) ? 2.0 * r * wq
                         : (k == 4 || k == 6 || k == 8) ? 2.0 * wq : wq;
        mom[((long)a * P.cells + n) * kMom + k] = v * scl;
    }
}

// one thread per species: the once-integrated diffusion equation marched from the wall,
// d(chi U + W)/dx1 = G - (N delta / r) P~, P~_B = P_B, P~_A = x1 - P_B (P~_A = -P_B without the
// source); dU, the corrected U and q, and the flow rates M_a = sqrt(m) sum trap U,
// Q_a = sqrt(m) sum trap q.  The block first stages the moments and the node coefficients in
// shared memory (the march itself is a short serial recurrence).
constexpr int kMarchMax = 1001;
__global__ void __launch_bounds__(256) k_mix_march(MixSisDev P, const double* __restrict__ mom,
                                                   const double* __restrict__ geo, double* __restrict__ dU,
                                                   double* __restrict__ Uout, double* __restrict__ rates) {
    extern __shared__ double sm[];  // [2 kMom n] moments, [5 n] geometry
    const int n = P.cells;
    for (int i = threadIdx.x; i < 2 * kMom * n; i += blockDim.x) sm[i] = mom[i];
    for (int i = threadIdx.x; i < 5 * n; i += blockDim.x) sm[2 * kMom * n + i] = geo[i];
    __syncthreads();
    const int a = threadIdx.x;
    if (a >= 2) return;
    // ia: reciprocals of the stencil's diagonal (host)
    const double *x = sm + 2 * kMom * n, *ia = x + n, *fb = x + 2 * n, *fc = x + 3 * n, *trap = x + 4 * n;
    const double* ma = sm + a * n * kMom;
    const double* mB = sm + n * kMom;
    const double kN = P.Nd[a] / P.r[a], chi = P.chi[a], cU = P.cU[a], cq = P.cq[a];
    double Mr = 0.0, Qr = 0.0, y1 = 0.0, y2 = 0.0;
    for (int i = 0; i < n; ++i) {
        const double U = ma[kMom * i], q = ma[kMom * i + 1], W = ma[kMom * i + 2];
        double d = 0.0;
        if (P.sis) {
            double Y;
            if (i == 0) {
                Y = chi * U + W;
            } else {
                const double Pt = a == 0 ? (P.src ? x[i] : 0.0) - mB[kMom * i + 3] : mB[kMom * i + 3];
                double sr = ma[kMom * i + 4] - kN * Pt - fb[i] * y1;
                if (i >= 2) sr -= fc[i] * y2;
                Y = sr * ia[i];
            }
            y2 = y1;
            y1 = Y;
            d = (Y - W) / chi - U;
        }
        dU[a * n + i] = d;
        const double Uc = U + d * cU, qc = q + d * cq;
        Uout[a * n + i] = Uc;
        Mr += trap[i] * Uc;
        Qr += trap[i] * qc;
    }
    rates[a] = P.sqm * Mr;
    rates[2 + a] = P.sqm * Qr;
}

// Ducts: one block per species solves Eqs. LBE2_true1 / LBE2_true2 on the interior
// mx x my = (nx - 2) x (ny - 2) cells (cell (i, j) at i ny + j), U = U^(k+1/2) on the ring:
//   chi_a lap U_a = -(N_a delta / r_a) D_a - (d11 W1 + 2 d12 X12 + d22 W2) + d1 G1 + d2 G2,
// D_B = d1 P_B13 + d2 P_B23, D_A = 1 - D_B (-D_B without the source), five-point Laplacian and
// central differences; by the DST-I: U = Sx ((Sx R Sy) ./ lam) Sy (Sx, Sy orthonormal and
// symmetric).  Then dU, the corrected U and q, and the flow rates sqrt(m) times cell means.
struct MixDuctDev {
    int nx, ny;
    double dx, dy;
};
__global__ void __launch_bounds__(512) k_mix_poisson2d(MixSisDev P, MixDuctDev D, const double* __restrict__ mom,
                                                       const double* __restrict__ Sx, const double* __restrict__ Sy,
                                                       const double* __restrict__ lam, double* __restrict__ work,
                                                       double* __restrict__ dU, double* __restrict__ Uout,
                                                       double* __restrict__ rates) {
    const int a = blockIdx.x, nx = D.nx, ny = D.ny, mx = nx - 2, my = ny - 2, n = P.cells;
    const long mm = (long)mx * my;
    double* B = work + a * 2 * mm;
    double* T1 = B + mm;
    auto M = [&](int sp, int i, int j, int k) { return mom[((long)sp * n + (long)i * ny + j) * kMom + k]; };
    if (P.sis) {
        const double dx = D.dx, dy = D.dy, kN = P.Nd[a] / P.r[a], chi = P.chi[a];
        for (long k = threadIdx.x; k < mm; k += blockDim.x) {
            const int p = (int)(k / my), q = (int)(k % my), i = p + 1, j = q + 1;
            auto d1 = [&](int sp, int c) { return (M(sp, i + 1, j, c) - M(sp, i - 1, j, c)) / (2.0 * dx); };
            auto d2 = [&](int sp, int c) { return (M(sp, i, j + 1, c) - M(sp, i, j - 1, c)) / (2.0 * dy); };
            const double DB = d1(1, 3) + d2(1, 7);
            const double Dd = a == 0 ? (P.src ? 1.0 : 0.0) - DB : DB;
            double b = -kN * Dd - (M(a, i + 1, j, 2) - 2.0 * M(a, i, j, 2) + M(a, i - 1, j, 2)) / (dx * dx) -
                       2.0 * (M(a, i + 1, j + 1, 6) - M(a, i + 1, j - 1, 6) - M(a, i - 1, j + 1, 6) +
                              M(a, i - 1, j - 1, 6)) / (4.0 * dx * dy) -
                       (M(a, i, j + 1, 5) - 2.0 * M(a, i, j, 5) + M(a, i, j - 1, 5)) / (dy * dy) + d1(a, 4) +
                       d2(a, 8);
            b /= chi;
            if (p == 0) b -= M(a, 0, j, 0) / (dx * dx);
            if (p == mx - 1) b -= M(a, nx - 1, j, 0) / (dx * dx);
            if (q == 0) b -= M(a, i, 0, 0) / (dy * dy);
            if (q == my - 1) b -= M(a, i, ny - 1, 0) / (dy * dy);
            B[k] = b;
        }
        __syncthreads();
        // T1 = Sx B; B = (T1 Sy) ./ lam; T1 = Sx B; B = T1 Sy
        for (int stage = 0; stage < 4; ++stage) {
            const bool left = stage % 2 == 0;
            const double* X = left ? B : T1;
            double* Yv = left ? T1 : B;
            for (long k = threadIdx.x; k < mm; k += blockDim.x) {
                const int p = (int)(k / my), q = (int)(k % my);
                double v = 0.0;
                if (left)
                    for (int t = 0; t < mx; ++t) v += Sx[(long)p * mx + t] * X[(long)t * my + q];
                else
                    for (int t = 0; t < my; ++t) v += X[(long)p * my + t] * Sy[(long)t * my + q];
                if (stage == 1) v /= lam[k];
                Yv[k] = v;
            }
            __syncthreads();
        }
    }
    double sU = 0.0, sq = 0.0;
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
        const int i = c / ny, j = c % ny;
        const double Uh = M(a, i, j, 0), q = M(a, i, j, 1);
        const bool in = i > 0 && i < nx - 1 && j > 0 && j < ny - 1;
        const double d = (P.sis && in) ? B[(long)(i - 1) * my + (j - 1)] - Uh : 0.0;
        dU[a * n + c] = d;
        const double Uc = Uh + d * P.cU[a];
        Uout[a * n + c] = Uc;
        sU += Uc;
        sq += q + d * P.cq[a];
    }
    __shared__ double red[2][16];
    for (int o = 16; o > 0; o >>= 1) {
        sU += __shfl_xor_sync(0xffffffffu, sU, o);
        sq += __shfl_xor_sync(0xffffffffu, sq, o);
    }
    if ((threadIdx.x & 31) == 0) red[0][threadIdx.x >> 5] = sU, red[1][threadIdx.x >> 5] = sq;
    __syncthreads();
    if (threadIdx.x == 0) {
        double u = 0.0, v = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) u += red[0][w], v += red[1][w];
        rates[a] = P.sqm * u / n;
        rates[2 + a] = P.sqm * v / n;
    }
}

// ---- the periodic unit cell with solid cells (a square array of cylinders) -----------------------
// Upwind derivative weights along one direction of the march (spacing d): `u` a fluid line,
// `w1` a solid upwind neighbour (first order from its face, where the diffuse wall emits h = 0),
// `w2` a solid second neighbour (three points through that face).
struct PorousDev {
    int n;
    double ua, ub, uc, w1a, w2a, w2b;
};

// The two species' operands of one porous sweep (per species: L h, h, nu / delta, v, v3 feq).
template <typename T>
struct PorousSweepArgs {
    const T* rhs[2];
    T* h[2];
    const T* nu1[2];
    const T* vel[2];
    const T* feq[2];
};

constexpr int kPorousSweepWarps = 16;

// nu h + v1 dh/dx1 + v2 dh/dx2 = rhs + v3 feq (feq = 0: no source) for every velocity of the duct
// orbit layout (i1, i2, j3 < nv / 2), in place in h: the cells are taken in upwind order of the
// velocity's (v1, v2) quadrant, so a periodic neighbour not yet swept still holds the previous
// sweep's value; solid cells are set to zero.  In upwind coordinates (ii, jj) a cell depends on
// (ii - 1, jj), (ii - 2, jj), (ii, jj - 1), (ii, jj - 2) of this sweep, and on wrapped
// neighbours that lie on a later anti-diagonal ii + jj, so the anti-diagonals are swept in order
// and the cells of one anti-diagonal in parallel: the values read are those of the sequential
// row-by-row sweep.  Block: 32 consecutive velocities (lanes) of species blockIdx.y, its warps
// taking the cells of each anti-diagonal in turn, a block barrier between anti-diagonals.
template <typename T>
__global__ void __launch_bounds__(32 * kPorousSweepWarps, 3) k_mix_sweep_porous(PorousSweepArgs<T> A,
                                                                          const unsigned char* __restrict__ solid,
                                                                          PorousDev G, int nv, double delta) {
    const int H = nv / 2, sp = blockIdx.y, w = threadIdx.x >> 5, W = blockDim.x >> 5;
    const int q = blockIdx.x * 32 + (threadIdx.x & 31);
    const bool live = q < nv * nv * H;
    const long n3 = (long)nv * nv * nv;
    const int i1 = live ? q / (nv * H) : 0, i2 = live ? q / H % nv : 0, j3 = live ? q % H : 0;
    const long vf = ((long)i1 * nv + i2) * nv + j3;
    // species by selection, not by a runtime index into the parameter struct
    const T* __restrict__ rhs = sp ? A.rhs[1] : A.rhs[0];
    T* h = sp ? A.h[1] : A.h[0];
    const T* vel = sp ? A.vel[1] : A.vel[0];
    const T v1 = vel[i1], v2 = vel[i2];
    const int s1 = v1 > T(0) ? 1 : -1, s2 = v2 > T(0) ? 1 : -1;
    const T u1 = v1 > T(0) ? v1 : -v1, u2 = v2 > T(0) ? v2 : -v2;
    const T nu = (T)delta * (sp ? A.nu1[1] : A.nu1[0])[vf], S = vel[j3] * (sp ? A.feq[1] : A.feq[0])[vf];
    const int n = G.n;
    auto at = [&](int i, int j) -> long { return ((long)i * n + j) * n3 + q; };
    for (int d = 0; d <= 2 * (n - 1); ++d) {
        if (live)
            for (int jj = (d > n - 1 ? d - (n - 1) : 0) + w; jj <= d && jj < n; jj += W) {
                const int ii = d - jj;
                const int j = s2 > 0 ? jj : n - 1 - jj, i = s1 > 0 ? ii : n - 1 - ii;
                if (solid[i * n + j]) {
                    h[at(i, j)] = T(0);
                    continue;
                }
                const int j1 = (j - s2 + n) % n, j2 = (j - 2 * s2 + 2 * n) % n;
                const int i1c = (i - s1 + n) % n, i2c = (i - 2 * s1 + 2 * n) % n;
                T ax, bx, cx, ay, by, cy;
                if (solid[i1c * n + j]) ax = (T)G.w1a, bx = T(0), cx = T(0);
                else if (solid[i2c * n + j]) ax = (T)G.w2a, bx = (T)G.w2b, cx = T(0);
                else ax = (T)G.ua, bx = (T)G.ub, cx = (T)G.uc;
                if (solid[i * n + j1]) ay = (T)G.w1a, by = T(0), cy = T(0);
                else if (solid[i * n + j2]) ay = (T)G.w2a, by = (T)G.w2b, cy = T(0);
                else ay = (T)G.ua, by = (T)G.ub, cy = (T)G.uc;
                T num = rhs[at(i, j)] + S;
                if (bx != T(0)) num -= u1 * bx * h[at(i1c, j)];
                if (cx != T(0)) num -= u1 * cx * h[at(i2c, j)];
                if (by != T(0)) num -= u2 * by * h[at(i, j1)];
                if (cy != T(0)) num -= u2 * cy * h[at(i, j2)];
                h[at(i, j)] = num / (nu + u1 * ax + u2 * ay);
            }
        __syncthreads();
    }
}

template <typename T>
void launch_sweep_porous(const T* rhs, T* h, long per, const DevTables* tb, bool f32, const unsigned char* solid,
                         const PorousDev& G, int nv, double delta, cudaStream_t s) {
    PorousSweepArgs<T> A;
    for (int a = 0; a < 2; ++a) {
        A.rhs[a] = rhs + a * per;
        A.h[a] = h + a * per;
        A.nu1[a] = (const T*)(f32 ? (const void*)tb[a].nu1_f : (const void*)tb[a].nu1_d);
        A.vel[a] = (const T*)(f32 ? (const void*)tb[a].vel_f : (const void*)tb[a].vel_d);
        A.feq[a] = (const T*)(f32 ? (const void*)tb[a].feq_f : (const void*)tb[a].feq_d);
    }
    const int nq = nv * nv * (nv / 2);
    k_mix_sweep_porous<T><<<dim3((nq + 31) / 32, 2), 32 * kPorousSweepWarps, 0, s>>>(A, solid, G, nv, delta);
}

// One block per species: Eqs. LBE2_true1 / LBE2_true2 on the m interior cells (fluid cells whose
// eight periodic neighbours are fluid; list `inner`, and per interior cell its four neighbours
// `nb` as an interior index k >= 0 or a ring cell -1 - cell), the other fluid cells held at
// U^(k+1/2), periodic central differences; solved by conjugate gradients on -lap (symmetric
// positive definite) to a residual of rtol times the right-hand side (at most 20000 steps).  Then
// dU, the corrected U and q, and the flow rates sqrt(m) times means over all n^2 cells.
__global__ void __launch_bounds__(1024) k_mix_poisson_porous(MixSisDev P, PorousDev G, const double* __restrict__ mom,
                                                             const int* __restrict__ inner, const int* __restrict__ nb,
                                                             int m, double* __restrict__ work,
                                                             double* __restrict__ dU, double* __restrict__ Uout,
                                                             double* __restrict__ rates, int* __restrict__ cg_steps,
                                                             double rtol) {
    const int a = blockIdx.x, n = G.n, ncell = n * n;
    const double d = 1.0 / n, id2 = 1.0 / (d * d);
    double* x = work + (long)a * 5 * m;
    double* r = x + m;
    double* p = r + m;
    double* Ap = p + m;
    double* b = Ap + m;
    auto M = [&](int sp, int cell, int k) { return mom[((long)sp * ncell + cell) * kMom + k]; };
    __shared__ double red[32];
    __shared__ double bc;
    auto block_sum = [&](double v) -> double {
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        __syncthreads();
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
            bc = t;
        }
        __syncthreads();
        return bc;
    };
    if (P.sis) {
        const double kN = P.Nd[a] / P.r[a], chi = P.chi[a];
        for (int k = threadIdx.x; k < m; k += blockDim.x) {
            const int c = inner[k], i = c / n, j = c % n;
            auto C = [&](int di, int dj) { return ((i + di + n) % n) * n + (j + dj + n) % n; };
            auto d1 = [&](int sp, int q) { return (M(sp, C(1, 0), q) - M(sp, C(-1, 0), q)) / (2.0 * d); };
            auto d2 = [&](int sp, int q) { return (M(sp, C(0, 1), q) - M(sp, C(0, -1), q)) / (2.0 * d); };
            const double DB = d1(1, 3) + d2(1, 7);
            const double Dd = a == 0 ? (P.src ? 1.0 : 0.0) - DB : DB;
            double v = -kN * Dd - (M(a, C(1, 0), 2) - 2.0 * M(a, c, 2) + M(a, C(-1, 0), 2)) * id2 -
                       2.0 * (M(a, C(1, 1), 6) - M(a, C(1, -1), 6) - M(a, C(-1, 1), 6) + M(a, C(-1, -1), 6)) /
                           (4.0 * d * d) -
                       (M(a, C(0, 1), 5) - 2.0 * M(a, c, 5) + M(a, C(0, -1), 5)) * id2 + d1(a, 4) + d2(a, 8);
            v /= chi;
            for (int e = 0; e < 4; ++e) {
                const int t = nb[4 * k + e];
                if (t < 0) v -= M(a, -1 - t, 0) * id2;
            }
            b[k] = -v;                   // -lap U = -rhs: positive definite
            x[k] = M(a, c, 0);           // start from U^(k+1/2)
        }
        __syncthreads();
        auto apply = [&](const double* y, double* z) {  // z = -lap y on the interior (ring terms in b)
            for (int k = threadIdx.x; k < m; k += blockDim.x) {
                double v = 4.0 * y[k];
                for (int e = 0; e < 4; ++e) {
                    const int t = nb[4 * k + e];
                    if (t >= 0) v -= y[t];
                }
                z[k] = v * id2;
            }
            __syncthreads();
        };
        apply(x, Ap);
        double rr = 0.0, bb = 0.0;
        for (int k = threadIdx.x; k < m; k += blockDim.x) {
            r[k] = b[k] - Ap[k];
            p[k] = r[k];
            rr += r[k] * r[k];
            bb += b[k] * b[k];
        }
        rr = block_sum(rr);
        bb = block_sum(bb);
        int it = 0;
        const double tol = rtol * rtol * (bb > 0.0 ? bb : 1.0);
        while (rr > tol && it < 20000) {
            apply(p, Ap);
            double pAp = 0.0;
            for (int k = threadIdx.x; k < m; k += blockDim.x) pAp += p[k] * Ap[k];
            pAp = block_sum(pAp);
            const double al = rr / pAp;
            double rn = 0.0;
            for (int k = threadIdx.x; k < m; k += blockDim.x) {
                x[k] += al * p[k];
                r[k] -= al * Ap[k];
                rn += r[k] * r[k];
            }
            rn = block_sum(rn);
            const double be = rn / rr;
            rr = rn;
            for (int k = threadIdx.x; k < m; k += blockDim.x) p[k] = r[k] + be * p[k];
            __syncthreads();
            ++it;
        }
        if (threadIdx.x == 0) cg_steps[a] = it;
    }
    // interior cells: the solved U; everything else keeps U^(k+1/2) (solid cells hold zero)
    for (int c = threadIdx.x; c < ncell; c += blockDim.x) dU[a * ncell + c] = 0.0;
    __syncthreads();
    if (P.sis)
        for (int k = threadIdx.x; k < m; k += blockDim.x) {
            const int c = inner[k];
            dU[a * ncell + c] = x[k] - M(a, c, 0);
        }
    __syncthreads();
    double sU = 0.0, sq = 0.0;
    for (int c = threadIdx.x; c < ncell; c += blockDim.x) {
        const double dd = dU[a * ncell + c];
        const double Uc = M(a, c, 0) + dd * P.cU[a];
        Uout[a * ncell + c] = Uc;
        sU += Uc;
        sq += M(a, c, 1) + dd * P.cq[a];
    }
    sU = block_sum(sU);
    sq = block_sum(sq);
    if (threadIdx.x == 0) {
        rates[a] = P.sqm * sU / ncell;
        rates[2 + a] = P.sqm * sq / ncell;
    }
}

// y = x (float to double), the porous sweep's lag state when the iteration leaves float
__global__ void k_mix_widen(const float* __restrict__ x, long n, double* __restrict__ y) {
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < n; t += (long)gridDim.x * blockDim.x)
        y[t] = (double)x[t];
}

// x += y (float state plus a double increment), y += x (double plus float)
__global__ void k_mix_add_fd(float* __restrict__ x, const double* __restrict__ y, long n) {
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < n; t += (long)gridDim.x * blockDim.x)
        x[t] = (float)((double)x[t] + y[t]);
}
__global__ void k_mix_add_df(double* __restrict__ y, const float* __restrict__ x, long n) {
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < n; t += (long)gridDim.x * blockDim.x)
        y[t] += (double)x[t];
}

// y = a + s b over n values
__global__ void k_mix_axpy(const double* __restrict__ a, double s, const double* __restrict__ b, long n,
                           double* __restrict__ y) {
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < n; t += (long)gridDim.x * blockDim.x)
        y[t] = a[t] + s * b[t];
}

// h_a = hh_a + 2 r_a dU_a v3 f_a,eq on the representatives
template <typename T>
__global__ void __launch_bounds__(256) k_mix_correct(MixSisDev P, const T* __restrict__ hh,
                                                     double* __restrict__ h, const double* __restrict__ dU,
                                                     const double* __restrict__ feq, const double* __restrict__ vel) {
    // thread: orbit representative q; blocks in y walk the (species, cell) pairs
    const int N = P.nv, H = N / 2, nq = N * (P.layout == 1 ? H : N) * H;
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nq) return;
    const long n3 = (long)N * N * N;
    int i1, i2, i3;
    orbit_point(q, N, P.layout, &i1, &i2, &i3);
    const long vf = ((long)i1 * N + i2) * N + i3;
    const double c0 = 2.0 * P.r[0] * vel[i3] * feq[vf], c1 = 2.0 * P.r[1] * vel[i3] * feq[n3 + vf];
    for (long an = blockIdx.y; an < 2L * P.cells; an += gridDim.y) {
        const long off = an * n3 + q;
        h[off] = (double)hh[off] + dU[an] * (an < P.cells ? c0 : c1);
    }
}

// h = h^(k+1/2) + 2 r_a dU v3 f_a,eq on every (species, cell) of the orbit layout
template <typename T>
void launch_correct(const MixSisDev& P, const T* hh, double* h, const double* dU, const double* feq,
                    const double* vel, int nq, cudaStream_t s) {
    const long pairs = 2L * P.cells;
    const dim3 g((nq + 255) / 256, (unsigned)(pairs < 8192 ? pairs : 8192));
    k_mix_correct<T><<<g, 256, 0, s>>>(P, hh, h, dU, feq, vel);
}

int grid_for(long total) {
    const long g = (total + 255) / 256;
    const long cap = 32L * sm_count();
    return (int)(g < cap ? g : cap);
}

std::string mix_key(const lbe_mixture& m, int nv, double vmax, int M, double R, int layout) {
    char b[256];
    snprintf(b, sizeof b, "%.17g/%.17g/%.17g/%d/%.17g/%d/%.17g/%d", m.mass_ratio, m.diam_ratio, m.chi_A, nv, vmax, M,
             R, layout);
    return b;
}

lbe_status check_mixture(Ctx* c, const lbe_mixture* m, int nv, double vmax, int M, double R) {
    if (!m) return bad_arg(c, "null mixture");
    if (!(m->mass_ratio > 0) || !(m->diam_ratio > 0) || !(m->chi_A > 0 && m->chi_A < 1))
        return bad_arg(c, "mixture: mass_ratio, diam_ratio > 0 and 0 < chi_A < 1");
    if (nv < 4 || nv > 32 || nv % 4) return bad_arg(c, "mixture: nv must be a multiple of 4 in 4..32");
    if (!(vmax > 0) || M < 2 || M > 64 || (M & (M - 1))) return bad_arg(c, "mixture: vmax > 0, M a power of two <= 64");
    if (!(R > 0)) return bad_arg(c, "mixture: R must be > 0");
    return LBE_OK;
}

void free_mixop(Ctx* c, MixOp* o) {
    if (!o) return;
    if (o->L) dev_free(c, o->L, sizeof(double) * 4 * (size_t)o->nr * o->nr);
    const size_t n3 = (size_t)o->nv * o->nv * o->nv;
    if (o->nu) dev_free(c, o->nu, sizeof(double) * 2 * n3);
    if (o->feq) dev_free(c, o->feq, sizeof(double) * 2 * n3);
    if (o->vel) dev_free(c, o->vel, sizeof(double) * o->nv);
    if (o->part) dev_free(c, o->part, o->part_bytes);
    if (o->Ldf) dev_free(c, o->Ldf, sizeof(float2) * 4 * (size_t)o->nr * o->nr);
    if (o->Xdf) dev_free(c, o->Xdf, o->xdf_bytes);
    if (o->tc) mix_tc_release(c, o->tc);
    if (o->zero) dev_free(c, o->zero, sizeof(double) * n3);
    if (o->ftab) dev_free(c, o->ftab, sizeof(float) * (5 * n3 + o->nv));
    delete o;
}

lbe_status build_mixop(Ctx* c, MixOp& o, cudaStream_t s) {
    const int N = o.nv, H = N / 2, M = o.M;
    const long n3 = (long)N * N * N;
    const double dv = 2.0 * o.vmax / N, dv3 = dv * dv * dv;
    std::vector<double> v(N);
    for (int j = 0; j < N; ++j) v[j] = -o.vmax + (j + 0.5) * dv;
    std::vector<double> e, w;
    hemisphere_rule(M, e, w);
    // Maxwellians and their spectra
    std::vector<double> feq(2 * n3);
    std::vector<std::vector<std::complex<double>>> fh(2, std::vector<std::complex<double>>(n3));
    for (int a = 0; a < 2; ++a) {
        const double pre = o.chi[a] * std::pow(o.r[a] / M_PI, 1.5);
        for (long i = 0; i < n3; ++i) {
            const double c2 = v[i / (N * N)] * v[i / (N * N)] + v[i / N % N] * v[i / N % N] + v[i % N] * v[i % N];
            feq[a * n3 + i] = pre * std::exp(-o.r[a] * c2);
            fh[a][i] = feq[a * n3 + i];
        }
        host_dft3(fh[a], N, -1);
        for (auto& z : fh[a]) z /= (double)n3;
    }
    // direction factors per mode
    std::vector<double> xi(N);
    for (int k = 0; k < N; ++k) xi[k] = ((k < N / 2) ? k : k - N) * M_PI / o.vmax;
    std::vector<double> sp((size_t)M * n3), ps((size_t)M * n3), phown((size_t)M * n3);
    std::vector<unsigned char> keep(n3);
    for (long m = 0; m < n3; ++m) {
        const int a1 = (int)(m / (N * N)), a2 = (int)(m / N % N), a3 = (int)(m % N);
        keep[m] = (a1 != N / 2 && a2 != N / 2 && a3 != N / 2);
        const double x2 = xi[a1] * xi[a1] + xi[a2] * xi[a2] + xi[a3] * xi[a3];
        for (int p = 0; p < M; ++p) {
            const double sv = xi[a1] * e[3 * p] + xi[a2] * e[3 * p + 1] + xi[a3] * e[3 * p + 2];
            sp[(size_t)p * n3 + m] = sv;
            ps[(size_t)p * n3 + m] = keep[m] ? carleman_psi(std::sqrt(std::max(x2 - sv * sv, 0.0)), o.R) : 0.0;
            phown[(size_t)p * n3 + m] = keep[m] ? carleman_phi(sv, o.R) : 0.0;
        }
    }
    auto bab = [&](int a, int b) {
        const double dab = 0.5 * (o.d[a] + o.d[b]) / o.d[0];
        return o.b0 * dab * dab;
    };
    // loss multipliers G_ab and nu_a = sum_b F^-1(G_ab F f_b)
    std::vector<double> G(4 * n3, 0.0);
    o.nu_h.assign(2 * n3, 0.0);
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
            double* g = &G[(2 * a + b) * n3];
            for (int p = 0; p < M; ++p) {
                const double wpp = 2.0 * bab(a, b) * w[p];
                for (long m = 0; m < n3; ++m) g[m] += wpp * phown[(size_t)p * n3 + m] * ps[(size_t)p * n3 + m];
            }
            std::vector<std::complex<double>> z(n3);
            for (long m = 0; m < n3; ++m) z[m] = g[m] * fh[b][m];
            host_dft3(z, N, +1);
            for (long i = 0; i < n3; ++i) o.nu_h[a * n3 + i] += z[i].real();
        }
    for (int a = 0; a < 2; ++a) {
        double nb = 0, su = 0, sq = 0;
        for (long i = 0; i < n3; ++i) {
            const double v3 = v[i % N], c2 = v[i / (N * N)] * v[i / (N * N)] + v[i / N % N] * v[i / N % N] + v3 * v3;
            nb += o.nu_h[a * n3 + i] * feq[a * n3 + i] * dv3;
            su += v3 * v3 * feq[a * n3 + i] * dv3;
            sq += (o.r[a] * c2 - 2.5) * v3 * v3 * feq[a * n3 + i] * dv3;
        }
        o.Nal[a] = nb / o.chi[a];
        o.cU[a] = 2.0 * o.r[a] * su / o.chi[a];
        o.cq[a] = 2.0 * o.r[a] * sq;
    }
    // separable pass tables: columns (DFT index -> basis), rows (DFT index -> representative)
    // layout 1 folds v2 (even) and v3 (odd), layout 2 only v3 (odd)
    const bool fold2 = o.layout == 1, fold3 = o.layout >= 1;
    const int co[3] = {N, fold2 ? H : N, fold3 ? H : N};
    std::vector<std::vector<double2>> colC(3), rowC(3);
    for (int ax = 0; ax < 3; ++ax) {
        colC[ax].resize((size_t)co[ax] * N);
        rowC[ax].resize((size_t)co[ax] * N);
        for (int j = 0; j < co[ax]; ++j)
            for (int a = 0; a < N; ++a) {
                std::complex<double> z = std::polar(1.0, -2.0 * M_PI * ((long)a * j % N) / N);
                if ((ax == 1 && fold2) || (ax == 2 && fold3)) {
                    const std::complex<double> zr = std::polar(1.0, -2.0 * M_PI * ((long)a * (N - 1 - j) % N) / N);
                    z = ax == 1 ? z + zr : z - zr;  // even in v2, odd in v3
                }
                z /= (double)N;
                colC[ax][(size_t)j * N + a] = make_double2(z.real(), z.imag());
                const std::complex<double> y = std::polar(1.0, 2.0 * M_PI * ((long)a * j % N) / N);
                rowC[ax][(size_t)j * N + a] = make_double2(y.real(), y.imag());
            }
    }
    const long nr = (long)co[0] * co[1] * co[2];
    o.nr = (int)nr;
    // device buffers
    lbe_status st = LBE_OK;
    auto take = [&](void** p, size_t bytes) {
        if (st == LBE_OK) st = dev_alloc(c, p, bytes);
    };
    void *d_s = nullptr, *d_ps = nullptr, *d_keep = nullptr, *d_fh = nullptr, *d_G = nullptr, *d_wp = nullptr;
    void *d_B0 = nullptr, *d_B1 = nullptr, *d_K = nullptr, *d_Y = nullptr, *d_C = nullptr, *d_T = nullptr;
    const size_t nn = (size_t)n3 * n3;
    take(&d_s, sizeof(double) * M * n3);
    take(&d_ps, sizeof(double) * M * n3);
    take(&d_keep, n3);
    take(&d_fh, sizeof(double2) * 2 * n3);
    take(&d_G, sizeof(double) * 4 * n3);
    take(&d_wp, sizeof(double) * 4 * M);
    take(&d_C, sizeof(double2) * 6 * N * N);
    take(&d_T, sizeof(double2) * 2 * M * n3);
    take(&d_B0, sizeof(double) * nn);
    take(&d_B1, sizeof(double) * nn);
    take(&d_K, sizeof(double2) * nn);
    take(&d_Y, sizeof(double2) * nn);
    take((void**)&o.L, sizeof(double) * 4 * (size_t)nr * nr);
    take((void**)&o.nu, sizeof(double) * 2 * n3);
    take((void**)&o.feq, sizeof(double) * 2 * n3);
    take((void**)&o.vel, sizeof(double) * N);
    if (st == LBE_OK) {
        std::vector<double2> fh2(2 * n3);
        for (int a = 0; a < 2; ++a)
            for (long m = 0; m < n3; ++m) fh2[a * n3 + m] = make_double2(fh[a][m].real(), fh[a][m].imag());
        std::vector<double> wpv(4 * M);
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b)
                for (int p = 0; p < M; ++p) wpv[(2 * a + b) * M + p] = 2.0 * bab(a, b) * w[p];
        std::vector<double2> Ct;
        for (int ax = 0; ax < 3; ++ax) Ct.insert(Ct.end(), colC[ax].begin(), colC[ax].end());
        for (int ax = 0; ax < 3; ++ax) Ct.insert(Ct.end(), rowC[ax].begin(), rowC[ax].end());
        cudaMemcpyAsync(d_s, sp.data(), sizeof(double) * M * n3, cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(d_ps, ps.data(), sizeof(double) * M * n3, cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(d_keep, keep.data(), n3, cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(d_fh, fh2.data(), sizeof(double2) * 2 * n3, cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(d_G, G.data(), sizeof(double) * 4 * n3, cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(d_wp, wpv.data(), sizeof(double) * 4 * M, cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(d_C, Ct.data(), sizeof(double2) * Ct.size(), cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(o.nu, o.nu_h.data(), sizeof(double) * 2 * n3, cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(o.feq, feq.data(), sizeof(double) * 2 * n3, cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(o.vel, v.data(), sizeof(double) * N, cudaMemcpyHostToDevice, s);
        g_h2d += sizeof(double) * (2 * M * n3 + 8 * n3 + 4 * M + N) + n3;
        const double2* fhd = (const double2*)d_fh;
        const double2* Cd = (const double2*)d_C;
        // column and row tables of axis ax start at Cd + off_c[ax] / off_r[ax]
        long off_c[3], off_r[3], acc = 0;
        for (int ax = 0; ax < 3; ++ax) off_c[ax] = acc, acc += (long)co[ax] * N;
        for (int ax = 0; ax < 3; ++ax) off_r[ax] = acc, acc += (long)co[ax] * N;
        const int gb = grid_for((long)nn);
        for (int a = 0; a < 2 && st == LBE_OK; ++a) {
            for (int b = 0; b < 2; ++b) {
                const double mub = o.r[b] / (o.r[a] + o.r[b]), cc = (o.r[b] - o.r[a]) / (o.r[a] + o.r[b]);
                double2* TL = (double2*)d_T;
                double2* TM = TL + (long)M * n3;
                k_mix_trig<<<grid_for((long)M * n3), 256, 0, s>>>(TL, (const double*)d_s, (long)M * n3, o.R * mub);
                k_mix_trig<<<grid_for((long)M * n3), 256, 0, s>>>(TM, (const double*)d_s, (long)M * n3,
                                                                  0.5 * o.R * cc);
                k_mix_beta<<<gb, 256, 0, s>>>((double*)(b ? d_B1 : d_B0), (const double*)d_s, TL, TM,
                                              (const double*)d_ps, (const unsigned char*)d_keep,
                                              (const double*)d_wp + (2 * a + b) * M, M, n3, 2.0 * mub, cc, o.R);
                g_launches += 2;
            }
            for (int b = 0; b < 2; ++b) {
                k_mix_fourier<<<gb, 256, 0, s>>>((double2*)d_K, (const double*)(b ? d_B1 : d_B0),
                                                 (const double*)d_B0, (const double*)d_B1, fhd + a * n3, fhd,
                                                 fhd + n3, (const double*)d_G + (2 * a + b) * n3, N, a == b);
                // columns: m3, m2, m1 -> basis
                double2 *X = (double2*)d_K, *Y = (double2*)d_Y;
                long inner = 1;
                long outer = n3 * N * N;
                for (int ax = 2; ax >= 0; --ax) {
                    k_axis_pass<<<grid_for(outer * co[ax] * inner), 256, 0, s>>>(X, Y, Cd + off_c[ax], outer, N, inner,
                                                                                   co[ax]);
                    std::swap(X, Y);
                    inner *= co[ax];
                    outer /= N;
                }
                // rows: k3, k2, k1 -> representatives (X now holds [k][nr])
                inner = nr;
                outer = (long)N * N;
                for (int ax = 2; ax >= 0; --ax) {
                    k_axis_pass<<<grid_for(outer * co[ax] * inner), 256, 0, s>>>(X, Y, Cd + off_r[ax], outer, N, inner,
                                                                                   co[ax]);
                    std::swap(X, Y);
                    inner *= co[ax];
                    outer /= N;
                }
                k_mix_store<<<grid_for(nr * nr), 256, 0, s>>>(o.L, X, nr, 2 * nr, a * nr, b * nr);
                g_launches += 9;
            }
            g_launches += 2;
        }
        st = cuda_status(c, cudaStreamSynchronize(s), "mixture operator build");
    }
    for (void* p : {d_B0, d_B1, d_K, d_Y})
        if (p) dev_free(c, p, p == d_B0 || p == d_B1 ? sizeof(double) * nn : sizeof(double2) * nn);
    if (d_s) dev_free(c, d_s, sizeof(double) * M * n3);
    if (d_ps) dev_free(c, d_ps, sizeof(double) * M * n3);
    if (d_keep) dev_free(c, d_keep, n3);
    if (d_fh) dev_free(c, d_fh, sizeof(double2) * 2 * n3);
    if (d_G) dev_free(c, d_G, sizeof(double) * 4 * n3);
    if (d_wp) dev_free(c, d_wp, sizeof(double) * 4 * M);
    if (d_C) dev_free(c, d_C, sizeof(double2) * 6 * N * N);
    if (d_T) dev_free(c, d_T, sizeof(double2) * 2 * M * n3);
    if (st != LBE_OK) return st;
    if ((st = dev_alloc(c, (void**)&o.zero, sizeof(double) * n3)) != LBE_OK) return st;
    cudaMemsetAsync(o.zero, 0, sizeof(double) * n3, s);
    if ((st = dev_alloc(c, (void**)&o.ftab, sizeof(float) * (5 * n3 + N))) != LBE_OK) return st;
    {
        std::vector<float> ft(5 * n3 + N, 0.f);
        for (long i = 0; i < 2 * n3; ++i) ft[i] = (float)feq[i];
        for (long i = 0; i < 2 * n3; ++i) ft[2 * n3 + i] = (float)o.nu_h[i];
        for (int j = 0; j < N; ++j) ft[5 * n3 + j] = (float)v[j];
        cudaMemcpy(o.ftab, ft.data(), sizeof(float) * ft.size(), cudaMemcpyHostToDevice);
        g_h2d += sizeof(float) * ft.size();
    }
    for (int a = 0; a < 2; ++a) {
        DevTables& t = o.tab[a];
        t.nv = N;
        t.vmax = o.vmax;
        t.R = o.R;
        t.dv = dv;
        t.M = M;
        t.vel_d = o.vel;
        t.feq_d = o.feq + a * n3;
        t.nu1_d = o.nu + a * n3;
        t.feq_f = o.ftab + a * n3;
        t.nu1_f = o.ftab + 2 * n3 + a * n3;
        t.vel_f = o.ftab + 5 * n3;
        o.tab0[a] = t;
        o.tab0[a].feq_d = o.zero;
        o.tab0[a].feq_f = o.ftab + 4 * n3;
    }
    return cuda_status(c, cudaStreamSynchronize(s), "mixture tables");
}

MixOp* get_mixop(Ctx* c, const lbe_mixture& m, int nv, double vmax, int M, double R, int layout, cudaStream_t s,
                 lbe_status* st) {
    const std::string key = mix_key(m, nv, vmax, M, R, layout);
    std::lock_guard<std::mutex> lk(c->tables_mu);
    auto it = c->mix_ops.find(key);
    if (it != c->mix_ops.end()) return it->second;
    MixOp* o = new MixOp();
    o->nv = nv;
    o->M = M;
    o->layout = layout;
    o->vmax = vmax;
    o->R = R;
    o->r[1] = m.mass_ratio;
    o->d[1] = m.diam_ratio;
    o->chi[0] = m.chi_A;
    o->chi[1] = 1.0 - m.chi_A;
    o->mbar = o->chi[0] + o->chi[1] * o->r[1];
    o->mu1 = viscosity1(o->r[1], o->d[1], o->chi[0]);
    o->b0 = o->mu1 * std::sqrt(2.0 / o->mbar) / 4.0;
    *st = build_mixop(c, *o, s);
    if (*st != LBE_OK) {
        free_mixop(c, o);
        return nullptr;
    }
    c->mix_ops[key] = o;
    return o;
}

// K split: the smallest count S (slices of at least 256 k) whose S x tiles spreads over the SMs
// within 3 % of even, else the one that comes closest.
int mix_split(long tiles, int K) {
    const int P = sm_count(), smax = std::max(1, K / 256);
    int best = 1;
    double best_eff = 0.0;
    for (int S = 1; S <= smax; ++S) {
        const long n = tiles * S;
        const double eff = (double)n / (double)(((n + P - 1) / P) * P);
        if (eff > best_eff + 1e-9) best = S, best_eff = eff;
        if (eff >= 0.97) break;
    }
    return best;
}

lbe_status mix_gemm(Ctx* c, MixOp& o, const double* hA, const double* hB, long cs, int cells, double scale,
                    double* yA, double* yB, cudaStream_t s, bool df = false, const int* map = nullptr) {
    if (df && !o.Ldf) {
        const long nn = 4L * o.nr * o.nr;
        lbe_status st = dev_alloc(c, (void**)&o.Ldf, sizeof(float2) * nn);
        if (st != LBE_OK) return st;
        k_mix_to_df<<<grid_for(nn), 256, 0, s>>>(o.L, nn, o.Ldf);
        g_launches += 1;
    }
    const int K = 2 * o.nr;
    dim3 g((2 * o.nr + kMT - 1) / kMT, (cells + kNT - 1) / kNT);
    int S = mix_split((long)g.x * g.y, K);
    int kc = (K + S - 1) / S;
    kc = (kc + kKT - 1) / kKT * kKT;
    S = (K + kc - 1) / kc;
    g.z = S;
    const size_t need = S > 1 ? sizeof(double) * (size_t)S * cells * K : 0;
    if (need > o.part_bytes) {
        if (o.part) cudaStreamSynchronize(s), dev_free(c, o.part, o.part_bytes), o.part = nullptr, o.part_bytes = 0;
        lbe_status st = dev_alloc(c, (void**)&o.part, need);
        if (st != LBE_OK) return st;
        o.part_bytes = need;
    }
    // with kernel timing on, each launch is bracketed by events and waited for (lbe_get_stats)
    cudaEvent_t ev[2];
    const bool timed = g_time_kernels.load() != 0 && cudaEventCreate(&ev[0]) == cudaSuccess &&
                       cudaEventCreate(&ev[1]) == cudaSuccess;
    if (timed) cudaEventRecord(ev[0], s);
    if (df) {
        const size_t xb = sizeof(float2) * (size_t)K * cells;
        if (xb > o.xdf_bytes) {
            if (o.Xdf) cudaStreamSynchronize(s), dev_free(c, o.Xdf, o.xdf_bytes), o.Xdf = nullptr, o.xdf_bytes = 0;
            lbe_status st = dev_alloc(c, (void**)&o.Xdf, xb);
            if (st != LBE_OK) return st;
            o.xdf_bytes = xb;
        }
        k_mix_h_to_df<<<grid_for((long)K * cells), 256, 0, s>>>(hA, hB, cs, o.nr, cells, o.Xdf, map);
        k_mix_gemm_df<<<g, 256, 0, s>>>(o.Ldf, o.nr, o.Xdf, cs, cells, scale, yA, yB, kc, S > 1 ? o.part : nullptr,
                                        map);
        g_launches += 1;
    }
    else
        k_mix_gemm<<<g, 256, 0, s>>>(o.L, o.nr, hA, hB, cs, cells, scale, yA, yB, kc, S > 1 ? o.part : nullptr, map);
    g_launches += 1;
    if (S > 1) {
        k_mix_reduce<<<grid_for((long)K * cells), 256, 0, s>>>(o.part, S, o.nr, cells, cs, scale, yA, yB, map);
        g_launches += 1;
    }
    if (timed) {
        cudaEventRecord(ev[1], s);
        cudaEventSynchronize(ev[1]);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev[0], ev[1]);
        add_gemm_time(ms);
        cudaEventDestroy(ev[0]);
        cudaEventDestroy(ev[1]);
    }
    return LBE_OK;
}

cudaStream_t use_stream(Ctx* c, void* stream) { return stream ? (cudaStream_t)stream : c->stream; }

}  // namespace

void mix_release(Ctx* c) {
    for (auto& kv : c->mix_ops) free_mixop(c, kv.second);
    c->mix_ops.clear();
}

}  // namespace lbe

using namespace lbe;

extern "C" lbe_status lbe_mix_info(lbe_ctx* ctx, const lbe_mixture* mix, int nv, double vmax, int M, double R,
                                   double* out4, double* nu_out) {
    if (!ctx || !out4) return bad_arg(ctx, "null argument");
    lbe_status st = check_mixture(ctx, mix, nv, vmax, M, R);
    if (st != LBE_OK) return st;
    cudaSetDevice(ctx->device);
    MixOp* o = get_mixop(ctx, *mix, nv, vmax, M, R, 1, ctx->stream, &st);
    if (!o) return st;
    out4[0] = o->b0;
    out4[1] = o->Nal[0];
    out4[2] = o->Nal[1];
    out4[3] = o->mu1;
    if (nu_out) std::memcpy(nu_out, o->nu_h.data(), sizeof(double) * o->nu_h.size());
    return LBE_OK;
}

extern "C" lbe_status lbe_mix_apply_L(lbe_ctx* ctx, const lbe_mixture* mix, int nv, double vmax, int M, double R,
                                      int cells, double delta, const double* hA, const double* hB, double* LplusA,
                                      double* LA, double* LplusB, double* LB, void* stream) {
    if (!ctx || !hA || !hB || !LplusA || !LplusB) return bad_arg(ctx, "null argument");
    lbe_status st = check_mixture(ctx, mix, nv, vmax, M, R);
    if (st != LBE_OK) return st;
    if (cells < 0 || !(delta >= 0)) return bad_arg(ctx, "cells >= 0 and delta >= 0");
    if (cells == 0) return LBE_OK;
    cudaSetDevice(ctx->device);
    cudaStream_t s = use_stream(ctx, stream);
    MixOp* o = get_mixop(ctx, *mix, nv, vmax, M, R, 0, s, &st);
    if (!o) return st;
    const long n3 = (long)nv * nv * nv;
    if ((st = mix_gemm(ctx, *o, hA, hB, n3, cells, delta, LplusA, LplusB, s)) != LBE_OK) return st;
    const long total = (long)cells * n3;
    if (LA) k_mix_loss<<<grid_for(total), 256, 0, s>>>(LplusA, hA, o->nu, delta, n3, total, LA), g_launches += 1;
    if (LB) k_mix_loss<<<grid_for(total), 256, 0, s>>>(LplusB, hB, o->nu + n3, delta, n3, total, LB), g_launches += 1;
    g_levals += cells;
    return cuda_status(ctx, cudaGetLastError(), "mixture apply");
}

extern "C" lbe_status lbe_mix_solve(lbe_ctx* ctx, const lbe_mix_problem* pb, lbe_mix_result* out, double* U_out,
                                    double* h_out) {
    if (!ctx || !pb || !out) return bad_arg(ctx, "null argument");
    lbe_status st = check_mixture(ctx, &pb->mix, pb->nv, pb->vmax, pb->M, pb->R);
    if (st != LBE_OK) return st;
    const lbe_geometry& gm = pb->geom;
    if (gm.dim == 1 ? (gm.ns < 2 || gm.ns > 1000 || (gm.grid_kind != 0 && gm.grid_kind != 1))
                    : (gm.dim != 2 || gm.nx < 3 || gm.ny < 3 || gm.nx > 256 || gm.ny > 256 || !(gm.width > 0)))
        return bad_arg(ctx, "mixture geometry: plates 2 <= ns <= 1000, grid_kind 0 or 1; ducts 3 <= nx, ny <= 256, "
                            "width > 0");
    if (!(pb->delta >= 0) || pb->max_iter < 1 || !(pb->eps >= 0) || (pb->scheme != LBE_CIS && pb->scheme != LBE_SIS))
        return bad_arg(ctx, "mixture: delta >= 0, max_iter >= 1, eps >= 0, scheme CIS or SIS");
    if (pb->precision != LBE_FP64 && pb->precision != LBE_DF32 && pb->precision != LBE_BF16 &&
        pb->precision != LBE_BF16_REFINED)
        return bad_arg(ctx, "mixture: precision FP64, DF32, BF16 or BF16_REFINED");
    const bool porous = pb->solid_fraction > 0;
    if (porous && (gm.dim != 2 || gm.nx != gm.ny || gm.nx < 4 || !(pb->solid_fraction < 0.78)))
        return bad_arg(ctx, "mixture porous cell: ducts geometry with nx = ny >= 4 and 0 < solid_fraction < 0.78");
    if (!(pb->solid_fraction >= 0)) return bad_arg(ctx, "mixture: solid_fraction >= 0");
    cudaSetDevice(ctx->device);
    cudaStream_t s = ctx->stream;
    const int dim = gm.dim, layout = dim == 1 ? 1 : 2;
    MixOp* o = get_mixop(ctx, pb->mix, pb->nv, pb->vmax, pb->M, pb->R, layout, s, &st);
    if (!o) return st;
    // operator on the tensor cores (BF16 hi / lo); the FP64-class GEMM in double-float
    bool lo = pb->precision == LBE_BF16 || pb->precision == LBE_BF16_REFINED;
    const bool dfg = pb->precision == LBE_DF32 || pb->precision == LBE_BF16_REFINED;
    if (lo && !o->tc && (st = mix_tc_build(ctx, o->L, 2 * o->nr, &o->tc, s)) != LBE_OK) return st;
    lbe_problem geo{};
    geo.geom = gm;
    SweepGeom g;
    build_sweep_geom(g, geo);
    const int n = g.cells, N = pb->nv;
    const long n3 = (long)N * N * N, per = (long)n * n3;
    std::vector<double> coef, geov;
    if (dim == 1) {
        for (auto* vv : {&g.fa, &g.fb, &g.fc, &g.ba, &g.bb, &g.bc}) coef.insert(coef.end(), vv->begin(), vv->end());
        std::vector<double> ia(g.fa.size());
        for (size_t i = 0; i < ia.size(); ++i) ia[i] = g.fa[i] != 0.0 ? 1.0 / g.fa[i] : 0.0;
        for (auto* vv : {&g.x, &ia, &g.fb, &g.fc, &g.trap}) geov.insert(geov.end(), vv->begin(), vv->end());
    } else {
        for (auto* vv : {&g.xa, &g.xb, &g.xc, &g.ya, &g.yb, &g.yc}) coef.insert(coef.end(), vv->begin(), vv->end());
        // DST-I of the interior (orthonormal, symmetric) and the Laplacian's eigenvalues
        const int mx = gm.nx - 2, my = gm.ny - 2;
        const double dx = gm.width / gm.nx, dy = 1.0 / gm.ny;
        geov.resize((size_t)mx * mx + (size_t)my * my + (size_t)mx * my);
        for (int i = 0; i < mx; ++i)
            for (int k = 0; k < mx; ++k)
                geov[(size_t)i * mx + k] = std::sqrt(2.0 / (mx + 1)) * std::sin(M_PI * (i + 1) * (k + 1) / (mx + 1));
        double* sy = geov.data() + (size_t)mx * mx;
        for (int i = 0; i < my; ++i)
            for (int k = 0; k < my; ++k)
                sy[(size_t)i * my + k] = std::sqrt(2.0 / (my + 1)) * std::sin(M_PI * (i + 1) * (k + 1) / (my + 1));
        double* lm = sy + (size_t)my * my;
        for (int p = 0; p < mx; ++p)
            for (int q = 0; q < my; ++q) {
                const double sp = std::sin(M_PI * (p + 1) / (2.0 * (mx + 1)));
                const double sq = std::sin(M_PI * (q + 1) / (2.0 * (my + 1)));
                lm[(size_t)p * my + q] = -4.0 * sp * sp / (dx * dx) - 4.0 * sq * sq / (dy * dy);
            }
    }
    // the periodic unit cell: solid cells, interior cells of the correction and their neighbours
    PorousDev PG{};
    std::vector<unsigned char> solid;
    std::vector<int> inner, nbl, fluid;
    if (porous) {
        const int nn = gm.nx;
        const double d = 1.0 / nn, R2 = pb->solid_fraction / M_PI;
        solid.assign((size_t)nn * nn, 0);
        for (int i = 0; i < nn; ++i)
            for (int j = 0; j < nn; ++j) {
                const double x = (i + 0.5) * d - 0.5, y = (j + 0.5) * d - 0.5;
                solid[(size_t)i * nn + j] = x * x + y * y < R2;
            }
        auto fl = [&](int i, int j) { return !solid[(size_t)((i + nn) % nn) * nn + (j + nn) % nn]; };
        // the operator's columns: fluid cells only (h and L h stay zero in solid cells)
        for (int c = 0; c < nn * nn; ++c)
            if (!solid[c]) fluid.push_back(c);
        std::vector<int> kof((size_t)nn * nn, -1);
        for (int i = 0; i < nn; ++i)
            for (int j = 0; j < nn; ++j) {
                bool in = fl(i, j);
                for (int di = -1; di <= 1; ++di)
                    for (int dj = -1; dj <= 1; ++dj) in = in && fl(i + di, j + dj);
                if (in) kof[(size_t)i * nn + j] = (int)inner.size(), inner.push_back(i * nn + j);
            }
        for (int c : inner) {
            const int i = c / nn, j = c % nn;
            const int di[4] = {1, -1, 0, 0}, dj[4] = {0, 0, 1, -1};
            for (int e = 0; e < 4; ++e) {
                const int cc = ((i + di[e] + nn) % nn) * nn + (j + dj[e] + nn) % nn;
                nbl.push_back(kof[cc] >= 0 ? kof[cc] : -1 - cc);
            }
        }
        // three-point backward differences (Lagrange) on nodes x0 - h1 - h2, x0 - h1, x0
        auto bw = [](double h1, double h2, double* a, double* b, double* c) {
            *a = (2.0 * h1 + h2) / (h1 * (h1 + h2));
            *b = -(h1 + h2) / (h1 * h2);
            *c = h1 / (h2 * (h1 + h2));
        };
        double cdum;
        PG.n = nn;
        bw(d, d, &PG.ua, &PG.ub, &PG.uc);
        PG.w1a = 2.0 / d;
        bw(d, 0.5 * d, &PG.w2a, &PG.w2b, &cdum);
    }
    MixSisDev P{};
    for (int a = 0; a < 2; ++a) {
        P.r[a] = o->r[a];
        P.chi[a] = o->chi[a];
        const double Nin = a ? pb->N_B : pb->N_A;
        P.Nd[a] = (Nin > 0 ? Nin : o->Nal[a]) * pb->delta;
        P.cU[a] = o->cU[a];
        P.cq[a] = o->cq[a];
    }
    P.delta = pb->delta;
    P.dv3 = std::pow(2.0 * pb->vmax / N, 3);
    P.sqm = std::sqrt(o->mbar);
    P.nv = N;
    P.cells = n;
    P.sis = pb->scheme == LBE_SIS;
    P.layout = layout;
    MixDuctDev D{gm.nx, gm.ny, dim == 2 ? gm.width / gm.nx : 0.0, dim == 2 ? 1.0 / gm.ny : 0.0};
    const int nq = N * (layout == 1 ? N / 2 : N) * (N / 2);
    SweepJobDev job{};
    job.cell_off = 0;
    job.ncell = n;
    job.nx = dim == 2 ? gm.nx : 0;
    job.ny = dim == 2 ? gm.ny : 0;
    job.coef_off = 0;
    job.forcing = LBE_POISEUILLE;
    job.delta = pb->delta;
    // device workspace
    const size_t b_state = sizeof(double) * 2 * per;
    const size_t n_work = porous ? 10 * inner.size() + 2 : (dim == 2 ? 4 * (size_t)(gm.nx - 2) * (gm.ny - 2) : 0);
    const size_t b_small = sizeof(double) * (2 * kMom * n + 4 * n + 8 + n_work) +
                           sizeof(double) * (coef.size() + geov.size());
    void *d_h = nullptr, *d_hh = nullptr, *d_lp = nullptr, *d_small = nullptr, *d_job = nullptr;
    auto take = [&](void** p, size_t bytes) {
        if (st == LBE_OK) st = dev_alloc(ctx, p, bytes);
    };
    const bool refined = pb->precision == LBE_BF16_REFINED;
    void *d_hp = nullptr, *d_e = nullptr, *d_x = nullptr, *d_d = nullptr, *d_lp32 = nullptr, *d_hh32 = nullptr;
    if (lo) {
        take(&d_lp32, b_state / 2);
        take(&d_hh32, b_state / 2);
    }
    take(&d_h, b_state);
    take(&d_hh, b_state);
    take(&d_lp, b_state);
    void *d_gs = nullptr, *d_dg = nullptr;  // porous: the lag state before the FP64 step, its change
    if (refined) {
        take(&d_hp, b_state);
        take(&d_e, b_state);
        take(&d_x, b_state);
        take(&d_d, b_state);
        if (porous) {
            take(&d_gs, b_state);
            take(&d_dg, b_state);
        }
    }
    take(&d_small, b_small);
    take(&d_job, sizeof job);
    void* d_por = nullptr;
    const size_t b_por = porous ? solid.size() + sizeof(int) * (inner.size() + nbl.size() + fluid.size() + 2) + 64 : 0;
    if (porous) take(&d_por, b_por);
    unsigned char* dsolid = (unsigned char*)d_por;
    int* dinner = porous ? (int*)(((uintptr_t)d_por + solid.size() + 15) / 16 * 16) : nullptr;
    int* dnb = porous ? dinner + inner.size() : nullptr;
    int* dfluid = porous ? dnb + nbl.size() : nullptr;
    int* dcg = porous ? dfluid + fluid.size() : nullptr;
    // operator columns: all cells, or the porous cell's fluid cells through the list dfluid
    const int ncol = porous ? (int)fluid.size() : n;
    double* h = (double*)d_h;
    double* hh = (double*)d_hh;
    double* lp = (double*)d_lp;
    double* mom = (double*)d_small;           // [2][n][kMom]
    double* dU = mom + 2 * kMom * n;          // [2][n]
    double* Uc = dU + 2 * n;                  // [2][n]
    double* rates = Uc + 2 * n;               // [8]
    double* dwork = rates + 8;                // ducts: [2][2][mx my]
    double* dcoef = dwork + n_work;
    double* dgeo = dcoef + coef.size();       // plates: x, fa, fb, fc, trap; ducts: Sx, Sy, lam
    const double* dSx = dgeo;
    const double* dSy = dim == 2 ? dgeo + (size_t)(gm.nx - 2) * (gm.nx - 2) : nullptr;
    const double* dlam = dim == 2 ? dSy + (size_t)(gm.ny - 2) * (gm.ny - 2) : nullptr;
    double hr[4] = {0, 0, 0, 0}, old[4] = {0, 0, 0, 0};
    int it = 0, it64 = 0;
    bool conv = false, bad = false;
    static std::once_flag march_attr;  // the march stages up to 23 x 1001 doubles
    std::call_once(march_attr, [] {
        cudaFuncSetAttribute(k_mix_march, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)((2 * kMom + 5) * kMarchMax * sizeof(double)));
    });
    const size_t march_smem = (2 * kMom + 5) * (size_t)n * sizeof(double);
    // one iteration hin -> hout (hout may be hin) with the operator in FP64 or on the tensor
    // cores; homog: the source-free iteration (no S_a in the sweep, no x1 in the march); r
    // receives the flow rates of hout
    auto step = [&](const double* hin, double* hout, bool tc, bool homog, double* r) -> lbe_status {
        MixSisDev Q = P;
        Q.src = homog ? 0 : 1;
        lbe_status e;
        if (tc) {
            // low precision: the tensor-core operator read back as float, float sweeps, FP64 state
            float* lp32 = (float*)d_lp32;
            float* hh32 = (float*)d_hh32;
            e = mix_tc_apply(ctx, o->tc, ncol, hin, hin + per, n3, o->nr, pb->delta, lp32, lp32 + per, true, s,
                             dfluid);
            if (e != LBE_OK) return e;
            if (porous)
                launch_sweep_porous<float>(lp32, hh32, per, homog ? o->tab0 : o->tab, true, dsolid, PG, N,
                                           pb->delta, s);
            else
                for (int a = 0; a < 2; ++a) {
                    const DevTables& tb = homog ? o->tab0[a] : o->tab[a];
                    launch_sweep<float>(tb, dim, 1, (int)coef.size(), lp32 + a * per, hh32 + a * per,
                                        (const SweepJobDev*)d_job, nullptr, dcoef, s, 1);
                }
            k_mix_moments<float><<<dim3(n, 2), 256, 0, s>>>(Q, hh32, hin, lp32, o->nu, o->vel, mom);
            if (porous)  // the low-precision iteration's floor is far above 1e-9
                k_mix_poisson_porous<<<2, 1024, 0, s>>>(Q, PG, mom, dinner, dnb, (int)inner.size(), dwork, dU, Uc,
                                                        rates, dcg, 1e-9);
            else if (dim == 1)
                k_mix_march<<<1, 256, march_smem, s>>>(Q, mom, dgeo, dU, Uc, rates);
            else
                k_mix_poisson2d<<<2, 512, 0, s>>>(Q, D, mom, dSx, dSy, dlam, dwork, dU, Uc, rates);
            launch_correct<float>(Q, hh32, hout, dU, o->feq, o->vel, nq, s);
        } else {
            e = mix_gemm(ctx, *o, hin, hin + per, n3, ncol, pb->delta, lp, lp + per, s, dfg, dfluid);
            if (e != LBE_OK) return e;
            if (porous)
                launch_sweep_porous<double>(lp, hh, per, homog ? o->tab0 : o->tab, false, dsolid, PG, N,
                                            pb->delta, s);
            else
                for (int a = 0; a < 2; ++a) {
                    const DevTables& tb = homog ? o->tab0[a] : o->tab[a];
                    launch_sweep<double>(tb, dim, 1, (int)coef.size(), lp + a * per, hh + a * per,
                                         (const SweepJobDev*)d_job, nullptr, dcoef, s, 1);
                }
            k_mix_moments<double><<<dim3(n, 2), 256, 0, s>>>(Q, hh, hin, lp, o->nu, o->vel, mom);
            if (porous)
                k_mix_poisson_porous<<<2, 1024, 0, s>>>(Q, PG, mom, dinner, dnb, (int)inner.size(), dwork, dU, Uc,
                                                        rates, dcg, 1e-13);
            else if (dim == 1)
                k_mix_march<<<1, 256, march_smem, s>>>(Q, mom, dgeo, dU, Uc, rates);
            else
                k_mix_poisson2d<<<2, 512, 0, s>>>(Q, D, mom, dSx, dSy, dlam, dwork, dU, Uc, rates);
            launch_correct<double>(Q, hh, hout, dU, o->feq, o->vel, nq, s);
        }
        g_launches += 3;
        g_levals += n;
        cudaMemcpyAsync(r, rates, 4 * sizeof(double), cudaMemcpyDeviceToHost, s);
        g_d2h += 4 * sizeof(double);
        if ((e = cuda_status(ctx, cudaStreamSynchronize(s), "mixture iteration")) != LBE_OK) return e;
        if (tc && (e = mix_tc_check(ctx, o->tc)) != LBE_OK) return e;
        ++it;
        if (!tc) ++it64;
        for (int k = 0; k < 4; ++k)
            if (!std::isfinite(r[k])) bad = true;
        return LBE_OK;
    };
    auto axpy = [&](const double* x, double sc, const double* y, double* z) {
        k_mix_axpy<<<grid_for(2 * per), 256, 0, s>>>(x, sc, y, 2 * per, z);
        g_launches += 1;
    };
    if (st == LBE_OK) {
        cudaMemsetAsync(h, 0, b_state, s);
        cudaMemsetAsync(hh, 0, b_state, s);  // the porous sweep's periodic inflow starts from zero
        cudaMemsetAsync(lp, 0, b_state, s);  // L h in solid cells, which the operator skips
        for (void* q : {d_hp, d_e, d_x, d_d})
            if (q) cudaMemsetAsync(q, 0, b_state, s);
        for (void* q : {d_lp32, d_hh32})
            if (q) cudaMemsetAsync(q, 0, b_state / 2, s);
        if (porous) {
            cudaMemcpyAsync(dsolid, solid.data(), solid.size(), cudaMemcpyHostToDevice, s);
            cudaMemcpyAsync(dinner, inner.data(), sizeof(int) * inner.size(), cudaMemcpyHostToDevice, s);
            cudaMemcpyAsync(dnb, nbl.data(), sizeof(int) * nbl.size(), cudaMemcpyHostToDevice, s);
            cudaMemcpyAsync(dfluid, fluid.data(), sizeof(int) * fluid.size(), cudaMemcpyHostToDevice, s);
            g_h2d += solid.size() + sizeof(int) * (inner.size() + nbl.size() + fluid.size());
        }
        cudaMemcpyAsync(dcoef, coef.data(), sizeof(double) * coef.size(), cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(dgeo, geov.data(), sizeof(double) * geov.size(), cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(d_job, &job, sizeof job, cudaMemcpyHostToDevice, s);
        g_h2d += sizeof(double) * (coef.size() + geov.size()) + sizeof job;
        // plain iterations: FP64 and BF16 to their stopping tests, BF16_REFINED to the
        // low-precision floor.  FP64: every flow rate changes by < eps relative.  Tensor-core
        // iterations (float accumulation) cannot resolve a small flow rate below the larger
        // one's rounding, so their changes are measured against the larger molecular flow rate.
        int rising = 0;
        double prev = 1e300;
        while (it < pb->max_iter) {
            if ((st = step(h, h, lo, false, hr)) != LBE_OK || bad) break;
            const double scale = std::max(std::fabs(hr[0]), std::fabs(hr[1]));
            bool same = pb->eps > 0;
            double change = 0.0;
            for (int k = 0; k < 4; ++k) {
                const double dk = std::fabs(hr[k] - old[k]);
                change = std::max(change, dk);
                same = same && dk < pb->eps * (lo ? scale : std::fabs(hr[k]));
                old[k] = hr[k];
            }
            if (refined && lo) {
                // hand over at the floor: changes below 1e-5 of the scale, or no longer shrinking
                rising = change >= prev ? rising + 1 : 0;
                prev = change;
                if (change < 1e-5 * scale || rising >= 3) {
                    if (porous) {  // the FP64 lag state starts from the float half step
                        k_mix_widen<<<grid_for(2 * per), 256, 0, s>>>((const float*)d_hh32, 2 * per, hh);
                        g_launches += 1;
                    }
                    break;
                }
                continue;
            }
            if (same) {
                conv = true;
                break;
            }
        }
        // defect correction (BF16_REFINED).  The iteration is affine, Phi(h) = G h + c; from h,
        // one FP64 iteration h' = Phi(h) (its change is the stopping test), and the error of h'
        // solves e = G (e + d), d = h' - h, which the source-free iteration on the tensor cores
        // approximates (e_0 = 0, e_(j+1) = G_lo (e_j + d)); then h = h' + e, and the flow rates,
        // linear in h, are those of h' plus those of e.
        double* hp = (double*)d_hp;
        double* ev = (double*)d_e;
        double* xv = (double*)d_x;
        double* dv = (double*)d_d;
        // The porous sweep's last half step g (its periodic lag) is part of the iteration's state:
        // the map is affine on the pair (h, g), and the same correction runs on pairs, with
        // d_g = g' - g and e_g carried in the float lag buffer of the inner iterations.
        float* hh32f = (float*)d_hh32;
        double* gs = (double*)d_gs;
        double* dg = (double*)d_dg;
        while (refined && st == LBE_OK && !bad && it < pb->max_iter) {
            if (porous) cudaMemcpyAsync(gs, hh, b_state, cudaMemcpyDeviceToDevice, s);
            if ((st = step(h, hp, false, false, hr)) != LBE_OK || bad) break;
            bool same = pb->eps > 0;
            for (int k = 0; k < 4; ++k) same = same && std::fabs(hr[k] - old[k]) < pb->eps * std::fabs(hr[k]);
            if (same) {
                std::swap(h, hp);
                conv = true;
                break;
            }
            axpy(hp, -1.0, h, dv);
            cudaMemsetAsync(ev, 0, b_state, s);
            if (porous) {
                axpy(hh, -1.0, gs, dg);                       // d_g = g' - g
                cudaMemsetAsync(hh32f, 0, b_state / 2, s);    // e_g = 0
            }
            double re[4] = {0, 0, 0, 0};
            double pe = 1e300;
            int up = 0;
            for (int j = 0; j < 200 && it < pb->max_iter; ++j) {
                axpy(ev, 1.0, dv, xv);
                if (porous) {  // the sweep's lag input e_g + d_g; its output is the next e_g
                    k_mix_add_fd<<<grid_for(2 * per), 256, 0, s>>>(hh32f, dg, 2 * per);
                    g_launches += 1;
                }
                double r[4];
                if ((st = step(xv, ev, true, true, r)) != LBE_OK || bad) break;
                double change = 0.0;
                for (int k = 0; k < 4; ++k) change = std::max(change, std::fabs(r[k] - re[k])), re[k] = r[k];
                const double emag = std::max(std::fabs(re[0]), std::fabs(re[1]));
                up = change >= pe ? up + 1 : 0;
                pe = change;
                if (change <= 1e-4 * emag || up >= 3) break;
            }
            if (st != LBE_OK || bad) break;
            axpy(hp, 1.0, ev, h);
            if (porous) {  // g = g' + e_g
                k_mix_add_df<<<grid_for(2 * per), 256, 0, s>>>(hh, hh32f, 2 * per);
                g_launches += 1;
            }
            for (int k = 0; k < 4; ++k) old[k] = hr[k] + re[k];
        }
        if (refined && st == LBE_OK && !bad) {
            // U and the flow rates of the returned h
            MixSisDev Q = P;
            Q.sis = 0;
            k_mix_moments<double><<<dim3(n, 2), 256, 0, s>>>(Q, h, h, lp, o->nu, o->vel, mom);
            if (porous)
                k_mix_poisson_porous<<<2, 1024, 0, s>>>(Q, PG, mom, dinner, dnb, (int)inner.size(), dwork, dU, Uc,
                                                        rates, dcg, 1e-13);
            else if (dim == 1)
                k_mix_march<<<1, 256, march_smem, s>>>(Q, mom, dgeo, dU, Uc, rates);
            else
                k_mix_poisson2d<<<2, 512, 0, s>>>(Q, D, mom, dSx, dSy, dlam, dwork, dU, Uc, rates);
            cudaMemcpyAsync(hr, rates, 4 * sizeof(double), cudaMemcpyDeviceToHost, s);
            g_launches += 2;
            st = cuda_status(ctx, cudaStreamSynchronize(s), "mixture flow rates");
        }
    }
    if (st == LBE_OK && U_out) {
        cudaMemcpy(U_out, Uc, sizeof(double) * 2 * n, cudaMemcpyDeviceToHost);
        g_d2h += sizeof(double) * 2 * n;
    }
    if (st == LBE_OK && h_out) {
        // the orbit layout back to the full grid: odd in v3, and for plates even in v2
        const int H = N / 2, E2 = layout == 1 ? H : N;
        std::vector<double> q(2 * (size_t)n * nq);
        for (int a = 0; a < 2; ++a)
            for (int c = 0; c < n; ++c)
                cudaMemcpy(&q[((size_t)a * n + c) * nq], h + a * per + (long)c * n3, sizeof(double) * nq,
                           cudaMemcpyDeviceToHost);
        g_d2h += sizeof(double) * q.size();
        for (size_t ac = 0; ac < 2 * (size_t)n; ++ac)
            for (int i1 = 0; i1 < N; ++i1)
                for (int i2 = 0; i2 < N; ++i2)
                    for (int i3 = 0; i3 < N; ++i3) {
                        const int j2 = (layout == 2 || i2 < H) ? i2 : N - 1 - i2, j3 = i3 < H ? i3 : N - 1 - i3;
                        const double x = q[ac * nq + ((size_t)i1 * E2 + j2) * H + j3];
                        h_out[ac * n3 + ((size_t)i1 * N + i2) * N + i3] = i3 < H ? x : -x;
                    }
    }
    dev_free(ctx, d_h, b_state);
    dev_free(ctx, d_hh, b_state);
    dev_free(ctx, d_lp, b_state);
    dev_free(ctx, d_small, b_small);
    dev_free(ctx, d_job, sizeof job);
    for (void* q : {d_hp, d_e, d_x, d_d, d_gs, d_dg})
        if (q) dev_free(ctx, q, b_state);
    for (void* q : {d_lp32, d_hh32})
        if (q) dev_free(ctx, q, b_state / 2);
    if (d_por) dev_free(ctx, d_por, b_por);
    out->M_A = hr[0];
    out->M_B = hr[1];
    out->Q_A = hr[2];
    out->Q_B = hr[3];
    out->iters = it;
    out->fp64_iters = it64;
    out->N_A = P.Nd[0] / (pb->delta > 0 ? pb->delta : 1.0);
    out->N_B = P.Nd[1] / (pb->delta > 0 ? pb->delta : 1.0);
    out->status = st != LBE_OK ? st : bad ? LBE_NAN : conv ? LBE_OK : LBE_NOT_CONVERGED;
    return (lbe_status)out->status;
}

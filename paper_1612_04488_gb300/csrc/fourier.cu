// Fourier-mode convergence analysis of the CIS and the SIS (Sec. 2.3).
//
// A system periodic in x1 with one mode exp(2 pi i x1): the error of an iteration is a complex
// VDF e(v), and one iteration of the homogeneous error equation is
//   CIS (Eq. conv_iteration):        e <- L+(e) / (nu_eq + 2 pi i v1)
//   SIS (Eq. acceleratred_iteration, the U3 formula after it, Eq. guided):
//        e_half = L+(e) / (nu_eq + 2 pi i v1)
//        A1 = 2 int v1 v3 (L e + N delta e) dv      (the N-penalised split: L - L_BGK with
//                                                    L_BGK h read as -N delta h)
//        A2 = int (2 v1^2 - 1) v3 e_half dv,   U_half = int v3 e_half dv
//        U  = (-2 pi i A1 - 4 pi^2 A2) / (4 pi^2)   (the source term drops from the error map)
//        e  <- e_half + 2 (U - U_half) v3 f_eq
// The convergence factor omega is the modulus of the map's dominant eigenvalue on the errors
// of the plate and duct problems, which are odd in v3; the paper fits U3(k) = U_inf +
// C exp(-lambda k), which the power iteration reproduces: with e_{k+1} = P map(e_k) / |e_k|
// (P the projection onto functions odd in v3), the ratio |e_{k+1}| converges to omega.
// Without P, rounding seeds the even (density-type) modes, which the SIS correction does not
// act on and which then overtake the odd ones after a few dozen iterations.
//
// Layout: the real and imaginary parts of e are two "cells" of the operator's batch (L is
// real-linear), so one FP64 operator call serves both.  Reductions run per block into
// partial sums that the host adds in block order (deterministic).
#include <cmath>
#include <vector>

#include "lbe_internal.h"
#include "sweep.h"

namespace lbe {

namespace {

constexpr int kBlocks = 64, kThreads = 256;

// sum |e|^2 over both parts, per block
__global__ void k_norm2(const double* __restrict__ e, long n, double* __restrict__ part) {
    __shared__ double red[kThreads];
    double s = 0.0;
    for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < n; k += (long)gridDim.x * blockDim.x)
        s += e[k] * e[k];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// e_half = L+ e / (delta nu + 2 pi i v1), written over e; the SIS moments A1, A2, U_half
// (complex: 6 doubles per block).  lp and lo hold (re, im) of L+ e and L e.
__global__ void k_half(double* __restrict__ e, const double* __restrict__ lp, const double* __restrict__ lo,
                       const double* __restrict__ nu1, const double* __restrict__ vel, int nv, double delta,
                       double nd, double dv3, double* __restrict__ part) {
    __shared__ double red[6][kThreads];
    const long n3 = (long)nv * nv * nv;
    double a[6] = {0, 0, 0, 0, 0, 0};  // A1 re/im, A2 re/im, U_half re/im
    for (long v = blockIdx.x * (long)blockDim.x + threadIdx.x; v < n3; v += (long)gridDim.x * blockDim.x) {
        const double v1 = vel[v / (nv * nv)], v3 = vel[v % nv];
        const double er = e[v], ei = e[n3 + v];
        const double Lr = lo[v], Li = lo[n3 + v];
        const double pr = lp[v], pi = lp[n3 + v];
        // (pr + i pi) / (dr + i di)
        const double dr = delta * nu1[v], di = 2.0 * M_PI * v1;
        const double den = dr * dr + di * di;
        const double hr = (pr * dr + pi * di) / den, hi = (pi * dr - pr * di) / den;
        e[v] = hr;
        e[n3 + v] = hi;
        const double w = 2.0 * v1 * v3 * dv3;
        a[0] += w * (Lr + nd * er);
        a[1] += w * (Li + nd * ei);
        const double c2 = (2.0 * v1 * v1 - 1.0) * v3 * dv3;
        a[2] += c2 * hr;
        a[3] += c2 * hi;
        a[4] += v3 * dv3 * hr;
        a[5] += v3 * dv3 * hi;
    }
    for (int k = 0; k < 6; ++k) red[k][threadIdx.x] = a[k];
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o)
            for (int k = 0; k < 6; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int k = 0; k < 6; ++k) part[blockIdx.x * 6 + k] = red[k][0];
}

// e = (e_half + 2 dU v3 f_eq) / n0, dU complex (zero for the CIS), then projected onto the
// functions odd in v3: e(v) = (e(v) - e(R3 v)) / 2, one thread per mirror pair
__global__ void k_finish(double* __restrict__ e, const double* __restrict__ vel, const double* __restrict__ feq,
                         int nv, double dUr, double dUi, double n0) {
    const long n3 = (long)nv * nv * nv;
    const int H = nv / 2;
    for (long p = blockIdx.x * (long)blockDim.x + threadIdx.x; p < n3 / 2; p += (long)gridDim.x * blockDim.x) {
        const long row = p / H;
        const int i3 = (int)(p % H);
        const long a = row * nv + i3, b = row * nv + (nv - 1 - i3);
        const double ga = 2.0 * vel[i3] * feq[a], gb = 2.0 * vel[nv - 1 - i3] * feq[b];
        for (int part = 0; part < 2; ++part) {
            const double dU = part ? dUi : dUr;
            double* x = e + part * n3;
            const double ea = (x[a] + dU * ga) / n0, eb = (x[b] + dU * gb) / n0;
            const double o = 0.5 * (ea - eb);
            x[a] = o;
            x[b] = -o;
        }
    }
}

double host_sum(const std::vector<double>& p, int stride, int k) {
    double s = 0.0;
    for (size_t b = 0; b * stride + k < p.size(); ++b) s += p[b * stride + k];
    return s;
}

}  // namespace

}  // namespace lbe

using namespace lbe;

extern "C" lbe_status lbe_fourier_omega(lbe_ctx* ctx, int nv, double vmax, int M, double R, double delta, double N,
                                        lbe_scheme scheme, int iters, const double* e0, double* ratios) {
    if (!ctx) return LBE_BAD_ARG;
    if (nv != 8 && nv != 16 && nv != 24 && nv != 32) return bad_arg(ctx, "nv must be 8, 16, 24 or 32");
    if (M < 2 || M > 64 || (M & (M - 1))) return bad_arg(ctx, "M must be a power of two in [2, 64]");
    if (!(vmax > 0) || R > 2 * vmax) return bad_arg(ctx, "bad vmax or R");
    if (!(delta > 0)) return bad_arg(ctx, "delta must be > 0");
    if (scheme != LBE_CIS && scheme != LBE_SIS) return bad_arg(ctx, "bad scheme");
    if (iters < 1 || !e0 || !ratios) return bad_arg(ctx, "need iters >= 1, e0 and ratios");
    cudaSetDevice(ctx->device);
    lbe_status st;
    DevTables* t = get_tables(ctx, nv, vmax, M, R, &st);
    if (!t) return st;
    const long n3 = (long)nv * nv * nv;
    const double nd = (N > 0 ? N : 1.25) * delta;
    const double dv3 = t->dv * t->dv * t->dv;
    int chunk = 1;
    const size_t scr = fsm_cc_scratch_bytes(*t, 2, 8, &chunk);
    void *e = nullptr, *lp = nullptr, *lo = nullptr, *sc = nullptr, *dd = nullptr, *part = nullptr;
    const size_t vb = 2 * n3 * 8;
    st = dev_alloc(ctx, &e, vb);
    if (st == LBE_OK) st = dev_alloc(ctx, &lp, vb);
    if (st == LBE_OK) st = dev_alloc(ctx, &lo, vb);
    if (st == LBE_OK) st = dev_alloc(ctx, &sc, scr);
    if (st == LBE_OK) st = dev_alloc(ctx, &dd, 2 * 8);
    if (st == LBE_OK) st = dev_alloc(ctx, &part, kBlocks * 6 * 8);
    cudaStream_t s = ctx->stream;
    std::vector<double> hp(kBlocks * 6), hn(kBlocks);
    if (st == LBE_OK) {
        const double dl[2] = {delta, delta};
        cudaMemcpyAsync(dd, dl, sizeof dl, cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(e, e0, vb, cudaMemcpyHostToDevice, s);
        g_h2d += vb + sizeof dl;
        auto norm = [&](double* out) -> lbe_status {  // |e| over both parts
            k_norm2<<<kBlocks, kThreads, 0, s>>>((const double*)e, 2 * n3, (double*)part);
            g_launches += 1;
            cudaMemcpyAsync(hn.data(), part, kBlocks * 8, cudaMemcpyDeviceToHost, s);
            lbe_status q = cuda_status(ctx, cudaStreamSynchronize(s), "norm");
            *out = std::sqrt(host_sum(hn, 1, 0));
            return q;
        };
        double n0 = 0.0;
        st = norm(&n0);
        for (int k = 0; k < iters && st == LBE_OK; ++k) {
            st = fsm_cc_apply<double>(*t, 2, (const double*)dd, (const double*)e, (double*)lp, (double*)lo, sc,
                                      chunk, s, 0);
            if (st != LBE_OK) break;
            k_half<<<kBlocks, kThreads, 0, s>>>((double*)e, (const double*)lp, (const double*)lo, t->nu1_d, t->vel_d,
                                                nv, delta, nd, dv3, (double*)part);
            g_launches += 1;
            cudaMemcpyAsync(hp.data(), part, kBlocks * 6 * 8, cudaMemcpyDeviceToHost, s);
            if ((st = cuda_status(ctx, cudaStreamSynchronize(s), "fourier moments")) != LBE_OK) break;
            double dUr = 0.0, dUi = 0.0;
            if (scheme == LBE_SIS) {
                const double A1r = host_sum(hp, 6, 0), A1i = host_sum(hp, 6, 1);
                const double A2r = host_sum(hp, 6, 2), A2i = host_sum(hp, 6, 3);
                const double Uhr = host_sum(hp, 6, 4), Uhi = host_sum(hp, 6, 5);
                const double p2 = 4.0 * M_PI * M_PI;
                // U = (-2 pi i A1 - 4 pi^2 A2) / (4 pi^2)
                const double Ur = (2.0 * M_PI * A1i - p2 * A2r) / p2;
                const double Ui = (-2.0 * M_PI * A1r - p2 * A2i) / p2;
                dUr = Ur - Uhr;
                dUi = Ui - Uhi;
            }
            k_finish<<<kBlocks, kThreads, 0, s>>>((double*)e, t->vel_d, t->feq_d, nv, dUr, dUi, n0);
            g_launches += 1;
            double r = 0.0;
            if ((st = norm(&r)) != LBE_OK) break;
            ratios[k] = r;
            n0 = r;
        }
    }
    dev_free(ctx, e, vb);
    dev_free(ctx, lp, vb);
    dev_free(ctx, lo, vb);
    dev_free(ctx, sc, scr);
    dev_free(ctx, dd, 2 * 8);
    dev_free(ctx, part, kBlocks * 6 * 8);
    return st;
}

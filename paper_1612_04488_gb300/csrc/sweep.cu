// Transport sweeps, moments, SIS diffusion correction and flow rates (steps A5-A8).
//
// A5  nu_eq h + v.grad h = rhs, second-order upwind (Sec. 2 below Eq. LBE_iteration),
//     first order at the first node after an inflow boundary.  One thread per velocity
//     (1D: per mirror pair v1 > 0 / v1 < 0), marching over the spatial nodes; consecutive
//     threads hold consecutive v3, so every load/store of a node is a coalesced row of the
//     [cell][v] layout.  1D plates: diffuse wall (incoming h = 0) at x1 = -1/2, specular
//     symmetry plane at x1 = 0 with a mirror ghost node (Sec. 2.4).  2D ducts: diffuse walls
//     on all faces, the march over cells in upwind order; the two previous rows are read
//     back from the output array (this thread's own earlier stores).
// A6  U3, q3, F201/4, F021/4, F111/4 per cell (the moment equations of Sec. 2, the
//     non-accelerated moments below Eq. Uz2), one block per cell, fixed reduction order.
// A7  SIS diffusion correction: 1D Eq. first_order (with the N-penalty), marched from the
//     wall; 2D Eq. diffusion_LBE on the interior with U3 = U3^(k+1/2) on the wall ring,
//     solved exactly by DST-I diagonalisation of the five-point Laplacian (FP64).
// A8  Eq. guided correction, flow rates M, Q (Sec. 2.4), relative-change test.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <mutex>

#include "common.cuh"
#include "lbe_internal.h"
#include "sweep.h"

namespace lbe {

namespace {

// Source S of Sec. 2 with X_P = X_T = -1 at velocity (v1, v2, v3).
template <typename T>
__device__ __forceinline__ T source(int forcing, T v1, T v2, T v3, T f) {
    if (forcing == 0) return v3 * f;
    if (forcing == 1) return v3 * (v1 * v1 + v2 * v2 + v3 * v3 - T(2.5)) * f;
    return T(0);  // homogeneous map (refinement correction solves)
}

constexpr int kPre = 8;  // prefetch depth of the sweeps (nodes)

// 4-byte asynchronous copy global -> shared (completes through cp.async.wait_group)
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(smem)),
                 "l"(gmem)
                 : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((unsigned)__cvta_generic_to_shared(smem)),
                 "l"(gmem)
                 : "memory");
}

// Explicitly rounded arithmetic of the march (no contraction into fused multiply-adds), so
// that every schedule of the same march gives the same bits.
template <typename T> struct Rn;
template <> struct Rn<float> {
    static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
    static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
    static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
    static __device__ __forceinline__ float fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
    // the hardware reciprocal approximation (relative error below 2^-22): one instruction and
    // deterministic, so every schedule still computes the same bits
    static __device__ __forceinline__ float rcp(float x) {
        float r;
        asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
        return r;
    }
};
template <> struct Rn<double> {
    static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
    static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
    static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
    static __device__ __forceinline__ double fma(double a, double b, double c) { return __fma_rn(a, b, c); }
    // 1/x without the FP64 divide (the FP64 pipe is this GPU's narrow one): the float reciprocal
    // of x (relative error <= 2^-23 after rounding x to float) refined by two Newton steps
    // r <- r + r (1 - x r), each squaring the error: 2^-46, then the double rounding level
    // (within an ulp or two of the correctly rounded 1/x).  Outside the float range, the divide.
    static __device__ __forceinline__ double rcp(double x) {
        const float xf = (float)x;
        const float ax = fabsf(xf);
        if (!(ax > 1e-30f && ax < 1e30f)) return __ddiv_rn(1.0, x);
        double r = (double)__frcp_rn(xf);
        r = __fma_rn(r, __fma_rn(-x, r, 1.0), r);
        r = __fma_rn(r, __fma_rn(-x, r, 1.0), r);
        return r;
    }
};
// one node of the second-order upwind march: h_i = (rhs_i + S - u (b h_(i-1) + c h_(i-2))) inv,
// inv = 1 / (nu + u a), in fused multiply-adds
template <typename T>
__device__ __forceinline__ T march_node(T r, T S, T u, T b, T c, T hm1, T hm2, T inv) {
    using R = Rn<T>;
    return R::mul(R::fma(-u, R::fma(b, hm1, R::mul(c, hm2)), R::add(r, S)), inv);
}
template <typename T>
__device__ __forceinline__ T march_inv(T nu, T u, T a) {
    using R = Rn<T>;
    return R::rcp(R::fma(u, a, nu));
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init1(uint64_t* bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)));
}
__device__ __forceinline__ void mbar_expect(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
// bounded wait for the phase `parity` of an mbarrier (~2 s); false when the deadline passed
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
    const uint32_t a = smem_addr(bar);
    const long long t0 = clock64();
    for (;;) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(a), "r"(parity)
            : "memory");
        if (ok) return true;
        if (clock64() - t0 > 4000000000LL) return false;
    }
}
// one contiguous global -> shared copy by the bulk-copy (TMA) engine, completing on `bar`
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// 1D sweep (plates): one thread per mirror pair (v1 > 0, v1 < 0) of velocities, marching the
// nodes wall -> symmetry plane for v1 > 0, then back for v1 < 0 starting from the specular
// reflection.  Two schedules of the same arithmetic:
//   SCHED 0  (float) every right-hand side of the thread's two columns is copied to shared
//            memory up front (cp.async, 4 bytes each), so all loads are in flight at once;
//            ~1 KB of shared memory per node and block limits residency to a few blocks per SM;
//   SCHED 1  a register ring: the right-hand sides of the next RING nodes are in flight while a
//            node is solved, no shared memory beyond the coefficients, so the SM holds as many
//            threads as the registers allow;
//   SCHED 2  (float; W a multiple of 128) a ring of node rows in shared memory filled by the
//            bulk-copy (TMA) engine, 512 bytes per node and column, one mbarrier per half ring:
//            up to 32 nodes in flight per block at 16 KB of shared memory;
//   SCHED 3  (float; W a multiple of 128) staged like SCHED 0, each node's 512-byte row copied by
//            32 lanes in 16-byte pieces, then a barrier per column.
// The march coefficients [fa|fb|fc|ba|bb|bc] (n each) are converted once per block into shared
// memory when `staged`, as one float4 per node and direction (a double-to-float conversion per
// node and thread would run at the FP64 rate).
constexpr int kRing = 16;
template <typename T, int SCHED>
__global__ void __launch_bounds__(128) k_sweep1d(const T* __restrict__ rhs, T* __restrict__ h,
                                                 const T* __restrict__ nu1, const T* __restrict__ vel,
                                                 const T* __restrict__ feq,
                                                 const SweepJobDev* __restrict__ jobs,
                                                 const int* __restrict__ active,
                                                 const double* __restrict__ coef, int nv, int staged,
                                                 int quarter) {
    extern __shared__ __align__(16) unsigned char sweep_smem[];
    const SweepJobDev jb = jobs[active ? active[blockIdx.y] : blockIdx.y];
    const int half = nv / 2, n2 = nv * nv;
    // velocities per i1 plane of the data: the whole plane, or in the orbit layout the quarter
    // (j2, j3 < nv / 2) that represents it
    const int W = quarter ? half * half : n2;
    const long n3 = (long)n2 * nv;
    const int n = jb.ncell;
    const double* cg = coef + jb.coef_off;
    // staged (float): per node and direction one float4 {a, b, c, 0} (a: the 1 / (nu + u a)
    // coefficient, b, c: those of h_(i-1), h_(i-2)), direction 0 forward, 1 backward
    float4* sc4 = reinterpret_cast<float4*>(sweep_smem);
    T* sc = reinterpret_cast<T*>(sweep_smem + (size_t)2 * n * sizeof(float4));
    if (staged) {
        for (int k = threadIdx.x; k < 2 * n; k += blockDim.x) {
            const int dir = k / n, i = k % n;
            const double* g = cg + 3 * dir * n + i;
            sc4[k] = make_float4((float)g[0], (float)g[n], (float)g[2 * n], 0.f);
        }
        __syncthreads();
    }
    struct Co3 {
        T a, b, c;
    };
    auto CO = [&](int dir, int i) -> Co3 {
        if (staged) {
            const float4 q = sc4[dir * n + i];
            return {(T)q.x, (T)q.y, (T)q.z};
        }
        const double* g = cg + 3 * dir * n + i;
        return {(T)g[0], (T)g[n], (T)g[2 * n]};
    };
    auto march_co = [&](T x, T S, T uu, const Co3& q, T m1, T m2, T nux) {
        return march_node(x, S, uu, q.b, q.c, m1, m2, march_inv(nux, uu, q.a));
    };
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= half * W) return;
    const int i1p = half + t / W, rem = t % W;
    const int vpos = i1p * W + rem, vneg = (nv - 1 - i1p) * W + rem;  // in the data
    const int i2 = quarter ? rem / half : rem / nv, i3 = quarter ? rem % half : rem % nv;
    const int fpos = (i1p * nv + i2) * nv + i3, fneg = ((nv - 1 - i1p) * nv + i2) * nv + i3;  // in the tables
    const T* r = rhs + jb.cell_off * n3;
    T* o = h + jb.cell_off * n3;
    const T d = (T)jb.delta;
    const T v1 = vel[i1p];
    const T nup = d * nu1[fpos];
    const T w2 = vel[i2], w3 = vel[i3];
    const T Sp = source<T>(jb.forcing, v1, w2, w3, feq[fpos]);
    const T Sn = source<T>(jb.forcing, vel[nv - 1 - i1p], w2, w3, feq[fneg]);
    const T u = -vel[nv - 1 - i1p];
    const T nun = d * nu1[fneg];
    T hm1 = T(0), hm2 = T(0);
    o[vpos] = T(0);
    if constexpr (SCHED == 0) {
        // every right-hand side of this thread's two columns goes in flight at once (after the
        // staged coefficients); the thread waits for its own copies only, so no barrier is
        // needed.  Layout [column][node][thread].
        T* cp = sc;
        T* cn = cp + (long)n * blockDim.x;
        const int tx = threadIdx.x;
        for (int i = 1; i < n; ++i) cp_async4(cp + i * blockDim.x + tx, r + (long)i * n3 + vpos);
        asm volatile("cp.async.commit_group;" ::: "memory");
        for (int i = 0; i + 1 < n; ++i) cp_async4(cn + i * blockDim.x + tx, r + (long)i * n3 + vneg);
        asm volatile("cp.async.commit_group;" ::: "memory");
        asm volatile("cp.async.wait_group 1;" ::: "memory");
#pragma unroll 4
        for (int i = 1; i < n; ++i) {
            const T hi = march_co(cp[i * blockDim.x + tx], Sp, v1, CO(0, i), hm1, hm2, nup);
            o[(long)i * n3 + vpos] = hi;
            hm2 = hm1;
            hm1 = hi;
        }
        // specular symmetry plane: h(x_Ns, v1 < 0) = h(x_Ns, -v1); the ghost node carries
        // h(x_(Ns-1), -v1)
        T g1 = hm1, g2 = hm2;
        o[(long)(n - 1) * n3 + vneg] = hm1;
        asm volatile("cp.async.wait_group 0;" ::: "memory");
#pragma unroll 4
        for (int i = n - 2; i >= 0; --i) {
            const T hi = march_co(cn[i * blockDim.x + tx], Sn, u, CO(1, i), g1, g2, nun);
            o[(long)i * n3 + vneg] = hi;
            g2 = g1;
            g1 = hi;
        }
    } else if constexpr (SCHED == 3) {
        // as SCHED 0, but the block's 128 velocities are contiguous in both columns (W a multiple
        // of 128, float), so each node's 512-byte row is copied by 32 lanes in 16-byte pieces:
        // a quarter of the copy instructions, then a barrier per column.  Layout as SCHED 0.
        T* cp = sc;
        T* cn = cp + (long)n * blockDim.x;
        const int tx = threadIdx.x;
        const long cpos0 = vpos - tx, cneg0 = vneg - tx;
        if constexpr (sizeof(T) == 4) {
            for (int q = tx; q < (n - 1) * 32; q += blockDim.x) {  // forward rows: nodes 1 .. n-1
                const int i = 1 + (q >> 5), pc = 4 * (q & 31);
                cp_async16(cp + i * 128 + pc, r + (long)i * n3 + cpos0 + pc);
            }
            asm volatile("cp.async.commit_group;" ::: "memory");
            for (int q = tx; q < (n - 1) * 32; q += blockDim.x) {  // backward rows: nodes 0 .. n-2
                const int i = q >> 5, pc = 4 * (q & 31);
                cp_async16(cn + i * 128 + pc, r + (long)i * n3 + cneg0 + pc);
            }
            asm volatile("cp.async.commit_group;" ::: "memory");
        }
        asm volatile("cp.async.wait_group 1;" ::: "memory");
        __syncthreads();
#pragma unroll 4
        for (int i = 1; i < n; ++i) {
            const T hi = march_co(cp[i * blockDim.x + tx], Sp, v1, CO(0, i), hm1, hm2, nup);
            o[(long)i * n3 + vpos] = hi;
            hm2 = hm1;
            hm1 = hi;
        }
        T g1 = hm1, g2 = hm2;
        o[(long)(n - 1) * n3 + vneg] = hm1;
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        __syncthreads();
#pragma unroll 4
        for (int i = n - 2; i >= 0; --i) {
            const T hi = march_co(cn[i * blockDim.x + tx], Sn, u, CO(1, i), g1, g2, nun);
            o[(long)i * n3 + vneg] = hi;
            g2 = g1;
            g1 = hi;
        }
    } else if constexpr (SCHED == 2) {
        // The block's 128 velocities are contiguous in both columns (W is a multiple of 128),
        // so each node is one 512-byte row per column, copied by the bulk-copy engine into a
        // ring of two halves of HR rows in shared memory.  The two columns form one stream of
        // 2 (n - 1) rows: forward nodes 1 .. n-1, then backward nodes n-2 .. 0.  Half k sits
        // in slot k & 1, completes on that slot's mbarrier (its use number k >> 1 gives the
        // phase), and is refilled with half k + 2 once every thread has read it.
        constexpr int HR = 16;
        const int tx = threadIdx.x;
        const int P = 2 * (n - 1), nh = (P + HR - 1) / HR;
        T* ring = reinterpret_cast<T*>(sweep_smem + (size_t)2 * n * sizeof(float4));
        uint64_t* bar = reinterpret_cast<uint64_t*>(ring + 2 * HR * 128);
        const long cpos0 = vpos - tx, cneg0 = vneg - tx;  // the block's first velocity per column
        int issued = 0, landed = 0;  // halves issued (thread 0) / seen complete by every thread
        auto issue = [&](int k) {  // thread 0: rows of half k
            if (k >= nh) return;
            issued = k + 1;
            const int cnt = min(HR, P - k * HR);
            uint64_t* bk = bar + (k & 1);
            mbar_expect(bk, (uint32_t)(cnt * 128 * sizeof(T)));
            for (int q = 0; q < cnt; ++q) {
                const int p = k * HR + q;
                const long src = p < n - 1 ? (long)(p + 1) * n3 + cpos0 : (long)(n - 2 - (p - (n - 1))) * n3 + cneg0;
                bulk_g2s(ring + ((k & 1) * HR + q) * 128, r + src, 128 * sizeof(T), bk);
            }
        };
        if (tx == 0) {
            mbar_init1(&bar[0]);
            mbar_init1(&bar[1]);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        __syncthreads();
        if (tx == 0) {
            issue(0);
            issue(1);
        }
        T g1 = T(0), g2 = T(0);
        for (int p = 0; p < P; ++p) {
            const int k = p / HR;
            if (p % HR == 0) {  // every thread saw half k land, or all give up together
                const bool ok = mbar_wait_bounded(&bar[k & 1], (uint32_t)((k >> 1) & 1));
                if (!__syncthreads_and(ok)) break;
                landed = k + 1;
            }
            const T x = ring[((k & 1) * HR + p % HR) * 128 + tx];
            if (p < n - 1) {
                const int i = p + 1;
                const T hi = march_co(x, Sp, v1, CO(0, i), hm1, hm2, nup);
                o[(long)i * n3 + vpos] = hi;
                hm2 = hm1;
                hm1 = hi;
                if (i == n - 1) {  // specular symmetry plane, then the backward march
                    g1 = hm1;
                    g2 = hm2;
                    o[(long)(n - 1) * n3 + vneg] = hm1;
                }
            } else {
                const int i = n - 2 - (p - (n - 1));
                const T hi = march_co(x, Sn, u, CO(1, i), g1, g2, nun);
                o[(long)i * n3 + vneg] = hi;
                g2 = g1;
                g1 = hi;
            }
            if (p % HR == HR - 1 && p + 1 < P) {  // half k read by every thread: refill its slot
                __syncthreads();
                if (tx == 0) {
                    // order the block's reads of the slot before the copy engine's writes
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    issue(k + 2);
                }
            }
        }
        // after a failed wait: the copies still in flight land before the block leaves
        if (tx == 0)
            for (int k = landed; k < issued; ++k) mbar_wait_bounded(&bar[k & 1], (uint32_t)((k >> 1) & 1));
    } else {
        T rb[kRing];
#pragma unroll
        for (int k = 0; k < kRing; ++k) rb[k] = 1 + k < n ? r[(long)(1 + k) * n3 + vpos] : T(0);
        for (int i0 = 1; i0 < n; i0 += kRing) {
#pragma unroll
            for (int k = 0; k < kRing; ++k) {
                const int i = i0 + k;
                if (i < n) {
                    const T ri = rb[k];
                    if (i + kRing < n) rb[k] = r[(long)(i + kRing) * n3 + vpos];
                    const T hi = march_co(ri, Sp, v1, CO(0, i), hm1, hm2, nup);
                    o[(long)i * n3 + vpos] = hi;
                    hm2 = hm1;
                    hm1 = hi;
                }
            }
        }
        T g1 = hm1, g2 = hm2;
        o[(long)(n - 1) * n3 + vneg] = hm1;
#pragma unroll
        for (int k = 0; k < kRing; ++k) {
            const int i = n - 2 - k;
            rb[k] = i >= 0 ? r[(long)i * n3 + vneg] : T(0);
        }
        for (int i0 = n - 2; i0 >= 0; i0 -= kRing) {
#pragma unroll
            for (int k = 0; k < kRing; ++k) {
                const int i = i0 - k;
                if (i >= 0) {
                    const T ri = rb[k];
                    if (i - kRing >= 0) rb[k] = r[(long)(i - kRing) * n3 + vneg];
                    const T hi = march_co(ri, Sn, u, CO(1, i), g1, g2, nun);
                    o[(long)i * n3 + vneg] = hi;
                    g2 = g1;
                    g1 = hi;
                }
            }
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(128) k_sweep2d(const T* __restrict__ rhs, T* __restrict__ h,
                                                 const T* __restrict__ nu1, const T* __restrict__ vel,
                                                 const T* __restrict__ feq,
                                                 const SweepJobDev* __restrict__ jobs,
                                                 const int* __restrict__ active,
                                                 const double* __restrict__ coef, int nv, int staged, int half) {
    extern __shared__ __align__(16) unsigned char sweep_smem[];
    const SweepJobDev jb = jobs[active ? active[blockIdx.y] : blockIdx.y];
    const int n2 = nv * nv;
    const long n3 = (long)n2 * nv;
    const int nx = jb.nx, ny = jb.ny;
    const int W3 = half ? nv / 2 : nv;  // i3 values of the data (half: the v3 < 0 half)
    // [xa|xb|xc] (nx each) [ya|yb|yc] (ny each), staged as in the 1D sweep
    const double* cg = coef + jb.coef_off;
    T* sc = reinterpret_cast<T*>(sweep_smem);
    if (staged) {
        for (int k = threadIdx.x; k < 3 * (nx + ny); k += blockDim.x) sc[k] = (T)cg[k];
        __syncthreads();
    }
    auto CX = [&](int a, int i) -> T { return staged ? sc[a * nx + i] : (T)cg[a * nx + i]; };
    auto CY = [&](int a, int j) -> T { return staged ? sc[3 * nx + a * ny + j] : (T)cg[3 * nx + a * ny + j]; };
    const int v = blockIdx.x * blockDim.x + threadIdx.x;  // in the data
    if (v >= n2 * W3) return;
    const int i1 = v / (nv * W3), i2 = (v / W3) % nv, i3 = v % W3;
    const int vf = (i1 * nv + i2) * nv + i3;  // in the tables
    const bool s1 = i1 >= nv / 2, s2 = i2 >= nv / 2;
    const T u1 = s1 ? vel[i1] : -vel[i1];
    const T u2 = s2 ? vel[i2] : -vel[i2];
    const T nu = (T)jb.delta * nu1[vf];
    const T S = source<T>(jb.forcing, vel[i1], vel[i2], vel[i3], feq[vf]);
    const T* r = rhs + jb.cell_off * n3;
    T* o = h + jb.cell_off * n3;
    const int dj = s2 ? -1 : 1;  // offset to the upwind row in j
    // the right-hand side and the two upwind-row values (this thread's own outputs of the two
    // previous rows) of the next D cells are in flight while a cell is solved
    constexpr int D = sizeof(T) == 4 ? 16 : 8;
    for (int mj = 0; mj < ny; ++mj) {
        const int j = s2 ? mj : ny - 1 - mj;
        T hm1 = T(0), hm2 = T(0);
        const T ay = CY(0, mj), by = CY(1, mj), cy = CY(2, mj);
        auto cell_of = [&](int m) { return (long)(s1 ? m : nx - 1 - m) * ny + j; };
        T buf[D], y1[D], y2[D];
        const T diag = nu + u2 * ay;
        auto fetch = [&](int k, int m) {
            const long cell = cell_of(m);
            buf[k] = r[cell * n3 + v];
            y1[k] = mj >= 1 ? o[(cell + dj) * n3 + v] : T(0);
            y2[k] = mj >= 2 ? o[(cell + 2 * dj) * n3 + v] : T(0);
        };
#pragma unroll
        for (int k = 0; k < D; ++k)
            if (k < nx) fetch(k, k);
        for (int m0 = 0; m0 < nx; m0 += D) {
#pragma unroll
            for (int k = 0; k < D; ++k) {
                const int mi = m0 + k;
                if (mi < nx) {
                    const long cell = cell_of(mi);
                    T acc = buf[k] + S;
                    const T w1 = y1[k], w2 = y2[k];
                    if (mi + D < nx) fetch(k, mi + D);
                    const T inv = Rn<T>::rcp(diag + u1 * CX(0, mi));
                    if (mi >= 1) acc -= u1 * CX(1, mi) * hm1;
                    if (mi >= 2) acc -= u1 * CX(2, mi) * hm2;
                    if (mj >= 1) acc -= u2 * by * w1;
                    if (mj >= 2) acc -= u2 * cy * w2;
                    const T hij = acc * inv;
                    o[cell * n3 + v] = hij;
                    hm2 = hm1;
                    hm1 = hij;
                }
            }
        }
    }
}

// 2D sweep as a wavefront.  For one velocity the upwind march over the nx x ny cells is a
// recurrence in both directions, but the cells of one anti-diagonal (march indices
// mi + mj = d) are independent.  A block takes 32 consecutive velocities (one per lane) and
// strips of WR rows (march order in y): warp w owns row mj = base + w and at step d solves
// its cell mi = d - w, with its own two previous cells in x in registers and the two cells
// below it in y from the warps w - 1, w - 2 of the previous steps through a 3-slot ring in
// shared memory (one barrier per step); the last two rows of a strip are kept for the first
// two warps of the next.  Loads and stores are coalesced rows of 32 velocities.  Each
// warp's next right-hand sides are prefetched D cells ahead in a register queue.  The
// arithmetic is that of the per-velocity march.
template <typename T, int WR>
__global__ void __launch_bounds__(32 * WR) k_sweep2d_wave(const T* __restrict__ rhs, T* __restrict__ h,
                                                          const T* __restrict__ nu1, const T* __restrict__ vel,
                                                          const T* __restrict__ feq,
                                                          const SweepJobDev* __restrict__ jobs,
                                                          const int* __restrict__ active,
                                                          const double* __restrict__ coef, int nv, int half) {
    constexpr int D = 8;
    extern __shared__ __align__(16) unsigned char sweep_smem[];
    const SweepJobDev jb = jobs[active ? active[blockIdx.y] : blockIdx.y];
    const int n2 = nv * nv;
    const long n3 = (long)n2 * nv;
    const int nx = jb.nx, ny = jb.ny;
    T* cxs = reinterpret_cast<T*>(sweep_smem);  // [xa|xb|xc] (nx each)
    T* cys = cxs + 3 * nx;                       // [ya|yb|yc] (ny each)
    T* ring = cys + 3 * ny;                      // [3][WR][32]
    T* prev = ring + 3 * WR * 32;                // [2][nx][32]: rows base - 2, base - 1
    const double* cg = coef + jb.coef_off;
    for (int k = threadIdx.x; k < 3 * (nx + ny); k += blockDim.x) cxs[k] = (T)cg[k];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int W3 = half ? nv / 2 : nv;  // i3 values of the data (half: the v3 < 0 half)
    const int v = blockIdx.x * 32 + lane;  // in the data
    const bool vok = v < n2 * W3;
    const int vv = vok ? v : 0;
    const int i1 = vv / (nv * W3), i2 = (vv / W3) % nv, i3 = vv % W3;
    const int vf = (i1 * nv + i2) * nv + i3;  // in the tables
    const bool s1 = i1 >= nv / 2, s2 = i2 >= nv / 2;
    const T u1 = s1 ? vel[i1] : -vel[i1];
    const T u2 = s2 ? vel[i2] : -vel[i2];
    const T nu = (T)jb.delta * nu1[vf];
    const T S = source<T>(jb.forcing, vel[i1], vel[i2], vel[i3], feq[vf]);
    const T* r = rhs + jb.cell_off * n3;
    T* o = h + jb.cell_off * n3;
    __syncthreads();
    for (int base = 0; base < ny; base += WR) {
        const int mj = base + w;
        const bool rowok = vok && mj < ny;
        const int j = s2 ? mj : ny - 1 - mj;
        const T ay = rowok ? cys[mj] : T(0), by = rowok ? cys[ny + mj] : T(0), cy = rowok ? cys[2 * ny + mj] : T(0);
        const T diag = nu + u2 * ay;
        auto cell_of = [&](int m) { return (long)(s1 ? m : nx - 1 - m) * ny + j; };
        T q[D];  // right-hand sides of cells mi .. mi + D - 1 of this row
#pragma unroll
        for (int k = 0; k < D; ++k) q[k] = (rowok && k < nx) ? r[cell_of(k) * n3 + v] : T(0);
        T hm1 = T(0), hm2 = T(0);
        const int nsteps = nx + WR - 1;
        for (int d = 0; d < nsteps; ++d) {
            const int mi = d - w;
            if (rowok && mi >= 0 && mi < nx) {
                const T rq = q[0];
#pragma unroll
                for (int k = 0; k + 1 < D; ++k) q[k] = q[k + 1];
                q[D - 1] = mi + D < nx ? r[cell_of(mi + D) * n3 + v] : T(0);
                T w1 = T(0), w2 = T(0);  // h at (mi, mj - 1), (mi, mj - 2)
                if (mj >= 1) w1 = w >= 1 ? ring[(((d - 1) % 3) * WR + w - 1) * 32 + lane] : prev[(nx + mi) * 32 + lane];
                if (mj >= 2)
                    w2 = w >= 2 ? ring[(((d - 2) % 3) * WR + w - 2) * 32 + lane]
                                : prev[((w == 1 ? nx : 0) + mi) * 32 + lane];
                T acc = rq + S;
                const T inv = Rn<T>::rcp(diag + u1 * cxs[mi]);
                if (mi >= 1) acc -= u1 * cxs[nx + mi] * hm1;
                if (mi >= 2) acc -= u1 * cxs[2 * nx + mi] * hm2;
                if (mj >= 1) acc -= u2 * by * w1;
                if (mj >= 2) acc -= u2 * cy * w2;
                const T hij = acc * inv;
                o[cell_of(mi) * n3 + v] = hij;
                ring[((d % 3) * WR + w) * 32 + lane] = hij;
                if (w == WR - 2) prev[mi * 32 + lane] = hij;
                if (w == WR - 1) prev[(nx + mi) * 32 + lane] = hij;
                hm2 = hm1;
                hm1 = hij;
            }
            __syncthreads();
        }
    }
}

// Per-thread accumulator: plain double on the FP64 path; on the FP32 path a compensated
// (Kahan) float sum, whose error does not grow with the number of terms.
template <typename T> struct Acc;
template <> struct Acc<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double x) { s += x; }
    __device__ __forceinline__ double value() const { return s; }
};
template <> struct Acc<float> {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float x) {
        const float y = x - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
    __device__ __forceinline__ dfloat pair() const { return df_fast2sum(s, -c); }  // s - c
};

// mom[cell][5] = sum_v {v3, (|v|^2-5/2) v3, (2 v1^2-1) v3, (2 v2^2-1) v3, 2 v1 v2 v3} h dv^3
// One block of 8 NV threads per cell: thread t owns i3 = t % NV and the rows i2 = t/NV + 8k.
// v3 is fixed per thread and v2 per row, so they are factored out: per row the thread sums
// h, v1^2 h and v1 h over i1 and combines them with v2 and v3 once (the FP64 pipe is the
// limit of the double instance).
template <typename T, int NV>
__global__ void __launch_bounds__(8 * NV) k_moments(const T* __restrict__ h, const T* __restrict__ vel,
                                                    double dv3, long cell0, double* __restrict__ mom) {
    __shared__ double red[32 * 5];
    constexpr int R = NV / 8;  // rows per thread and plane
    const long cell = cell0 + blockIdx.x;
    constexpr long n3 = (long)NV * NV * NV;
    const int i3 = threadIdx.x % NV, r0 = threadIdx.x / NV;
    const T v3 = vel[i3];
    T v2s[R], v2v[R];
#pragma unroll
    for (int k = 0; k < R; ++k) {
        v2v[k] = vel[r0 + 8 * k];
        v2s[k] = v2v[k] * v2v[k];
    }
    // per row i2 the thread sums h, v1^2 h and v1 h over i1 (three operations per value);
    // the v2 and v3 factors are applied once afterwards
    const T* hc = h + cell * n3 + i3;
    Acc<T> S0[R], S1[R], S4[R];
    for (int i1 = 0; i1 < NV; ++i1) {
        const T v1 = vel[i1], v1s = v1 * v1;
        T x[R];
#pragma unroll
        for (int k = 0; k < R; ++k) x[k] = hc[((long)i1 * NV + r0 + 8 * k) * NV];
#pragma unroll
        for (int k = 0; k < R; ++k) {
            S0[k].add(x[k]);
            S1[k].add(v1s * x[k]);
            S4[k].add(v1 * x[k]);
        }
    }
    if constexpr (sizeof(T) == 4) {
        // float data: combine and reduce in double-float (the FP64 pipe is a small fraction of
        // the FP32 one here, and a double tail would cost more than the sums themselves)
        __shared__ dfloat redx[32 * 5];
        dfloat a0(0), a2(0), a3(0), a4(0);  // sums of h, v1^2 h, v2^2 h, v1 v2 h
#pragma unroll
        for (int k = 0; k < R; ++k) {
            const dfloat s0 = S0[k].pair(), s4 = S4[k].pair();
            a0 = a0 + s0;
            a2 = a2 + S1[k].pair();
            a3 = a3 + dfloat((float)v2s[k], 0.f) * s0;
            a4 = a4 + dfloat((float)v2v[k], 0.f) * s4;
        }
        const dfloat w3((float)v3, 0.f), w3s = w3 * w3;
        dfloat s[5] = {w3 * a0, w3 * ((a2 + a3) + (w3s - dfloat(2.5f, 0.f)) * a0), w3 * ((a2 + a2) - a0),
                       w3 * ((a3 + a3) - a0), (w3 + w3) * a4};
        block_reduce_df<5>(s, redx);
        if (threadIdx.x == 0)
            for (int k = 0; k < 5; ++k) mom[cell * 5 + k] = (double)s[k] * dv3;
    } else {
        double a0 = 0.0, a2 = 0.0, a3 = 0.0, a4 = 0.0;  // sums of h, v1^2 h, v2^2 h, v1 v2 h
#pragma unroll
        for (int k = 0; k < R; ++k) {
            const double s0 = S0[k].value();
            a0 += s0;
            a2 += S1[k].value();
            a3 += (double)v2s[k] * s0;
            a4 += (double)v2v[k] * S4[k].value();
        }
        const double w3 = (double)v3;
        double s[5] = {w3 * a0, w3 * (a2 + a3 + (w3 * w3 - 2.5) * a0), w3 * (2.0 * a2 - a0),
                       w3 * (2.0 * a3 - a0), 2.0 * w3 * a4};
        block_reduce<5>(s, red);
        if (threadIdx.x == 0)
            for (int k = 0; k < 5; ++k) mom[cell * 5 + k] = s[k] * dv3;
    }
}

// The same moments of a plate cell in the orbit layout (h[i1][j2][j3], j2, j3 < nv / 2, one
// value per orbit {1, R2, R3, R2 R3} of the parity odd in v3 and even in v2).  The first four
// integrands are even under both reflections, so each is four times its sum over the stored
// quarter; 2 v1 v2 v3 h is odd under R2 and sums to zero.  One thread per (j2, j3), the block
// rounded up to whole warps.
template <typename T, int NV>
__global__ void __launch_bounds__(256) k_moments_q(const T* __restrict__ h, const T* __restrict__ vel, double dv3,
                                                   long cell0, double* __restrict__ mom) {
    constexpr int H = NV / 2;
    constexpr long n3 = (long)NV * NV * NV;
    const long cell = cell0 + blockIdx.x;
    const int p = threadIdx.x;
    Acc<T> S0, S1;  // sums of h and v1^2 h over i1
    T v2 = T(0), v3 = T(0);
    if (p < H * H) {
        v2 = vel[p / H];
        v3 = vel[p % H];
        const T* hc = h + cell * n3 + p;
        for (int i1 = 0; i1 < NV; ++i1) {
            const T v1 = vel[i1], x = hc[(long)i1 * H * H];
            S0.add(x);
            S1.add(v1 * v1 * x);
        }
    }
    if constexpr (sizeof(T) == 4) {
        __shared__ dfloat redx[32 * 4];
        dfloat s[4] = {dfloat(0), dfloat(0), dfloat(0), dfloat(0)};
        if (p < H * H) {
            const dfloat a0 = S0.pair(), a2 = S1.pair(), a3 = dfloat((float)(v2 * v2), 0.f) * a0;
            const dfloat w3((float)v3, 0.f), w3s = w3 * w3;
            s[0] = w3 * a0;
            s[1] = w3 * ((a2 + a3) + (w3s - dfloat(2.5f, 0.f)) * a0);
            s[2] = w3 * ((a2 + a2) - a0);
            s[3] = w3 * ((a3 + a3) - a0);
        }
        block_reduce_df<4>(s, redx);
        if (threadIdx.x == 0) {
            for (int k = 0; k < 4; ++k) mom[cell * 5 + k] = 4.0 * (double)s[k] * dv3;
            mom[cell * 5 + 4] = 0.0;
        }
    } else {
        __shared__ double red[32 * 4];
        double s[4] = {0.0, 0.0, 0.0, 0.0};
        if (p < H * H) {
            const double a0 = S0.value(), a2 = S1.value(), a3 = (double)v2 * (double)v2 * a0;
            const double w3 = (double)v3;
            s[0] = w3 * a0;
            s[1] = w3 * (a2 + a3 + (w3 * w3 - 2.5) * a0);
            s[2] = w3 * (2.0 * a2 - a0);
            s[3] = w3 * (2.0 * a3 - a0);
        }
        block_reduce<4>(s, red);
        if (threadIdx.x == 0) {
            for (int k = 0; k < 4; ++k) mom[cell * 5 + k] = 4.0 * s[k] * dv3;
            mom[cell * 5 + 4] = 0.0;
        }
    }
}

// The same moments of a duct cell in the orbit layout (h[i1][i2][j3], j3 < nv / 2: one value per
// orbit {1, R3} of the parity odd in v3).  All five integrands are even under R3, so each is
// twice its sum over the stored half.  One thread per (i2, j3).
template <typename T, int NV>
__global__ void __launch_bounds__(512) k_moments_h(const T* __restrict__ h, const T* __restrict__ vel, double dv3,
                                                   long cell0, double* __restrict__ mom) {
    constexpr int H = NV / 2;
    constexpr long n3 = (long)NV * NV * NV;
    const long cell = cell0 + blockIdx.x;
    const int p = threadIdx.x;  // < NV * H
    const T v2 = vel[p / H], v3 = vel[p % H];
    Acc<T> S0, S1, S4;  // sums of h, v1^2 h and v1 h over i1
    const T* hc = h + cell * n3 + p;
    for (int i1 = 0; i1 < NV; ++i1) {
        const T v1 = vel[i1], x = hc[(long)i1 * NV * H];
        S0.add(x);
        S1.add(v1 * v1 * x);
        S4.add(v1 * x);
    }
    if constexpr (sizeof(T) == 4) {
        __shared__ dfloat redx[32 * 5];
        const dfloat a0 = S0.pair(), a2 = S1.pair(), a4 = S4.pair();
        const dfloat a3 = dfloat((float)(v2 * v2), 0.f) * a0;
        const dfloat w3((float)v3, 0.f), w3s = w3 * w3;
        dfloat sm[5] = {w3 * a0, w3 * ((a2 + a3) + (w3s - dfloat(2.5f, 0.f)) * a0), w3 * ((a2 + a2) - a0),
                        w3 * ((a3 + a3) - a0), (w3 + w3) * (dfloat((float)v2, 0.f) * a4)};
        block_reduce_df<5>(sm, redx);
        if (threadIdx.x == 0)
            for (int k = 0; k < 5; ++k) mom[cell * 5 + k] = 2.0 * (double)sm[k] * dv3;
    } else {
        __shared__ double red[32 * 5];
        const double a0 = S0.value(), a2 = S1.value(), a4 = S4.value(), w2 = (double)v2, w3 = (double)v3;
        const double a3 = w2 * w2 * a0;
        double sm[5] = {w3 * a0, w3 * (a2 + a3 + (w3 * w3 - 2.5) * a0), w3 * (2.0 * a2 - a0), w3 * (2.0 * a3 - a0),
                        2.0 * w3 * w2 * a4};
        block_reduce<5>(sm, red);
        if (threadIdx.x == 0)
            for (int k = 0; k < 5; ++k) mom[cell * 5 + k] = 2.0 * sm[k] * dv3;
    }
}

// 2D Poisson right-hand side of Eq. diffusion_LBE (N-penalised) on the interior cells.
__device__ double poisson_rhs(const double* mom, const double* G, int i, int j, int ny, double dx,
                              double dy, double ndsig) {
    auto W1 = [&](int a, int b) { return mom[((long)a * ny + b) * 5 + 2]; };
    auto W2 = [&](int a, int b) { return mom[((long)a * ny + b) * 5 + 3]; };
    auto X = [&](int a, int b) { return mom[((long)a * ny + b) * 5 + 4]; };
    auto G1 = [&](int a, int b) { return G[((long)a * ny + b) * 2 + 0]; };
    auto G2 = [&](int a, int b) { return G[((long)a * ny + b) * 2 + 1]; };
    return -ndsig - (W1(i + 1, j) - 2.0 * W1(i, j) + W1(i - 1, j)) / (dx * dx) -
           2.0 * (X(i + 1, j + 1) - X(i + 1, j - 1) - X(i - 1, j + 1) + X(i - 1, j - 1)) / (4.0 * dx * dy) -
           (W2(i, j + 1) - 2.0 * W2(i, j) + W2(i, j - 1)) / (dy * dy) +
           (G1(i + 1, j) - G1(i - 1, j)) / (2.0 * dx) + (G2(i, j + 1) - G2(i, j - 1)) / (2.0 * dy);
}

// One block per job: diffusion correction (SIS), corrected moments, flow rates, test.
__global__ void __launch_bounds__(256) k_sis_update(const SisJobDev* __restrict__ jobs,
                                                    const int* __restrict__ active,
                                                    const double* __restrict__ mom,
                                                    const double* __restrict__ G,
                                                    const double* __restrict__ coef,
                                                    double* __restrict__ work, double cU, double cq,
                                                    double* __restrict__ dU, double* __restrict__ U3,
                                                    JobState* __restrict__ state) {
    __shared__ double red[32 * 2];
    const int jid = active ? active[blockIdx.x] : blockIdx.x;
    const SisJobDev jb = jobs[jid];
    JobState* st = state + jid;
    if (st->done) {  // finished before this iteration: state, U3 and h stay as they are
        if (threadIdx.x == 0) st->skip = 1;
        return;
    }
    if (threadIdx.x == 0) st->skip = 0;
    const long c0 = jb.cell_off;
    const int n = jb.ncell;
    const double* m = mom + c0 * 5;
    double* du = dU + c0;
    if (jb.scheme == 0) {  // CIS: no correction
        for (int c = threadIdx.x; c < n; c += blockDim.x) du[c] = 0.0;
    } else if (jb.dim == 1) {
        // The march y_i = (rhs_i - fb_i y_(i-1) - fc_i y_(i-2)) / fa_i (coefficient block
        // [1/fa | fb | fc | x]) is the affine map Y_i = A_i Y_(i-1) + b_i of Y_i = (y_i, y_(i-1)),
        // A_i = [[-fb_i / fa_i, -fc_i / fa_i], [1, 0]], b_i = (rhs_i / fa_i, 0), from
        // Y_0 = (U(x0) + W(x0), 0).  Warp 0 runs it as a scan, 128 nodes per pass: each lane
        // composes the maps of its 4 consecutive nodes, a shuffle scan composes them across the
        // lanes, and each lane applies its exclusive prefix to the carried state and walks its
        // nodes.  du_i = y_i - W_i - U_i.
        if (threadIdx.x < 32) {
            const int lane = threadIdx.x;
            const double* fa = coef + jb.coef_off;
            const double* fb = fa + n;
            const double* fc = fb + n;
            const double* xs = fc + n;
            double s0y = m[0] + m[2], s1y = 0.0;  // the carried state Y_(s-1)
            if (lane == 0) du[0] = 0.0;
            for (int s0 = 1; s0 < n; s0 += 128) {
                const int e0 = s0 + 4 * lane;
                double ia[4], ib[4], ir[4];  // -fb / fa, -fc / fa, rhs / fa of the lane's nodes
                double a00 = 1.0, a01 = 0.0, a10 = 0.0, a11 = 1.0, b0 = 0.0, b1 = 0.0;  // identity
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int i = e0 + k;
                    if (i < n) {
                        const double f = fa[i];
                        ia[k] = -fb[i] * f;
                        ib[k] = i >= 2 ? -fc[i] * f : 0.0;
                        ir[k] = (-jb.ndsig * xs[i] + G[(c0 + i) * 2]) * f;
                        // (A_i, b_i) after the maps so far
                        const double n00 = ia[k] * a00 + ib[k] * a10, n01 = ia[k] * a01 + ib[k] * a11;
                        const double nb0 = ia[k] * b0 + ib[k] * b1 + ir[k];
                        a10 = a00;
                        a11 = a01;
                        b1 = b0;
                        a00 = n00;
                        a01 = n01;
                        b0 = nb0;
                    }
                }
                // inclusive scan over the lanes: this lane's maps after those of the lanes below
#pragma unroll
                for (int off = 1; off < 32; off <<= 1) {
                    const double p00 = __shfl_up_sync(0xffffffffu, a00, off), p01 = __shfl_up_sync(0xffffffffu, a01, off);
                    const double p10 = __shfl_up_sync(0xffffffffu, a10, off), p11 = __shfl_up_sync(0xffffffffu, a11, off);
                    const double q0 = __shfl_up_sync(0xffffffffu, b0, off), q1 = __shfl_up_sync(0xffffffffu, b1, off);
                    if (lane >= off) {
                        const double n00 = a00 * p00 + a01 * p10, n01 = a00 * p01 + a01 * p11;
                        const double n10 = a10 * p00 + a11 * p10, n11 = a10 * p01 + a11 * p11;
                        const double nb0 = a00 * q0 + a01 * q1 + b0, nb1 = a10 * q0 + a11 * q1 + b1;
                        a00 = n00;
                        a01 = n01;
                        a10 = n10;
                        a11 = n11;
                        b0 = nb0;
                        b1 = nb1;
                    }
                }
                // state before this lane's nodes: the exclusive prefix applied to the carry
                const double e00 = __shfl_up_sync(0xffffffffu, a00, 1), e01 = __shfl_up_sync(0xffffffffu, a01, 1);
                const double e10 = __shfl_up_sync(0xffffffffu, a10, 1), e11 = __shfl_up_sync(0xffffffffu, a11, 1);
                const double f0 = __shfl_up_sync(0xffffffffu, b0, 1), f1 = __shfl_up_sync(0xffffffffu, b1, 1);
                double y1 = s0y, y2 = s1y;
                if (lane > 0) {
                    y1 = e00 * s0y + e01 * s1y + f0;
                    y2 = e10 * s0y + e11 * s1y + f1;
                }
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int i = e0 + k;
                    if (i < n) {
                        const double yi = ia[k] * y1 + ib[k] * y2 + ir[k];
                        du[i] = (yi - m[i * 5 + 2]) - m[i * 5 + 0];
                        y2 = y1;
                        y1 = yi;
                    }
                }
                // the next pass starts from the state after all 128 nodes (lane 31's prefix)
                const double n0 = a00 * s0y + a01 * s1y + b0, n1 = a10 * s0y + a11 * s1y + b1;
                s0y = __shfl_sync(0xffffffffu, n0, 31);
                s1y = __shfl_sync(0xffffffffu, n1, 31);
            }
        }
    } else {
        // 2D: interior mx x my, U = Uh on the ring; DST-I solve in `work`
        const int nx = jb.nx, ny = jb.ny, mx = nx - 2, my = ny - 2;
        const double dx = jb.width / nx, dy = 1.0 / ny;
        double* B = work + jb.work_off;
        double* T1 = B + (long)mx * my;
        const double* Sx = coef + jb.coef_off;           // [mx][mx]
        const double* Sy = Sx + (long)mx * mx;           // [my][my]
        const double* lam = Sy + (long)my * my;          // [mx][my]
        const double* Gc = G + c0 * 2;
        for (int k = threadIdx.x; k < mx * my; k += blockDim.x) {
            const int p = k / my, q = k % my, i = p + 1, j = q + 1;
            double b = poisson_rhs(m, Gc, i, j, ny, dx, dy, jb.ndsig);
            if (p == 0) b -= m[((long)0 * ny + j) * 5] / (dx * dx);
            if (p == mx - 1) b -= m[((long)(nx - 1) * ny + j) * 5] / (dx * dx);
            if (q == 0) b -= m[((long)i * ny + 0) * 5] / (dy * dy);
            if (q == my - 1) b -= m[((long)i * ny + ny - 1) * 5] / (dy * dy);
            B[k] = b;
        }
        __syncthreads();
        for (int k = threadIdx.x; k < mx * my; k += blockDim.x) {  // T1 = Sx B
            const int p = k / my, q = k % my;
            double s = 0.0;
            for (int a = 0; a < mx; ++a) s += Sx[p * mx + a] * B[a * my + q];
            T1[k] = s;
        }
        __syncthreads();
        for (int k = threadIdx.x; k < mx * my; k += blockDim.x) {  // B = (T1 Sy) / lam
            const int p = k / my, q = k % my;
            double s = 0.0;
            for (int a = 0; a < my; ++a) s += T1[p * my + a] * Sy[a * my + q];
            B[k] = s / lam[k];
        }
        __syncthreads();
        for (int k = threadIdx.x; k < mx * my; k += blockDim.x) {  // T1 = Sx B
            const int p = k / my, q = k % my;
            double s = 0.0;
            for (int a = 0; a < mx; ++a) s += Sx[p * mx + a] * B[a * my + q];
            T1[k] = s;
        }
        __syncthreads();
        const double scale = 4.0 / ((mx + 1.0) * (my + 1.0));
        for (int c = threadIdx.x; c < n; c += blockDim.x) {
            const int i = c / ny, j = c % ny;
            if (i == 0 || j == 0 || i == nx - 1 || j == ny - 1) {
                du[c] = 0.0;
            } else {
                const int p = i - 1, q = j - 1;
                double s = 0.0;
                for (int a = 0; a < my; ++a) s += T1[p * my + a] * Sy[a * my + q];
                du[c] = s * scale - m[(long)c * 5];
            }
        }
    }
    __syncthreads();
    // moments of h^(k+1) and flow rates
    const double* trap = coef + jb.trap_off;
    double s[2] = {0.0, 0.0};
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
        const double u = m[c * 5 + 0] + 2.0 * du[c] * cU;
        const double q = m[c * 5 + 1] + 2.0 * du[c] * cq;
        U3[c0 + c] = u;
        s[0] += trap[c] * u;
        s[1] += trap[c] * q;
    }
    block_reduce<2>(s, red);
    if (threadIdx.x == 0) {
        const double Mn = s[0], Qn = s[1];
        const double rm = fabs(Mn - st->M) / fabs(Mn), rq = fabs(Qn - st->Q) / fabs(Qn);
        st->Mprev = st->M;
        st->Qprev = st->Q;
        st->M = Mn;
        st->Q = Qn;
        st->iters += 1;
        st->rel = fmax(rm, rq);
        if (!isfinite(Mn) || !isfinite(Qn)) {
            st->nan = 1;
            st->done = 1;
        } else if (jb.crit == 0 ? (fabs(Mn - st->Mprev) < jb.eps * fabs(Mn) && fabs(Qn - st->Qprev) < jb.eps * fabs(Qn))
                                : (fmax(fabs(Mn - st->Mprev), fabs(Qn - st->Qprev)) < jb.eps * fmax(fabs(Mn), fabs(Qn)))) {
            st->done = 1;
        } else if (st->iters >= jb.max_iter) {
            st->done = 1;
        }
    }
}

// h = P(hh + extra) + 2 dU v3 f_eq for the cells of the active jobs (Eq. guided), where P
// projects onto the parity group of the solution: plates odd in v3 and even in v2, ducts odd
// in v3 (the sources X_P v3 f_eq and X_T (c^2 - 5/2) v3 f_eq have it, and transport and the
// collision operator preserve it).  The exact iterates never leave that subspace, but
// rounding does (the FFT of the loss term is not mirror-exact), and outside it sits the
// density mode, which the diffusion correction does not accelerate and which the discrete
// operator, conserving mass only to quadrature accuracy, leaves at |lambda| ~ 1 for large
// delta: seeded at FP32 rounding it would never decay.  One thread per orbit, so the
// projection moves no extra bytes.  quarter: plates in the orbit layout (one value per orbit,
// at the orbit's index), where the projection is the identity.  hh = NULL: only hm, of the h
// already stored (a solve resumed from a checkpoint), with the same arithmetic.
template <typename T>
__global__ void __launch_bounds__(256) k_correct(const T* __restrict__ hh, T* __restrict__ h,
                                                 const double* __restrict__ dU, const T* __restrict__ extra,
                                                 const T* __restrict__ feq,
                                                 const T* __restrict__ vel, const SweepJobDev* __restrict__ jobs,
                                                 const int* __restrict__ active, int nv,
                                                 const JobState* __restrict__ state, double* __restrict__ hm,
                                                 const double* __restrict__ nd, const T* __restrict__ nu1,
                                                 double dv3, int quarter) {
    __shared__ dfloat redx[32 * 2];
    const int jid = active ? active[blockIdx.y] : blockIdx.y;
    if (state && state[jid].skip) return;  // finished before this iteration
    const SweepJobDev jb = jobs[jid];
    const int n3 = nv * nv * nv, hv = nv / 2;
    const bool plates = jb.ny == 0;  // 1D: orbits {1, R2, R3, R2R3}; 2D: {1, R3}
    // quarter: bit 0 plates in the orbit layout (handled here), bit 1 plates done by k_correct_q
    // (skipped here), bit 2 ducts in the orbit layout (one value per orbit {1, R3}, at index r)
    if (plates && (quarter & 2)) return;
    const bool dhalf = !plates && (quarter & 4);
    const int norb = plates ? n3 / 4 : n3 / 2;
    const bool only_hm = hh == nullptr;  // hm of the stored h alone (a resumed solve); h unchanged
    for (int c = blockIdx.x; c < jb.ncell; c += gridDim.x) {
        const long g0 = (jb.cell_off + c) * (long)n3;
        const T d = only_hm ? T(0) : (T)(2.0 * dU[jb.cell_off + c]);
        const T* src = only_hm ? nullptr : hh + g0;
        T* dst = h + g0;
        const T* ex = extra ? extra + g0 : nullptr;
        const float ndc = hm ? (float)nd[jb.cell_off + c] : 0.f, dl = (float)jb.delta;
        float a0 = 0.f, c0 = 0.f, a1 = 0.f, c1 = 0.f;  // compensated sums of the two moments
        auto kahan = [](float& sum, float& comp, float x) {
            const float y = x - comp;
            const float t = sum + y;
            comp = (t - sum) - y;
            sum = t;
        };
        // the h part of the L-moments at the orbit of (i1, i2, i3) (plates) or (i1, i2, i3) and
        // its R3 image (ducts), y the value at the representative
        auto add_hm = [&](int i1, int i2, int i3, T y) {
            const int va = (i1 * nv + i2) * nv + i3, vc = (i1 * nv + i2) * nv + nv - 1 - i3;
            if (plates) {  // v3 h is the same at the four points; v2 flips sign under R2
                const int vb = (i1 * nv + nv - 1 - i2) * nv + i3, vd = (i1 * nv + nv - 1 - i2) * nv + nv - 1 - i3;
                const float wa = ndc - dl * (float)nu1[va], wb = ndc - dl * (float)nu1[vb];
                const float wc = ndc - dl * (float)nu1[vc], wd = ndc - dl * (float)nu1[vd];
                const float t = (float)vel[i3] * (float)y;
                kahan(a0, c0, (float)vel[i1] * t * ((wa + wb) + (wc + wd)));
                kahan(a1, c1, (float)vel[i2] * t * ((wa - wb) + (wc - wd)));
            } else {
                const float w = (ndc - dl * (float)nu1[va]) + (ndc - dl * (float)nu1[vc]);
                const float t = (float)vel[i3] * (float)y * w;
                kahan(a0, c0, (float)vel[i1] * t);
                kahan(a1, c1, (float)vel[i2] * t);
            }
        };
        if (plates && (quarter & 1)) {
            // orbit layout: the orbit's one stored value sits at index r.  Four orbits per
            // thread and pass, their loads issued together (the same order of sums as one at
            // a time).
            const int bd = blockDim.x;
            for (int r0 = threadIdx.x; r0 < norb; r0 += 4 * bd) {
                T x[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int r = r0 + k * bd;
                    x[k] = r < norb ? (only_hm ? dst[r] : src[r]) : T(0);
                }
                if (ex && !only_hm)
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const int r = r0 + k * bd;
                        if (r < norb) x[k] += ex[r];
                    }
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int r = r0 + k * bd;
                    if (r >= norb) break;
                    const int i3 = r % hv, i2 = (r / hv) % hv, i1 = r / (hv * hv);
                    T y = x[k];
                    if (!only_hm) {
                        y = x[k] + d * vel[i3] * feq[(i1 * nv + i2) * nv + i3];
                        dst[r] = y;
                    }
                    if (hm) add_hm(i1, i2, i3, y);
                }
            }
        } else {
            for (int r = threadIdx.x; r < norb; r += blockDim.x) {
                const int i3 = r % hv;
                int i1, i2;
                if (plates) {
                    i2 = (r / hv) % hv;
                    i1 = r / (hv * hv);
                } else {
                    i2 = (r / hv) % nv;
                    i1 = r / (hv * nv);
                }
                const int va = (i1 * nv + i2) * nv + i3;                    // v3 < 0 half
                const int vc = (i1 * nv + i2) * nv + nv - 1 - i3;           // R3
                const int vb = (i1 * nv + nv - 1 - i2) * nv + i3;           // R2 (plates)
                const int vd = (i1 * nv + nv - 1 - i2) * nv + nv - 1 - i3;  // R2 R3 (plates)
                T y;
                if (dhalf) {  // the orbit's one stored value at index r
                    y = only_hm ? dst[r] : (ex ? src[r] + ex[r] : src[r]) + d * vel[i3] * feq[va];
                    if (!only_hm) dst[r] = y;
                } else if (only_hm) {
                    y = dst[va];
                } else {
                    T xa = src[va], xc = src[vc];
                    if (ex) {
                        xa += ex[va];
                        xc += ex[vc];
                    }
                    if (plates) {
                        T xb = src[vb], xd = src[vd];
                        if (ex) {
                            xb += ex[vb];
                            xd += ex[vd];
                        }
                        y = (T)0.25 * ((xa + xb) - (xc + xd)) + d * vel[i3] * feq[va];
                        dst[va] = y;
                        dst[vb] = y;
                        dst[vc] = -y;
                        dst[vd] = -y;
                    } else {
                        y = (T)0.5 * (xa - xc) + d * vel[i3] * feq[va];
                        dst[va] = y;
                        dst[vc] = -y;
                    }
                }
                if (hm) add_hm(i1, i2, i3, y);
            }
        }
        if (hm) {
            dfloat sm[2] = {df_fast2sum(a0, -c0), df_fast2sum(a1, -c1)};
            block_reduce_df<2>(sm, redx);
            if (threadIdx.x == 0) {
                hm[2 * (jb.cell_off + c) + 0] = 2.0 * (double)sm[0] * dv3;
                hm[2 * (jb.cell_off + c) + 1] = 2.0 * (double)sm[1] * dv3;
            }
        }
    }
}

// The correction step for plates in the orbit layout (float): the orbit's one stored value at
// index r, y = hh + extra + 2 dU v3 f_eq, and the h part of the L-moments from the orbit
// constants orb = {v3 f_eq, v1 v3, sum of nu_eq over the orbit}: the orbit's four points carry
// v1 v3 y (N delta - delta nu) each, so Gh_1 = 2 sum_orbits v1 v3 y (4 N delta - delta sum nu)
// dv^3; Gh_2 = 0 (odd under R2).  hh = NULL: only hm, of the stored h (a resumed solve).  Grid
// sizes are compile-time constants; four orbits per thread and pass with their loads issued
// together.
template <int NV>
__global__ void __launch_bounds__(256) k_correct_q(const float* __restrict__ hh, float* __restrict__ h,
                                                   const double* __restrict__ dU, const float* __restrict__ extra,
                                                   const float4* __restrict__ orb,
                                                   const SweepJobDev* __restrict__ jobs,
                                                   const int* __restrict__ active,
                                                   const JobState* __restrict__ state, double* __restrict__ hm,
                                                   const double* __restrict__ nd, double dv3) {
    constexpr int H = NV / 2, NQ = NV * H * H;
    constexpr long n3 = (long)NV * NV * NV;
    __shared__ dfloat redx[32 * 2];
    const int jid = active ? active[blockIdx.y] : blockIdx.y;
    if (state && state[jid].skip) return;
    const SweepJobDev jb = jobs[jid];
    if (jb.ny != 0) return;  // plates only
    const bool only_hm = hh == nullptr;
    for (int c = blockIdx.x; c < jb.ncell; c += gridDim.x) {
        const long g0 = (jb.cell_off + c) * n3;
        const float d = only_hm ? 0.f : (float)(2.0 * dU[jb.cell_off + c]);
        const float* src = only_hm ? nullptr : hh + g0;
        float* dst = h + g0;
        const float* ex = extra ? extra + g0 : nullptr;
        const float ndc4 = hm ? 4.f * (float)nd[jb.cell_off + c] : 0.f, dl = (float)jb.delta;
        float a0 = 0.f, c0 = 0.f;
        for (int r0 = threadIdx.x; r0 < NQ; r0 += 4 * 256) {
            float x[4];
            float4 o[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int r = r0 + k * 256;
                if (r < NQ) {
                    x[k] = only_hm ? dst[r] : src[r];
                    o[k] = orb[r];
                }
            }
            if (ex && !only_hm)
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int r = r0 + k * 256;
                    if (r < NQ) x[k] += ex[r];
                }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int r = r0 + k * 256;
                if (r >= NQ) break;
                float y = x[k];
                if (!only_hm) {
                    y = x[k] + d * o[k].x;
                    dst[r] = y;
                }
                if (hm) {
                    const float v = o[k].y * y * (ndc4 - dl * o[k].z) - c0;
                    const float t = a0 + v;
                    c0 = (t - a0) - v;
                    a0 = t;
                }
            }
        }
        if (hm) {
            dfloat sm[2] = {df_fast2sum(a0, -c0), dfloat(0)};
            block_reduce_df<2>(sm, redx);
            if (threadIdx.x == 0) {
                hm[2 * (jb.cell_off + c) + 0] = 2.0 * (double)sm[0] * dv3;
                hm[2 * (jb.cell_off + c) + 1] = 0.0;
            }
        }
    }
}

}  // namespace

template <typename T>
static void sweep1d_sched(int sched, const DevTables& t, dim3 g, size_t smem_coef, size_t smem_full, int staged,
                          const T* rhs, T* h, const SweepJobDev* jobs, const int* active, const double* coef,
                          cudaStream_t s, int quarter) {
    const T* nu1 = sizeof(T) == 8 ? (const T*)t.nu1_d : (const T*)t.nu1_f;
    const T* vel = sizeof(T) == 8 ? (const T*)t.vel_d : (const T*)t.vel_f;
    const T* feq = sizeof(T) == 8 ? (const T*)t.feq_d : (const T*)t.feq_f;
    if (sched == 0)
        k_sweep1d<T, 0><<<g, 128, smem_full, s>>>(rhs, h, nu1, vel, feq, jobs, active, coef, t.nv, staged,
                                                   quarter);
    else if (sched == 3)
        k_sweep1d<T, 3><<<g, 128, smem_full, s>>>(rhs, h, nu1, vel, feq, jobs, active, coef, t.nv, staged,
                                                   quarter);
    else if (sched == 2)
        k_sweep1d<T, 2><<<g, 128, (smem_coef + 15) / 16 * 16 + 2 * 16 * 128 * sizeof(T) + 16, s>>>(
            rhs, h, nu1, vel, feq, jobs, active, coef, t.nv, staged, quarter);
    else
        k_sweep1d<T, 1><<<g, 128, smem_coef, s>>>(rhs, h, nu1, vel, feq, jobs, active, coef, t.nv, staged,
                                                   quarter);
}

template <typename T>
void launch_sweep(const DevTables& t, int dim, int njobs, int max_coef, const T* rhs, T* h,
                  const SweepJobDev* jobs, const int* active, const double* coef, cudaStream_t s, int quarter) {
    if (njobs <= 0) return;
    // float sweeps stage the coefficients when the largest job's fit in 48 KB
    // 1D: staged coefficients are a float4 per node and direction; 2D: the plain block
    const size_t sbytes = dim == 1 ? (size_t)(max_coef / 6) * 2 * sizeof(float4) : (size_t)max_coef * sizeof(T);
    const int staged = (sizeof(T) == 4 && max_coef > 0 && sbytes <= 48 * 1024) ? 1 : 0;
    const size_t smem = staged ? sbytes : 0;
    g_launches += 1;
    const int nv = t.nv;
    if (dim == 1) {
        const int W = quarter ? nv / 2 * (nv / 2) : nv * nv;  // velocities per i1 plane of the data
        const int nt = nv / 2 * W;
        dim3 g((nt + 127) / 128, njobs);
        // 1D float sweeps can also stage every right-hand side of their columns (schedule 0)
        // when that fits in 200 KB; which schedule is faster is measured at first use
        const size_t full = sbytes + 2 * (size_t)(max_coef / 6) * 128 * sizeof(T);
        int sched = 1;
        if (sizeof(T) == 4 && staged && full <= 200 * 1024 && t.tuning && (uintptr_t)rhs % 16 == 0) {
            static std::once_flag attr;  // opt-in shared memory beyond 48 KB (float instance)
            std::call_once(attr, [] {
                cudaFuncSetAttribute(k_sweep1d<T, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
                cudaFuncSetAttribute(k_sweep1d<T, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
            });
            int jb = 1;
            while (jb < njobs) jb *= 2;  // problems and nodes classes: the next power of two
            int nb = 1;
            while (nb < max_coef / 6) nb *= 2;
            const long long key = ((long long)quarter << 50) | ((long long)nv << 40) | ((long long)jb << 20) | nb;
            std::lock_guard<std::mutex> lk(t.tuning->mu);
            auto it = t.tuning->sweep.find(key);
            cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
            const bool capturing = cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone;
            if (it != t.tuning->sweep.end()) {
                sched = it->second;
            } else if (capturing) {
                sched = 0;
            } else {
                // every schedule twice, in turn; each writes the same h (same arithmetic).  The
                // bulk-copy ring and the row-staged schedule need whole 128-velocity rows per
                // block (W a multiple of 128).
                const int NS = W % 128 == 0 ? 4 : 2;
                if (t.tuning->side && t.tuning->side != s) cudaStreamSynchronize(t.tuning->side);
                cudaEvent_t ev[9];
                for (int k = 0; k <= 2 * NS; ++k) cudaEventCreate(&ev[k]);
                cudaEventRecord(ev[0], s);
                for (int k = 0; k < 2 * NS; ++k) {
                    sweep1d_sched<T>(k % NS, t, g, smem, full, staged, rhs, h, jobs, active, coef, s, quarter);
                    cudaEventRecord(ev[k + 1], s);
                }
                cudaEventSynchronize(ev[2 * NS]);
                float ms[8] = {};
                for (int k = 0; k < 2 * NS; ++k) cudaEventElapsedTime(&ms[k], ev[k], ev[k + 1]);
                for (int k = 0; k <= 2 * NS; ++k) cudaEventDestroy(ev[k]);
                float best[4] = {0.f, 0.f, 0.f, 0.f};
                for (int q = 0; q < NS; ++q) best[q] = std::min(ms[q], ms[q + NS]);
                sched = 0;
                for (int q = 1; q < NS; ++q)
                    if (best[q] < best[sched]) sched = q;
                t.tuning->sweep[key] = sched;
                static const char* names[4] = {"staged", "register ring", "bulk-copy ring", "row-staged"};
                char line[280];
                snprintf(line, sizeof line,
                         "sweep1d<float>%s nv=%d problems<=%d nodes<=%d: %s (staged %.1f us, register ring %.1f us, "
                         "bulk-copy ring %.1f us, row-staged %.1f us)",
                         quarter ? " orbit layout" : "", nv, jb, nb, names[sched], 1000.0f * best[0],
                         1000.0f * best[1], 1000.0f * best[2], 1000.0f * best[3]);
                t.tuning->log.push_back(line);
                g_launches += 2 * NS - 1;
                return;
            }
        }
        sweep1d_sched<T>(sched, t, g, smem, full, staged, rhs, h, jobs, active, coef, s, quarter);
    } else {
        const T* nu1 = sizeof(T) == 8 ? (const T*)t.nu1_d : (const T*)t.nu1_f;
        const T* vel = sizeof(T) == 8 ? (const T*)t.vel_d : (const T*)t.vel_f;
        const T* feq = sizeof(T) == 8 ? (const T*)t.feq_d : (const T*)t.feq_f;
        // the wavefront: blocks of 32 velocities x 16 rows; shared memory holds the
        // coefficients, the 3-step ring and the strip's last two rows
        constexpr int WR = 16;
        const int nt = quarter ? nv * nv * (nv / 2) : nv * nv * nv;  // ducts: quarter = the half layout
        const int mcx = max_coef / 3;  // largest nx + ny of the launch's jobs
        const size_t sm2 = (size_t)(3 * mcx + 3 * WR * 32 + 2 * mcx * 32) * sizeof(T);
        static std::once_flag attr;
        std::call_once(attr, [] {
            cudaFuncSetAttribute(k_sweep2d_wave<T, WR>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
        });
        if (sm2 <= 160 * 1024) {
            dim3 g((nt + 31) / 32, njobs);
            k_sweep2d_wave<T, WR><<<g, 32 * WR, sm2, s>>>(rhs, h, nu1, vel, feq, jobs, active, coef, nv, quarter);
        } else {
            dim3 g((nt + 127) / 128, njobs);
            k_sweep2d<T><<<g, 128, smem, s>>>(rhs, h, nu1, vel, feq, jobs, active, coef, nv, staged, quarter);
        }
    }
}

template <typename T>
void launch_moments(const DevTables& t, long cell0, int cells, const T* h, double* mom, cudaStream_t s,
                    int quarter) {
    if (cells <= 0) return;
    g_launches += 1;
    const T* vel = sizeof(T) == 8 ? (const T*)t.vel_d : (const T*)t.vel_f;
    const double dv3 = t.dv * t.dv * t.dv;
    if (quarter == 2) {  // ducts in the orbit layout (the half)
        switch (t.nv) {
            case 8: k_moments_h<T, 8><<<cells, 32, 0, s>>>(h, vel, dv3, cell0, mom); break;
            case 16: k_moments_h<T, 16><<<cells, 128, 0, s>>>(h, vel, dv3, cell0, mom); break;
            case 24: k_moments_h<T, 24><<<cells, 288, 0, s>>>(h, vel, dv3, cell0, mom); break;
            default: k_moments_h<T, 32><<<cells, 512, 0, s>>>(h, vel, dv3, cell0, mom); break;
        }
        return;
    }
    if (quarter) {
        switch (t.nv) {
            case 8: k_moments_q<T, 8><<<cells, 32, 0, s>>>(h, vel, dv3, cell0, mom); break;
            case 16: k_moments_q<T, 16><<<cells, 64, 0, s>>>(h, vel, dv3, cell0, mom); break;
            case 24: k_moments_q<T, 24><<<cells, 160, 0, s>>>(h, vel, dv3, cell0, mom); break;
            default: k_moments_q<T, 32><<<cells, 256, 0, s>>>(h, vel, dv3, cell0, mom); break;
        }
        return;
    }
    switch (t.nv) {
        case 8: k_moments<T, 8><<<cells, 64, 0, s>>>(h, vel, dv3, cell0, mom); break;
        case 16: k_moments<T, 16><<<cells, 128, 0, s>>>(h, vel, dv3, cell0, mom); break;
        case 24: k_moments<T, 24><<<cells, 192, 0, s>>>(h, vel, dv3, cell0, mom); break;
        default: k_moments<T, 32><<<cells, 256, 0, s>>>(h, vel, dv3, cell0, mom); break;
    }
}

void launch_sis_update(const DevTables& t, int njobs, const SisJobDev* jobs, const int* active,
                       const double* mom, const double* G, const double* coef, double* work, double* dU,
                       double* U3, JobState* state, cudaStream_t s) {
    if (njobs <= 0) return;
    g_launches += 1;
    k_sis_update<<<njobs, 256, 0, s>>>(jobs, active, mom, G, coef, work, t.cU, t.cq, dU, U3, state);
}

template <typename T>
void launch_correct(const DevTables& t, int njobs, const T* hh, T* h, const double* dU, const T* extra,
                    const SweepJobDev* jobs, const int* active, cudaStream_t s, const JobState* state, double* hm,
                    const double* nd, int quarter, int max_cells, int ducts) {
    if (njobs <= 0) return;
    g_launches += 1;
    const T* feq = sizeof(T) == 8 ? (const T*)t.feq_d : (const T*)t.feq_f;
    const T* vel = sizeof(T) == 8 ? (const T*)t.vel_d : (const T*)t.vel_f;
    // one block per cell of the largest job (max_cells > 0), or a grid-stride loop over cells
    dim3 g(max_cells > 0 ? max_cells : 2 * sm_count(), njobs);
    const T* nu1 = sizeof(T) == 8 ? (const T*)t.nu1_d : (const T*)t.nu1_f;
    const double dv3 = t.dv * t.dv * t.dv;
    if (sizeof(T) == 4 && quarter) {  // plates by the orbit kernel, then any ducts
        const float* hf = (const float*)hh;
        float* h_ = (float*)h;
        const float* ef = (const float*)extra;
        switch (t.nv) {
            case 8: k_correct_q<8><<<g, 256, 0, s>>>(hf, h_, dU, ef, t.orb_f, jobs, active, state, hm, nd, dv3); break;
            case 16: k_correct_q<16><<<g, 256, 0, s>>>(hf, h_, dU, ef, t.orb_f, jobs, active, state, hm, nd, dv3); break;
            case 24: k_correct_q<24><<<g, 256, 0, s>>>(hf, h_, dU, ef, t.orb_f, jobs, active, state, hm, nd, dv3); break;
            default: k_correct_q<32><<<g, 256, 0, s>>>(hf, h_, dU, ef, t.orb_f, jobs, active, state, hm, nd, dv3); break;
        }
        if (!ducts) return;
        g_launches += 1;
        k_correct<T><<<g, 256, 0, s>>>(hh, h, dU, extra, feq, vel, jobs, active, t.nv, state, hm, nd, nu1, dv3, 2 | 4);
        return;
    }
    k_correct<T><<<g, 256, 0, s>>>(hh, h, dU, extra, feq, vel, jobs, active, t.nv, state, hm, nd, nu1, dv3,
                                   quarter ? 1 | 4 : 0);
}

template void launch_sweep<double>(const DevTables&, int, int, int, const double*, double*,
                                   const SweepJobDev*, const int*, const double*, cudaStream_t, int);
template void launch_sweep<float>(const DevTables&, int, int, int, const float*, float*,
                                  const SweepJobDev*, const int*, const double*, cudaStream_t, int);
template void launch_moments<double>(const DevTables&, long, int, const double*, double*, cudaStream_t, int);
template void launch_moments<float>(const DevTables&, long, int, const float*, double*, cudaStream_t, int);
template void launch_correct<double>(const DevTables&, int, const double*, double*, const double*,
                                     const double*, const SweepJobDev*, const int*, cudaStream_t, const JobState*,
                                     double*, const double*, int, int, int);
template void launch_correct<float>(const DevTables&, int, const float*, float*, const double*, const float*,
                                    const SweepJobDev*, const int*, cudaStream_t, const JobState*, double*,
                                    const double*, int, int, int);

}  // namespace lbe

// Mixed-precision SIS: FP64 residuals, low-precision correction solves (defect correction).
//
// One FP64 SIS iteration is the affine map Phi(h) = A h + b (Sec. 2.2: sweep of Eq.
// syn_LBE, diffusion correction Eq. first_order / diffusion_LBE, Eq. guided); its fixed
// point is the FP64 SIS solution.  The driver repeats
//     r = Phi_64(h) - h                          (one FP64 iteration; also the stopping test:
//                                                 the flow rates of h and Phi_64(h) differ by
//                                                 less than eps, exactly the FP64 criterion)
//     solve (I - A) e = r approximately by e <- A_lo e + r   (low-precision SIS iterations
//                                                 of the homogeneous map: no source S and no
//                                                 momentum-balance term)
//     h <- h + e
// starting from h = the low-precision SIS solution of the full problem, so that a solve
// usually needs two FP64 iterations: one residual and one that certifies convergence.
// The answer is the FP64 SIS fixed point, while almost all collision-operator evaluations
// run in low precision.  h lives in FP64; e and r in FP32.  The FP64-class operator
// evaluations (at the base point h0 and when it is re-centred) run in double-float
// arithmetic (pairs of floats, ~2^-44 relative), which this GPU issues far faster than FP64.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "batch.h"
#include "lbe_internal.h"
#include "sweep.h"

namespace lbe {

namespace {

// Orbit layout (sweep.h; dim 1 plates, 2 ducts) index of the full-grid point f of a cell, and
// whether the point is the R3 image (negated); and the full-grid index of the representative
// of orbit q.
__device__ __forceinline__ long orbit_of(long f, int nv, int dim, bool* neg) {
    const int H = nv / 2;
    const int i3 = (int)(f % nv), i2 = (int)((f / nv) % nv), i1 = (int)(f / ((long)nv * nv));
    *neg = i3 >= H;
    const int j3 = i3 < H ? i3 : nv - 1 - i3;
    if (dim == 2) return ((long)i1 * nv + i2) * H + j3;
    const int j2 = i2 < H ? i2 : nv - 1 - i2;
    return ((long)i1 * H + j2) * H + j3;
}
__device__ __forceinline__ long full_of(long q, int nv, int dim) {
    const int H = nv / 2;
    const int R2 = dim == 2 ? nv : H;  // i2 values of the layout
    const int j3 = (int)(q % H), j2 = (int)((q / H) % R2), i1 = (int)(q / ((long)R2 * H));
    return ((long)i1 * nv + j2) * nv + j3;
}
__host__ __device__ inline long orbit_values(long n3, int dim) { return dim == 2 ? n3 / 2 : n3 / 4; }

}  // namespace

// The element-wise steps between the FP64 iterate (full grid) and the FP32 correction of a range
// of cells (orbit layout: the service's buckets).
__global__ void k_range_widen_q(const float* __restrict__ e, double* __restrict__ h, long cells, int nv, int dim) {
    const long n3 = (long)nv * nv * nv, n = cells * n3;
    for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < n; k += (long)gridDim.x * blockDim.x) {
        const long f = k % n3;
        bool neg;
        const double v = (double)e[k - f + orbit_of(f, nv, dim, &neg)];
        h[k] = neg ? -v : v;
    }
}
__global__ void k_range_correct_q(const double* __restrict__ h_old, const float* __restrict__ e,
                                  double* __restrict__ h, long cells, int nv, int dim) {
    const long n3 = (long)nv * nv * nv, n = cells * n3;
    for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < n; k += (long)gridDim.x * blockDim.x) {
        const long f = k % n3;
        bool neg;
        const double v = (double)e[k - f + orbit_of(f, nv, dim, &neg)];
        h[k] = h_old[k] + (neg ? -v : v);
    }
}
__global__ void k_range_residual_q(const double* __restrict__ h, const double* __restrict__ h_old,
                                   float* __restrict__ r, long cells, int nv, int dim) {
    const long n3 = (long)nv * nv * nv, nq = orbit_values(n3, dim), n = cells * nq;
    for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < n; k += (long)gridDim.x * blockDim.x) {
        const long c = k / nq, q = k % nq, f = c * n3 + full_of(q, nv, dim);
        r[c * n3 + q] = (float)(h[f] - h_old[f]);
    }
}
void range_widen_q(const float* e, double* h, long cells, int nv, int dim, cudaStream_t s) {
    g_launches += 1;
    k_range_widen_q<<<sm_count(), 256, 0, s>>>(e, h, cells, nv, dim);
}
void range_correct_q(const double* h_old, const float* e, double* h, long cells, int nv, int dim, cudaStream_t s) {
    g_launches += 1;
    k_range_correct_q<<<sm_count(), 256, 0, s>>>(h_old, e, h, cells, nv, dim);
}
void range_residual_q(const double* h, const double* h_old, float* r, long cells, int nv, int dim, cudaStream_t s) {
    g_launches += 1;
    k_range_residual_q<<<sm_count(), 256, 0, s>>>(h, h_old, r, cells, nv, dim);
}

__global__ void k_range_sub_f32_q(const double* __restrict__ h, const double* __restrict__ b, float* __restrict__ o,
                                  long cells, long n3, long nq) {
    const long n = cells * nq;
    for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < n; k += (long)gridDim.x * blockDim.x) {
        const long i = (k / nq) * n3 + k % nq;
        o[i] = (float)(h[i] - b[i]);
    }
}
__global__ void k_range_add_f64_q(const double* __restrict__ b, const float* __restrict__ inc,
                                  double* __restrict__ o, long cells, long n3, long nq) {
    const long n = cells * nq;
    for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < n; k += (long)gridDim.x * blockDim.x) {
        const long i = (k / nq) * n3 + k % nq;
        o[i] = b[i] + (double)inc[i];
    }
}
__global__ void k_range_copy_q(const double* __restrict__ a, double* __restrict__ b, long cells, long n3, long nq) {
    const long n = cells * nq;
    for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < n; k += (long)gridDim.x * blockDim.x) {
        const long i = (k / nq) * n3 + k % nq;
        b[i] = a[i];
    }
}
__global__ void k_orbit_unpack(const double* __restrict__ q, double* __restrict__ full, long cells, int nv, int dim) {
    const long n3 = (long)nv * nv * nv, n = cells * n3;
    for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < n; k += (long)gridDim.x * blockDim.x) {
        const long f = k % n3;
        bool neg;
        const double v = q[k - f + orbit_of(f, nv, dim, &neg)];
        full[k] = neg ? -v : v;
    }
}
__global__ void k_orbit_pack(const double* __restrict__ full, double* __restrict__ q, long cells, int nv, int dim) {
    const long n3 = (long)nv * nv * nv, nq = orbit_values(n3, dim), n = cells * nq;
    for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < n; k += (long)gridDim.x * blockDim.x) {
        const long c = k / nq, r = k % nq;
        q[c * n3 + r] = full[c * n3 + full_of(r, nv, dim)];
    }
}
void range_sub_f32_q(const double* h, const double* base, float* out, long cells, long n3, long nq, cudaStream_t s) {
    g_launches += 1;
    k_range_sub_f32_q<<<2 * sm_count(), 256, 0, s>>>(h, base, out, cells, n3, nq);
}
void range_add_f64_q(const double* base, const float* inc, double* out, long cells, long n3, long nq,
                     cudaStream_t s) {
    g_launches += 1;
    k_range_add_f64_q<<<2 * sm_count(), 256, 0, s>>>(base, inc, out, cells, n3, nq);
}
void range_copy_q(const double* a, double* b, long cells, long n3, long nq, cudaStream_t s) {
    g_launches += 1;
    k_range_copy_q<<<2 * sm_count(), 256, 0, s>>>(a, b, cells, n3, nq);
}
void orbit_unpack_dev(const double* q, double* full, long cells, int nv, int dim, cudaStream_t s) {
    g_launches += 1;
    k_orbit_unpack<<<2 * sm_count(), 256, 0, s>>>(q, full, cells, nv, dim);
}
void orbit_pack_dev(const double* full, double* q, long cells, int nv, int dim, cudaStream_t s) {
    g_launches += 1;
    k_orbit_pack<<<2 * sm_count(), 256, 0, s>>>(full, q, cells, nv, dim);
}

namespace {

// The per-job element-wise steps below run over the values a job's cells hold: all nv^3 of a
// cell, or with quarter the orbit-layout prefix (nv^3 / 4) of a plate's cells (sweep.h), where
// both sides of the step are in that layout.
__device__ __forceinline__ long job_values(const SweepJobDev& jb, long n3, int quarter) {
    return quarter ? (jb.ny == 0 ? n3 / 4 : n3 / 2) : n3;
}

// dst = src over the cells of the active jobs
__global__ void k_copy64(const double* __restrict__ src, double* __restrict__ dst,
                         const SweepJobDev* __restrict__ jobs, const int* __restrict__ active, long n3,
                         int quarter) {
    const SweepJobDev jb = jobs[active[blockIdx.y]];
    const long nq = job_values(jb, n3, quarter), total = (long)jb.ncell * nq, base = jb.cell_off * n3;
    for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < total; k += (long)gridDim.x * blockDim.x) {
        const long i = base + (k / nq) * n3 + k % nq;
        dst[i] = src[i];
    }
}

// r = (float)(h - h_old)
__global__ void k_residual(const double* __restrict__ h, const double* __restrict__ h_old, float* __restrict__ r,
                           const SweepJobDev* __restrict__ jobs, const int* __restrict__ active, long n3,
                           int quarter) {
    const SweepJobDev jb = jobs[active[blockIdx.y]];
    const long nq = job_values(jb, n3, quarter), total = (long)jb.ncell * nq, base = jb.cell_off * n3;
    for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < total; k += (long)gridDim.x * blockDim.x) {
        const long i = base + (k / nq) * n3 + k % nq;
        r[i] = (float)(h[i] - h_old[i]);
    }
}

// h = h_old + e
__global__ void k_apply_correction(const double* __restrict__ h_old, const float* __restrict__ e,
                                   double* __restrict__ h, const SweepJobDev* __restrict__ jobs,
                                   const int* __restrict__ active, long n3, int quarter) {
    const SweepJobDev jb = jobs[active[blockIdx.y]];
    const long nq = job_values(jb, n3, quarter), total = (long)jb.ncell * nq, base = jb.cell_off * n3;
    for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < total; k += (long)gridDim.x * blockDim.x) {
        const long i = base + (k / nq) * n3 + k % nq;
        h[i] = h_old[i] + (double)e[i];
    }
}

// h = (double)e
__global__ void k_widen(const float* __restrict__ e, double* __restrict__ h, const SweepJobDev* __restrict__ jobs,
                        const int* __restrict__ active, long n3, int quarter) {
    const SweepJobDev jb = jobs[active[blockIdx.y]];
    const long nq = job_values(jb, n3, quarter), total = (long)jb.ncell * nq, base = jb.cell_off * n3;
    for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < total; k += (long)gridDim.x * blockDim.x) {
        const long i = base + (k / nq) * n3 + k % nq;
        h[i] = (double)e[i];
    }
}

// state M, Q := flow rates of the moments in mom (so the next iteration measures its change
// against the current iterate)
__global__ void k_set_rates(const SisJobDev* __restrict__ jobs, const int* __restrict__ active,
                            const double* __restrict__ mom, const double* __restrict__ coef,
                            JobState* __restrict__ state) {
    const int jid = active[blockIdx.x];
    const SisJobDev jb = jobs[jid];
    if (threadIdx.x != 0) return;
    const double* m = mom + jb.cell_off * 5;
    const double* w = coef + jb.trap_off;
    double M = 0.0, Q = 0.0;
    for (int c = 0; c < jb.ncell; ++c) {
        M += w[c] * m[c * 5 + 0];
        Q += w[c] * m[c * 5 + 1];
    }
    state[jid].M = M;
    state[jid].Q = Q;
}

}  // namespace

void launch_set_rates(int njobs, const SisJobDev* jobs, const int* active, const double* mom, const double* coef,
                      JobState* state, cudaStream_t s) {
    g_launches += 1;
    k_set_rates<<<njobs, 32, 0, s>>>(jobs, active, mom, coef, state);
}

// Element-wise range kernels of the defect-correction steps (one range of cells).
__global__ void k_range_widen(const float* __restrict__ e, double* __restrict__ h, long n) {
    for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < n; k += (long)gridDim.x * blockDim.x)
        h[k] = (double)e[k];
}
__global__ void k_range_copy(const double* __restrict__ a, double* __restrict__ b, long n) {
    for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < n; k += (long)gridDim.x * blockDim.x) b[k] = a[k];
}
__global__ void k_range_residual(const double* __restrict__ h, const double* __restrict__ h_old, float* __restrict__ r,
                                 long n) {
    for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < n; k += (long)gridDim.x * blockDim.x)
        r[k] = (float)(h[k] - h_old[k]);
}
__global__ void k_range_correct(const double* __restrict__ h_old, const float* __restrict__ e, double* __restrict__ h,
                                long n) {
    for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < n; k += (long)gridDim.x * blockDim.x)
        h[k] = h_old[k] + (double)e[k];
}

__global__ void k_range_sub_f32(const double* __restrict__ h, const double* __restrict__ b, float* __restrict__ o,
                                long n) {
    for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < n; k += (long)gridDim.x * blockDim.x)
        o[k] = (float)(h[k] - b[k]);
}
__global__ void k_range_add_f64(const double* __restrict__ b, const float* __restrict__ inc, double* __restrict__ o,
                                long n) {
    for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < n; k += (long)gridDim.x * blockDim.x)
        o[k] = b[k] + (double)inc[k];
}
void range_sub_f32(const double* h, const double* base, float* out, long n, cudaStream_t s) {
    g_launches += 1;
    k_range_sub_f32<<<2 * sm_count(), 256, 0, s>>>(h, base, out, n);
}
void range_add_f64(const double* base, const float* inc, double* out, long n, cudaStream_t s) {
    g_launches += 1;
    k_range_add_f64<<<2 * sm_count(), 256, 0, s>>>(base, inc, out, n);
}

void range_widen(const float* e, double* h, long n, cudaStream_t s) {
    g_launches += 1;
    k_range_widen<<<sm_count(), 256, 0, s>>>(e, h, n);
}
void range_copy(const double* a, double* b, long n, cudaStream_t s) {
    g_launches += 1;
    k_range_copy<<<sm_count(), 256, 0, s>>>(a, b, n);
}
void range_residual(const double* h, const double* h_old, float* r, long n, cudaStream_t s) {
    g_launches += 1;
    k_range_residual<<<sm_count(), 256, 0, s>>>(h, h_old, r, n);
}
void range_correct(const double* h_old, const float* e, double* h, long n, cudaStream_t s) {
    g_launches += 1;
    k_range_correct<<<sm_count(), 256, 0, s>>>(h_old, e, h, n);
}

lbe_status refined_solve(Ctx* c, const lbe_problem* pbs, int n, lbe_result* outs, double* U3_out,
                         double* h_out) {
    auto t0 = std::chrono::steady_clock::now();
    cudaStream_t s = c->stream;
    std::vector<lbe_problem> po(pbs, pbs + n), pi(pbs, pbs + n);
    int max_outer = 1;
    for (int j = 0; j < n; ++j) {
        po[j].precision = LBE_FP64;
        pi[j].precision = LBE_FP32;  // phase 0: the full problem in low precision
        pi[j].eps = std::max(pbs[j].eps, 1e-5);
        pi[j].max_iter = 150;
        max_outer = std::max(max_outer, pbs[j].max_iter);
    }
    // the context's grow-only arenas: a warm context allocates nothing per solve
    Arena& ao = c->refine_arena[0];
    Arena& ai = c->refine_arena[1];
    Batch O, I;
    lbe_status st = batch_init(O, c, po.data(), n, &ao, s);
    if (st == LBE_OK) st = batch_init(I, c, pi.data(), n, &ai, s);
    if (st == LBE_OK) {  // low-precision phases test changes against the flow-rate scale
        I.use_tc = pbs[0].precision == LBE_BF16_REFINED && O.t->sym_reps2 > 0 && pbs[0].M >= 8;
        // BF16-refined: plates in the orbit layout on both sides (sweep.h)
        I.orbit = O.orbit = I.use_tc;
        for (int j = 0; j < n; ++j) I.ij[j].crit = 1;
        cudaMemcpyAsync(I.ijobs.p, I.ij.data(), n * sizeof(SisJobDev), cudaMemcpyHostToDevice, s);
    }
    const bool q = I.orbit;
    const int nv = pbs[0].nv;
    const long n3 = (long)nv * nv * nv;
    const size_t vol64 = O.cells * n3 * 8, vol32 = O.cells * n3 * 4;
    int inc_chunk = 1;
    const size_t inc_scr = st == LBE_OK ? fsm_cc_scratch_bytes(*O.t, (int)O.cells, 4, &inc_chunk) : 0;
    // h_old, r, base_h, base_lp, base_lh (the double-float operator's full-grid input and
    // outputs), with q their copies in the batch's layout, inc_h, inc_lp, inc_lh, FP32
    // operator scratch
    Arena& aw = c->refine_arena[2];
    double *h_old = nullptr, *base_h = nullptr, *base_lp = nullptr, *base_lh = nullptr;
    double *bq_h = nullptr, *bq_lp = nullptr, *bq_lh = nullptr;
    float *r = nullptr, *inc_h = nullptr, *inc_lp = nullptr, *inc_lh = nullptr;
    void* inc_scratch = nullptr;
    if (st == LBE_OK) {
        const size_t pad = 256;
        st = arena_reserve(c, aw, (q ? 7 : 4) * (vol64 + pad) + 4 * (vol32 + pad) + inc_scr + n * sizeof(int) + 2 * pad);
    }
    int* ident = nullptr;  // device [n]: ident[j] = j (one-problem launches of the per-job kernels)
    if (st == LBE_OK) {
        h_old = (double*)arena_take(aw, vol64);
        base_h = (double*)arena_take(aw, vol64);
        base_lp = (double*)arena_take(aw, vol64);
        base_lh = (double*)arena_take(aw, vol64);
        if (q) {
            bq_h = (double*)arena_take(aw, vol64);
            bq_lp = (double*)arena_take(aw, vol64);
            bq_lh = (double*)arena_take(aw, vol64);
        } else {
            bq_h = base_h;
            bq_lp = base_lp;
            bq_lh = base_lh;
        }
        r = (float*)arena_take(aw, vol32);
        inc_h = (float*)arena_take(aw, vol32);
        inc_lp = (float*)arena_take(aw, vol32);
        inc_lh = (float*)arena_take(aw, vol32);
        inc_scratch = arena_take(aw, inc_scr);
        ident = (int*)arena_take(aw, n * sizeof(int));
        if (!inc_scratch || !ident) st = LBE_INTERNAL;
    }
    if (st != LBE_OK) return st;
    {
        std::vector<int> id(n);
        for (int j = 0; j < n; ++j) id[j] = j;
        cudaMemcpyAsync(ident, id.data(), n * sizeof(int), cudaMemcpyHostToDevice, s);
        st = cuda_status(c, cudaStreamSynchronize(s), "refine set-up");
        if (st != LBE_OK) return st;
    }
    // The FP64-class operator of the current iterate of problems j0 .. j1 - 1 (consecutive, one
    // geometry, contiguous cells) becomes their base: h0 = h, base_lp / base_lh = L+ h0 / L h0 in
    // double-float arithmetic on the full grid, kept in the batch's layout.
    auto evaluate_base = [&](int j0, int j1, cudaStream_t s) {
        long cells = 0;
        for (int j = j0; j < j1; ++j) cells += O.sj[j].ncell;
        const long o = O.cell_off[j0] * n3;
        const int dim = O.geo[j0].dim;
        const double* h = O.h.as<double>() + o;
        if (q)
            orbit_unpack_dev(h, base_h + o, cells, nv, dim, s);
        else
            range_copy(h, base_h + o, cells * n3, s);
        fsm_df_apply(*O.t, (int)cells, O.delta.as<double>() + O.cell_off[j0], base_h + o, base_lp + o, base_lh + o,
                     O.scratch.p, O.chunk, s, dim == 1 ? 2 : 1);
        if (!q) return;
        range_copy_q(h, bq_h + o, cells, n3, dim == 1 ? n3 / 4 : n3 / 2, s);
        orbit_pack_dev(base_lp + o, bq_lp + o, cells, nv, dim, s);
        orbit_pack_dev(base_lh + o, bq_lh + o, cells, nv, dim, s);
    };
    std::vector<int> outer_it(n, 0), inner_it(n, 0), refs(n, 0);
    std::vector<double> t_done(n, 0.0);
    std::vector<double> prev_rel(n, 1e300);
    // problems whose last correction did not cut the change by 10x continue with plain FP64
    // SIS steps (the low-precision correction map has reached its precision floor)
    std::vector<char> plain(n, 0);
    std::vector<double> rel_before(n, 0.0);
    const bool trace = std::getenv("LBE_TRACE") != nullptr;  // per-step progress on stderr
    std::vector<char> rebase(n, 0);
    std::vector<int> active(n);
    for (int j = 0; j < n; ++j) active[j] = j;
    const dim3 blk(256);
    // phase 0: low-precision SIS of the full problem from h = 0.  Each problem, as soon as
    // batch_run sees it finish, is widened to FP64 and gets its FP64-class operator evaluation
    // (the base of the increments) on the context's low-priority side stream, overlapping the
    // iterations of the problems still running; the main stream waits for them afterwards.
    if (!c->side_stream) {
        int lo = 0, hi = 0;
        cudaDeviceGetStreamPriorityRange(&lo, &hi);
        if (cudaStreamCreateWithPriority(&c->side_stream, cudaStreamNonBlocking, lo) != cudaSuccess)
            c->side_stream = nullptr;
    }
    cudaStream_t s2 = c->side_stream ? c->side_stream : s;
    if (I.t->tuning) I.t->tuning->side = c->side_stream;
    I.on_done = [&](const std::vector<int>& fin) {
        std::vector<int> js(fin);
        std::sort(js.begin(), js.end());
        for (int j : js) {
            k_widen<<<dim3(sm_count(), 1), blk, 0, s2>>>(I.h.as<float>(), O.h.as<double>(), O.sjobs.as<SweepJobDev>(),
                                                        ident + j, n3, q ? 1 : 0);
            g_launches += 1;
        }
        // one call per run of consecutive finished problems of one geometry (plates: parity
        // mode 2, ducts: mode 1) whose cells are contiguous
        for (size_t a = 0; a < js.size();) {
            size_t b = a + 1;
            long end = O.cell_off[js[a]] + O.sj[js[a]].ncell;
            while (b < js.size() && js[b] == js[b - 1] + 1 && O.geo[js[b]].dim == O.geo[js[a]].dim &&
                   O.cell_off[js[b]] == end)
                end += O.sj[js[b++]].ncell;
            evaluate_base(js[a], js[b - 1] + 1, s2);
            a = b;
        }
    };
    if (st == LBE_OK) st = batch_run(I, 150);
    I.on_done = nullptr;
    if (s2 != s) {  // the main stream continues once every base evaluation is done
        cudaEvent_t ev;
        if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess) {
            cudaEventRecord(ev, s2);
            cudaStreamWaitEvent(s, ev, 0);
            cudaEventDestroy(ev);
        } else {
            cudaStreamSynchronize(s2);
        }
    }
    if (st == LBE_OK) {
        for (int j = 0; j < n; ++j) inner_it[j] += I.hstate[j].iters;
        // from now on the inner batch solves the homogeneous correction equation
        for (int j = 0; j < n; ++j) {
            I.sj[j].forcing = kForcingNone;
            I.ij[j].ndsig = 0.0;
            I.ij[j].eps = 1e-4;  // each correction solve reduces its flow-rate change to 1e-4
            I.ij[j].max_iter = 30;  // or runs 30 SIS iterations (omega <= 0.6: error x 2e-7)
        }
        cudaMemcpyAsync(I.sjobs.p, I.sj.data(), n * sizeof(SweepJobDev), cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(I.ijobs.p, I.ij.data(), n * sizeof(SisJobDev), cudaMemcpyHostToDevice, s);
        g_h2d += n * (sizeof(SweepJobDev) + sizeof(SisJobDev));
        // the one FP64-class collision-operator evaluation of the solve, at h0 = the phase-0
        // solution (above); every later FP64 iteration adds the low-precision operator of the
        // increment h - h0
        O.base_h = bq_h;
        O.base_lp = bq_lp;
        O.base_lh = bq_lh;
        O.inc_h = inc_h;
        O.inc_tc = I.use_tc;  // BF16-refined: the increment h - h0 (~1e-4 of h) takes the
                              // tensor-core operator too; its 2^-16 error is ~1e-9 of h
        O.inc_lp = inc_lp;
        O.inc_lh = inc_lh;
        O.inc_scratch = inc_scratch;
        O.inc_chunk = inc_chunk;
        st = cuda_status(c, cudaStreamSynchronize(s), "refine phase 0");
    }
    I.extra.p = r;
    I.extra.n = vol32;
    if (st != LBE_OK) active.clear();
    while (!active.empty()) {
        const int na = (int)active.size();
        cudaMemcpyAsync(O.act.p, active.data(), na * sizeof(int), cudaMemcpyHostToDevice, s);
        g_h2d += na * sizeof(int);
        // flow rates of the current iterate, then keep a copy of it
        {  // one launch per contiguous run of active problems' cells
            struct Run {
                long c0, n;
                int dim;
            };
            std::vector<Run> runs;
            for (int j : active) runs.push_back({O.cell_off[j], (long)O.sj[j].ncell, O.geo[j].dim});
            std::sort(runs.begin(), runs.end(), [](const Run& a, const Run& b) { return a.c0 < b.c0; });
            std::vector<Run> merged;
            for (auto& r : runs) {
                if (!merged.empty() && merged.back().c0 + merged.back().n == r.c0 && merged.back().dim == r.dim)
                    merged.back().n += r.n;
                else
                    merged.push_back(r);
            }
            for (auto& r : merged)
                launch_moments<double>(*O.t, r.c0, (int)r.n, O.h.as<double>(), O.mom.as<double>(), s,
                                       q ? r.dim : 0);
        }
        k_set_rates<<<na, 32, 0, s>>>(O.ijobs.as<SisJobDev>(), O.act.as<int>(), O.mom.as<double>(),
                                      O.coef.as<double>(), O.states.as<JobState>());
        k_copy64<<<dim3(sm_count(), na), blk, 0, s>>>(O.h.as<double>(), h_old, O.sjobs.as<SweepJobDev>(),
                                                     O.act.as<int>(), n3, q ? 1 : 0);
        g_launches += 2;
        // one FP64 SIS iteration: h = Phi(h_old), flags against the copy's flow rates
        O.active = active;
        batch_iterate<double>(O);
        if ((st = cuda_status(c, cudaStreamSynchronize(s), "refine outer")) != LBE_OK) break;
        if (O.inc_tc && (st = tc_check(c, O.t)) != LBE_OK) break;
        if ((st = O.op_status) != LBE_OK) break;
        std::vector<int> keep;
        const double tnow = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        for (int j : active) {
            ++outer_it[j];
            if (!O.hstate[j].done)
                keep.push_back(j);
            else
                t_done[j] = tnow;
            // the increment's FP32 error (~1e-7 |h - h0|) is the floor of this scheme; when the
            // change stalls near it, re-centre: evaluate the FP64 operator at the next iterate
            const double rel = O.hstate[j].rel, pr = prev_rel[j];
            rebase[j] = (rel > 0.5 * pr && rel < 1e-7) ? 1 : 0;
            prev_rel[j] = rel;
            if (!plain[j] && refs[j] >= 1 && rel > 0.1 * rel_before[j]) plain[j] = 1;
            rel_before[j] = rel;
            if (plain[j] && rel > 0.9 * pr) rebase[j] = 1;  // plain steps stalled: re-centre the operator
            if (trace) {
                const long o = O.cell_off[j] * n3, nn = (long)O.sj[j].ncell * n3;
                const long per = q ? (O.geo[j].dim == 1 ? n3 / 4 : n3 / 2) : n3;  // values held per cell
                std::vector<double> hh(nn), hb(nn);
                cudaMemcpy(hh.data(), h_old + o, nn * 8, cudaMemcpyDeviceToHost);
                cudaMemcpy(hb.data(), bq_h + o, nn * 8, cudaMemcpyDeviceToHost);
                double dmax = 0, hmax = 0;
                for (long k = 0; k < nn; ++k) {
                    if (k % n3 >= per) continue;
                    dmax = std::max(dmax, std::fabs(hh[k] - hb[k]));
                    hmax = std::max(hmax, std::fabs(hh[k]));
                }
                fprintf(stderr, "lbe refine: problem %d outer %d M %.17g Q %.17g rel %.3e |h-h0|/|h| %.3e%s%s\n", j,
                        outer_it[j], O.hstate[j].M, O.hstate[j].Q, rel, dmax / hmax, rebase[j] ? " re-centre" : "",
                        plain[j] ? " plain" : "");
            }
        }
        active.swap(keep);
        if (active.empty()) break;
        // correction solve for the unfinished problems (plain ones keep h = Phi(h_old))
        std::vector<int> corr, rb_plain;
        for (int j : active) (plain[j] ? rb_plain : corr).push_back(j);
        for (int j : rb_plain)
            if (rebase[j]) evaluate_base(j, j + 1, s);
        if (!corr.empty()) {
            const int nk = (int)corr.size();
            cudaMemcpyAsync(O.act.p, corr.data(), nk * sizeof(int), cudaMemcpyHostToDevice, s);
            k_residual<<<dim3(sm_count(), nk), blk, 0, s>>>(O.h.as<double>(), h_old, r, O.sjobs.as<SweepJobDev>(),
                                                           O.act.as<int>(), n3, q ? 1 : 0);
            g_launches += 1;
            for (int j : corr) {
                cudaMemsetAsync(I.h.as<float>() + I.cell_off[j] * n3, 0, I.sj[j].ncell * n3 * 4, s);
                cudaMemsetAsync(I.hmom.as<double>() + I.cell_off[j] * 2, 0, I.sj[j].ncell * 2 * 8, s);
                I.hstate[j] = JobState{};
            }
            cudaMemcpyAsync(I.states.p, I.hstate.data(), n * sizeof(JobState), cudaMemcpyHostToDevice, s);
            g_h2d += n * sizeof(JobState);
            I.active = corr;
            if ((st = batch_run(I, 30)) != LBE_OK) break;
            for (int j : corr) {
                inner_it[j] += I.hstate[j].iters;
                ++refs[j];
                if (trace)
                    fprintf(stderr, "lbe refine: problem %d correction %d inner iterations %d Me %.3e Qe %.3e rel %.3e\n",
                            j, refs[j], I.hstate[j].iters, I.hstate[j].M, I.hstate[j].Q, I.hstate[j].rel);
            }
            cudaMemcpyAsync(O.act.p, corr.data(), nk * sizeof(int), cudaMemcpyHostToDevice, s);
            k_apply_correction<<<dim3(sm_count(), nk), blk, 0, s>>>(h_old, I.h.as<float>(), O.h.as<double>(),
                                                                   O.sjobs.as<SweepJobDev>(), O.act.as<int>(), n3,
                                                                   q ? 1 : 0);
            g_launches += 1;
            for (int j : corr)
                if (rebase[j]) evaluate_base(j, j + 1, s);
        }
        // drop problems that reached their iteration cap
        std::vector<int> keep2;
        for (int j : active)
            if (outer_it[j] < pbs[j].max_iter) keep2.push_back(j);
        active.swap(keep2);
    }
    if (st == LBE_OK) st = cuda_status(c, cudaStreamSynchronize(s), "refine");
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    lbe_status worst = LBE_OK;
    if (st == LBE_OK) {
        for (int j = 0; j < n; ++j) {
            fill_result(O, j, &outs[j], secs);
            outs[j].iters = outer_it[j] + inner_it[j];
            outs[j].refinements = refs[j];
            outs[j].seconds = t_done[j] > 0 ? t_done[j] : secs;
            if (outs[j].status != LBE_OK && worst == LBE_OK) worst = (lbe_status)outs[j].status;
        }
        if (U3_out) {
            st = cuda_status(c, cudaMemcpy(U3_out, O.U3.p, O.cells * 8, cudaMemcpyDeviceToHost), "U3");
            g_d2h += O.cells * 8;
        }
        if (st == LBE_OK && h_out) {
            st = cuda_status(c, cudaMemcpy(h_out, O.h.p, vol64, cudaMemcpyDeviceToHost), "h");
            if (st == LBE_OK && q) {  // back to the full grid
                std::vector<double> hq;
                for (int j = 0; j < n; ++j) {
                    const long o = O.cell_off[j] * n3, nn = (long)O.sj[j].ncell * n3;
                    hq.assign(h_out + o, h_out + o + nn);
                    orbit_unpack_host(nv, O.sj[j].ncell, hq.data(), h_out + o, O.geo[j].dim);
                }
            }
        }
    }
    return st != LBE_OK ? st : worst;
}

}  // namespace lbe

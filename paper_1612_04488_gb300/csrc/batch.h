// A batch of problems sharing one velocity grid and precision: device state and the
// host-driven CIS / SIS iteration over it (api.cu), used by the solve calls, the resident
// batches, the refinement driver and the service.
#pragma once

#include <functional>
#include <vector>

#include "lbe_internal.h"
#include "sweep.h"

namespace lbe {

struct DevBuf {  // a piece of an arena
    void* p = nullptr;
    size_t n = 0;
    template <typename T> T* as() const { return (T*)p; }
};

struct Batch {
    Ctx* c = nullptr;
    Arena* arena = nullptr;
    cudaStream_t s = nullptr;
    DevTables* t = nullptr;
    int prec = 0;
    int njobs = 0;
    long cells = 0;
    std::vector<lbe_problem> pbs;
    std::vector<SweepGeom> geo;
    std::vector<SweepJobDev> sj;
    std::vector<SisJobDev> ij;
    std::vector<long> cell_off;
    DevBuf h, hh, lp, lh, scratch, mom, G, dU, U3, delta, nd, coef, work, sjobs, ijobs, states, act;
    DevBuf extra;  // optional additive source in the correction step (same type as h)
    // [cells][2]: the h part of the SIS L-moments of the current h, summed by the correction
    // step (tensor-core batches); zero wherever h is reset to zero
    DevBuf hmom;
    // Increment mode (FP64 batches of the refinement driver): the collision operator of h is
    // base_lp / base_lh (FP64 operator of base_h, computed once) plus the FP32 operator of
    // the increment h - base_h.  Unset: the operator runs in the batch's own arithmetic.
    const double* base_h = nullptr;
    const double* base_lp = nullptr;
    const double* base_lh = nullptr;
    float* inc_h = nullptr;
    float* inc_lp = nullptr;
    float* inc_lh = nullptr;
    void* inc_scratch = nullptr;
    int inc_chunk = 1;
    bool use_tc = false;  // FP32 batches: collision operator by the dense tensor-core GEMM
    // plates (1D problems) keep h, the operator output and the sweep output in the orbit
    // layout (sweep.h): a quarter of each cell's velocity points.  Set with use_tc, and on the
    // FP64 batch of a BF16-refined solve (its increments through the tensor-core operator).
    bool orbit = false;
    bool quarter() const { return orbit; }
    bool inc_tc = false;  // FP64 batches in increment mode: the increment's operator by that GEMM
    lbe_status op_status = LBE_OK;  // first failure of an operator launch inside an iteration
    int chunk = 1;
    std::vector<JobState> hstate;
    std::vector<int> active;
    double t_start = 0;            // host clock (s) when batch_run began
    std::vector<double> t_done;    // host clock (s) when each job's flag was seen
    std::vector<double> omega;     // observed contraction per iteration of each job's change
    // One iteration over a fixed active set captured as a CUDA graph (batch_run replays it
    // between convergence checks); re-captured when the active set changes.
    cudaGraphExec_t graph = nullptr;
    std::vector<int> graph_key;
    unsigned long long graph_launches = 0, graph_levals = 0;  // counters of one replay
    bool graphs_ok = true;          // false after a failed capture (then iterations are queued plainly)
    // Called by batch_run with the problems it has just seen finish (or reach its step limit),
    // after the host synchronised the stream: their iterates are final, and later iterations
    // leave them untouched.
    std::function<void(const std::vector<int>&)> on_done;
    Batch() = default;
    Batch(const Batch&) = delete;
    Batch& operator=(const Batch&) = delete;
    ~Batch() {
        if (graph) cudaGraphExecDestroy(graph);
    }
};

// Internal forcing value: no source term and no momentum-balance term (the homogeneous
// part of the SIS map, used by the refinement driver's correction solves).
constexpr int kForcingNone = 2;

// Host: the full velocity grid of `cells` cells from their orbit layout (sweep.h; cell stride
// nv^3; dim 1 plates, 2 ducts), restoring the R2 images (equal, plates) and the R3 images
// (negated).
template <typename TQ>
inline void orbit_unpack_host(int nv, long cells, const TQ* q, double* full, int dim = 1) {
    const int H = nv / 2, R2 = dim == 2 ? nv : H;
    const long n3 = (long)nv * nv * nv;
    for (long c = 0; c < cells; ++c)
        for (int i1 = 0; i1 < nv; ++i1)
            for (int i2 = 0; i2 < nv; ++i2)
                for (int i3 = 0; i3 < nv; ++i3) {
                    const int j2 = dim == 2 || i2 < H ? i2 : nv - 1 - i2, j3 = i3 < H ? i3 : nv - 1 - i3;
                    const double v = (double)q[c * n3 + ((long)i1 * R2 + j2) * H + j3];
                    full[c * n3 + ((long)i1 * nv + i2) * nv + i3] = i3 < H ? v : -v;
                }
}

lbe_status batch_init(Batch& B, Ctx* c, const lbe_problem* pbs, int n, Arena* arena, cudaStream_t stream);
// One iteration over B.active.  upload: copy the active list to the device first (it has not
// changed since the previous iteration otherwise); read: copy the convergence states back to
// B.hstate at the end (the host waits for that copy).
template <typename T> void batch_iterate(Batch& B, bool upload = true, bool read = true);
lbe_status batch_run(Batch& B, int max_steps);
void fill_result(const Batch& B, int j, lbe_result* r, double secs);

// refine.cu helpers shared with the service
void launch_set_rates(int njobs, const SisJobDev* jobs, const int* active, const double* mom, const double* coef,
                      JobState* state, cudaStream_t s);
void range_widen(const float* e, double* h, long n, cudaStream_t s);
void range_copy(const double* a, double* b, long n, cudaStream_t s);
void range_residual(const double* h, const double* h_old, float* r, long n, cudaStream_t s);
void range_correct(const double* h_old, const float* e, double* h, long n, cudaStream_t s);
void range_sub_f32(const double* h, const double* base, float* out, long n, cudaStream_t s);
void range_add_f64(const double* base, const float* inc, double* out, long n, cudaStream_t s);
// the same steps on the orbit-layout prefix (the first nq values: nv^3 / 4 plates, nv^3 / 2
// ducts) of `cells` cells, cell stride n3
void range_sub_f32_q(const double* h, const double* base, float* out, long cells, long n3, long nq, cudaStream_t s);
void range_add_f64_q(const double* base, const float* inc, double* out, long cells, long n3, long nq,
                     cudaStream_t s);
void range_copy_q(const double* a, double* b, long cells, long n3, long nq, cudaStream_t s);
// full grid <-> orbit layout of `cells` cells (FP64; dim 1 plates, 2 ducts): unpack restores the
// images of the orbit's representative
void orbit_unpack_dev(const double* q, double* full, long cells, int nv, int dim, cudaStream_t s);
void orbit_pack_dev(const double* full, double* q, long cells, int nv, int dim, cudaStream_t s);
// the same steps for `cells` cells whose FP32 side is in the orbit layout (sweep.h; dim 1
// plates, 2 ducts) and whose FP64 side is on the full grid
void range_widen_q(const float* e, double* h, long cells, int nv, int dim, cudaStream_t s);
void range_correct_q(const double* h_old, const float* e, double* h, long cells, int nv, int dim, cudaStream_t s);
void range_residual_q(const double* h, const double* h_old, float* r, long cells, int nv, int dim, cudaStream_t s);

}  // namespace lbe

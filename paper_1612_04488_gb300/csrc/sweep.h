// Device-side job descriptors shared by the sweep / SIS kernels and the host driver.
#pragma once

#include <cuda_runtime.h>

#include "../../include/lbe.h"

namespace lbe {

struct DevTables;
struct Ctx;

// fsm_dense.cu: tensor-core operator on the parity subspace (float in / out; mode 1 or 2)
// hm (may be NULL): per cell the h part of G (launch_correct); with it and without Lout the
// expand reads no h.
// quarter: h, Lplus and Lout in the orbit layout (below; plates a quarter, ducts a half); G needs
// hm and no Lout.
lbe_status tc_apply_sym(Ctx* c, DevTables* t, int mode, int cells, const double* delta, const float* h,
                        float* Lplus, float* Lout, cudaStream_t s, bool sync = true, const double* nd = nullptr,
                        double* G = nullptr, const double* hm = nullptr, bool quarter = false);
lbe_status tc_check(Ctx* c, DevTables* t);
void tc_release(Ctx* c, DevTables* t);
// the binary-mixture operator on the tensor cores: the FP64 matrix L ([n][n], both species)
// in BF16 hi / lo; apply: y_a = scale (L h) for cells whose unknowns are h_A, h_B at [c cs],
// nr per species (float accumulation; y float with f32, else double), GEMM column n being cell
// map[n] when a cell list is given; check reads the GEMM's failure word after the stream's
// synchronisation
struct MixTc;
lbe_status mix_tc_build(Ctx* c, const double* L, int n, MixTc** out, cudaStream_t s);
lbe_status mix_tc_apply(Ctx* c, MixTc* m, int cells, const double* hA, const double* hB, long cs, int nr,
                        double scale, void* yA, void* yB, bool f32, cudaStream_t s, const int* map = nullptr);
lbe_status mix_tc_check(Ctx* c, MixTc* m);
void mix_tc_release(Ctx* c, MixTc* m);
// refine.cu: BF16 operator inside an outer defect-correction loop
lbe_status refined_solve(Ctx* c, const lbe_problem* pbs, int n, lbe_result* outs, double* U3_out,
                         double* h_out);
// serve.cu
void stop_service(Ctx* c);
// mixture.cu: frees the cached mixture operators
void mix_release(Ctx* c);

struct SweepJobDev {
    long cell_off;   // first cell of the job in the batched [cell][v] arrays
    int ncell;       // 1D: nodes, 2D: nx * ny
    int nx, ny;      // 2D
    int coef_off;    // 1D: [fa|fb|fc|ba|bb|bc] (n each); 2D: [xa|xb|xc] (nx) [ya|yb|yc] (ny)
    int forcing;     // source S added to the right-hand side: 0 Poiseuille, 1 thermal transp.
    double delta;
};

struct SisJobDev {
    long cell_off;
    int ncell;
    int dim;
    int nx, ny;
    double width;
    int scheme;      // 0 CIS, 1 SIS
    int coef_off;    // 1D: [fa|fb|fc|x] (n each); 2D: [Sx (mx^2) | Sy (my^2) | lambda (mx*my)]
    int trap_off;    // flow-rate weights (n): M = sum w_c U_c
    long work_off;   // 2D scratch (2 * mx * my doubles)
    double ndsig;    // N delta sigma (sigma = 1 Poiseuille, 0 thermal transpiration)
    double eps;
    int max_iter;
    int crit;        // 0: |dM| < eps |M| and |dQ| < eps |Q| (Sec. 2.4); 1: both changes < eps max(|M|, |Q|)
};

// Convergence state of one problem.  skip = 1 while an iteration passes over a problem that
// was already done when the iteration began (the update and the correction leave it untouched,
// so iterations can be queued ahead of the host's convergence check).
struct JobState {
    double M, Q, Mprev, Qprev, rel;
    int iters, done, nan, skip;
};

// Orbit layout ("quarter" flags): each cell keeps one value per orbit of its problem's parity
// group, in the first places of the cell's nv^3 (the cell stride is unchanged).
//   plates (1D, odd in v3, even in v2): orbits {1, R2, R3, R2 R3}, the points i2, i3 < nv / 2 at
//     (i1 nv / 2 + i2) nv / 2 + i3 (a quarter); h(i1, nv-1-i2, i3) = h(i1, i2, i3);
//   ducts (2D, odd in v3): orbits {1, R3}, the points i3 < nv / 2 at (i1 nv + i2) nv / 2 + i3
//     (a half);
// and in both h(i1, i2, nv-1-i3) = -h(i1, i2, i3).  The tensor-core batches use it.
template <typename T>
void launch_sweep(const DevTables& t, int dim, int njobs, int max_coef, const T* rhs, T* h,
                  const SweepJobDev* jobs, const int* active, const double* coef, cudaStream_t s,
                  int quarter = 0);
template <typename T>
void launch_moments(const DevTables& t, long cell0, int cells, const T* h, double* mom, cudaStream_t s,
                    int quarter = 0);
void launch_sis_update(const DevTables& t, int njobs, const SisJobDev* jobs, const int* active,
                       const double* mom, const double* G, const double* coef, double* work, double* dU,
                       double* U3, JobState* state, cudaStream_t s);
// hm (may be NULL; [cells][2] double): per cell the L-moment part carried by the new h,
// Gh_j = 2 sum_v v_j v3 (N delta - delta nu) h dv^3 (j = 1, 2), with N delta per cell from nd --
// the tensor-core operator adds it to 2 sum v_j v3 L+ h dv^3 instead of reading h again.
template <typename T>
void launch_correct(const DevTables& t, int njobs, const T* hh, T* h, const double* dU, const T* extra,
                    const SweepJobDev* jobs, const int* active, cudaStream_t s, const JobState* state = nullptr,
                    double* hm = nullptr, const double* nd = nullptr, int quarter = 0, int max_cells = 0,
                    int ducts = 1);

// fsm_cc.cu
void init_twiddles_cc();
size_t fsm_cc_scratch_bytes(const DevTables& t, int cells, int elem_bytes, int* chunk_out);
template <typename T>
lbe_status fsm_cc_apply(const DevTables& t, int cells, const double* delta, const T* h, T* Lplus, T* Lout,
                        void* scratch, int chunk, cudaStream_t s, int mode = 0);
// the same operator in double-float arithmetic on double data (scratch as for double)
lbe_status fsm_df_apply(const DevTables& t, int cells, const double* delta, const double* h, double* Lplus,
                        double* Lout, void* scratch, int chunk, cudaStream_t s, int mode = 0);
template <typename T>
void lmoments(const DevTables& t, int cells, const T* Lh, const T* h, const double* nd, double* G,
              cudaStream_t s, int quarter = 0);

}  // namespace lbe

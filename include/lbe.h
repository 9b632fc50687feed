/*
 * lbe.h -- C ABI of the GB300 (sm_103a) steady linearized-Boltzmann solver.
 *
 * The solver follows Wu, Zhang, Liu, Zhang & Reese, "A fast iterative scheme for the
 * linearized Boltzmann equation" (arXiv:1612.04488):
 *   - problem statement: Sec. 2 (Eq. LBE, Eq. LBE_collision, the source S, the moments
 *     U3, P13, q3 and the flow rates M, Q);
 *   - conventional iterative scheme (CIS): Sec. 2, Eq. LBE_iteration;
 *   - synthetic iterative scheme (SIS): Sec. 2.2 (Eqs. syn_LBE, diffusion_LBE, guided),
 *     1D form Eq. first_order (Sec. 2.4), with the N-penalised split
 *     L = (L + N delta h) - N delta h (abstract; Sec. 4.1 footnote) and N = nu_bar/delta
 *     by default (Sec. 2.5);
 *   - plates on the clustered node map of Sec. 2.4, rectangular ducts (Sec. 2.4, Table 2).
 * The hard-sphere collision operator is evaluated by the fast spectral method (Sec. 2.4
 * cites it); the discrete operator is: midpoint velocity grid on [-vmax, vmax]^3, Carleman
 * truncation |x|,|y| <= R, M directions on a hemisphere (Gauss-Legendre in cos(theta) x
 * midpoint azimuths), loss term with the same per-direction multipliers, Nyquist planes
 * zeroed, collision strength fixed by nu_bar = 1.25 delta (Sec. 2.5).
 *
 * Conventions for every call:
 *   - every call returns an lbe_status and never aborts the process;
 *   - inputs are borrowed for the duration of the call; outputs go to caller-owned memory;
 *   - pointers named *_dev are CUDA device pointers on the context's device, all other
 *     pointers are host pointers;
 *   - velocity-space arrays are laid out [cell][i1][i2][i3] with i3 (v3) fastest, i.e.
 *     cell-major, nv^3 contiguous values per cell;
 *   - a context is used by one host thread at a time, except lbe_submit / lbe_poll, which
 *     are thread-safe.
 */
#ifndef LBE_H
#define LBE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LBE_OK = 0,
    LBE_NOT_CONVERGED = 1, /* iteration cap reached; outputs hold the last iterate       */
    LBE_NAN = 2,           /* a non-finite flow rate was detected on the device           */
    LBE_BAD_ARG = 3,       /* invalid argument; nothing was launched                      */
    LBE_OOM = 4,           /* device memory (or the context's HBM budget) exhausted       */
    LBE_TIMEOUT = 5,       /* a bounded device wait expired; the context stays usable     */
    LBE_INTERNAL = 6,      /* CUDA runtime error; see lbe_last_error()                    */
    LBE_UNSUPPORTED = 7,   /* valid request outside what this build implements            */
    LBE_CANCELLED = 8      /* a served request withdrawn by lbe_cancel                     */
} lbe_status;

/* Source term S of Sec. 2 with X_P = X_T = -1. */
typedef enum { LBE_POISEUILLE = 0, LBE_THERMAL_TRANSPIRATION = 1 } lbe_forcing;

/* Sec. 2 Eq. LBE_iteration (CIS) or Sec. 2.2 (SIS). */
typedef enum { LBE_CIS = 0, LBE_SIS = 1 } lbe_scheme;

/* Arithmetic of the collision operator and the sweeps.  LBE_FP64: everything in double.
 * LBE_FP32: float storage and transforms, double reductions and diffusion solve.
 * LBE_BF16_REFINED and LBE_FP32_REFINED: defect correction towards the FP64 SIS solution --
 * each outer step is one FP64 SIS iteration (its flow-rate change is the stopping test, as
 * for LBE_FP64), and the correction equation is solved by low-precision SIS iterations
 * whose collision operator runs as tcgen05 BF16 spectral GEMMs with FP32 accumulation
 * (BF16_REFINED) or as the FP32 CUDA-core transforms (FP32_REFINED).  max_iter caps the
 * FP64 iterations.  The FP64 iterations evaluate the operator as L(h0) + L(h - h0): L(h0)
 * once per solve (and when re-centred) in LBE_DF32 arithmetic, the small increment h - h0
 * with the same low-precision operator as the correction solves.
 * LBE_BF16 (solves only): the low-precision phase of LBE_BF16_REFINED on its own -- the
 * tcgen05 BF16 operator with FP32 everything else and FP64 reductions, no refinement; it
 * stops when both flow-rate changes fall below eps times the larger flow rate (a plain
 * relative change of a small flow rate cannot get below FP32 rounding).  Its flow rates
 * agree with LBE_FP64 to about 1e-5 relative.
 * LBE_DF32 (the operator entry points lbe_apply_L and lbe_apply_L_sym only): data in double,
 * arithmetic in double-float -- each value the unevaluated sum of two floats, about 2^-44
 * relative per operation when the pairs are normalised, on the FP32 pipes, which this GPU
 * issues at many times its FP64 rate.  Pairs are left unnormalised between operations
 * (|lo| may grow to a few ulps of hi), so the per-operation bound grows with |lo|/ulp(hi);
 * the agreement with LBE_FP64, about 1e-13 of the scale, is measured (parity tests), not
 * guaranteed by that bound.  Values below the float range (|x| < 1e-38, the far tails of
 * f_eq) are flushed to zero. */
typedef enum {
    LBE_FP64 = 0,
    LBE_FP32 = 1,
    LBE_BF16_REFINED = 2,
    LBE_FP32_REFINED = 3,
    LBE_DF32 = 4,
    LBE_BF16 = 5
} lbe_precision;

/* Geometry (Sec. 2.4).  dim = 1: plates at x1 = +-1/2, half channel -1/2 <= x1 <= 0 with a
 * specular symmetry plane at x1 = 0, ns sections (ns + 1 nodes), grid_kind 0 = uniform,
 * 1 = the clustered map x1 = (10 - 15 s + 6 s^2) s^3 - 1/2, s = (0..ns)/(2 ns).
 * dim = 2: duct [0, width] x [0, 1] (lengths scaled by the shorter side), nx x ny uniform
 * cells, diffuse walls on all four sides. */
typedef struct {
    int dim;
    int ns;
    int grid_kind;
    int nx, ny;
    double width;
} lbe_geometry;

typedef struct {
    lbe_geometry geom;
    double delta;        /* rarefaction parameter, Eq. delta; delta >= 0                      */
    double N;            /* SIS tuning parameter; <= 0 selects nu_bar/delta = 1.25 (Sec. 2.5)   */
    int nv;              /* velocity points per axis: 8, 16, 24 or 32                           */
    double vmax;         /* velocity box [-vmax, vmax]^3                                        */
    int M;               /* hemisphere directions: power of two, 4..64                          */
    double R;            /* Carleman truncation radius; <= 0 selects 0.75 * vmax                */
    lbe_forcing forcing;
    lbe_scheme scheme;
    lbe_precision precision;
    double eps;          /* stop when |dM| < eps |M| and |dQ| < eps |Q| (Sec. 2.4); 0 = never  */
    int max_iter;        /* iteration cap (>= 1)                                                */
} lbe_problem;

typedef struct {
    double mass_flow;        /* M of the last iterate                                         */
    double heat_flow;        /* Q of the last iterate                                         */
    int iters;               /* iterations performed (kinetic sweeps)                         */
    int status;              /* lbe_status of this solve                                      */
    double last_rel_change;  /* max(|dM/M|, |dQ/Q|) of the last iteration                      */
    double seconds;          /* wall time from admission to completion                        */
    int refinements;         /* outer defect-correction steps (LBE_BF16_REFINED), else 0       */
} lbe_result;

typedef struct lbe_ctx lbe_ctx;

/* Create a context on CUDA device `device`.  hbm_budget_bytes caps the device memory the
 * context allocates (0 = 90% of the free memory at creation).  *ctx receives the handle. */
lbe_status lbe_create(lbe_ctx** ctx, int device, size_t hbm_budget_bytes);

/* Release every resource of the context (waits for queued serving work to finish). */
lbe_status lbe_destroy(lbe_ctx* ctx);

const char* lbe_status_str(lbe_status s);

/* Text of the last CUDA / argument error seen by this context (never NULL). */
const char* lbe_last_error(lbe_ctx* ctx);

/* Number of cells (1D nodes or 2D cells) of a problem's spatial grid. */
int lbe_problem_cells(const lbe_problem* pb);

/* Solve one problem to convergence (or max_iter).  U3_out (host, [cells] or NULL) receives
 * U3 of the last iterate; h_out (host, [cells * nv^3] or NULL) receives h as double.  With
 * eps = 0 exactly max_iter iterations run (status LBE_NOT_CONVERGED). */
lbe_status lbe_solve(lbe_ctx* ctx, const lbe_problem* pb, lbe_result* out,
                     double* U3_out, double* h_out);

/* Solve n problems that share (nv, vmax, M, R, precision) together: one batched collision
 * launch and one batched sweep launch per iteration cover every unfinished problem.  outs
 * receives n results.  Finished problems stop iterating while the others continue. */
lbe_status lbe_solve_batch(lbe_ctx* ctx, const lbe_problem* pbs, int n, lbe_result* outs);

/* Resident batch: lbe_batch_create validates the problems (same rules as lbe_solve_batch),
 * allocates their device state and uploads the grids once; every lbe_batch_run restarts
 * all problems from h = 0 and iterates them to convergence with nothing but the per-
 * iteration convergence flags crossing to the host; outs receives n results.  The batch
 * keeps its own device memory until lbe_batch_destroy.  LBE_BF16_REFINED is not accepted
 * here (use lbe_solve_batch). */
typedef struct lbe_batch lbe_batch;
lbe_status lbe_batch_create(lbe_ctx* ctx, const lbe_problem* pbs, int n, lbe_batch** out);
lbe_status lbe_batch_run(lbe_batch* b, lbe_result* outs);
lbe_status lbe_batch_destroy(lbe_batch* b);

/* Collision operator on device data (steps A1-A4), over all M directions, for any h.
 * precision: LBE_FP64, LBE_DF32 or LBE_FP32 (the tensor-core form acts on the parity
 * subspace only: see lbe_apply_L_sym).  h_dev: [cells][nv^3] of double (FP64, DF32) or
 * float (FP32).  delta_dev: [cells] double, the rarefaction of each cell.
 * Outputs (same type as h, any may be NULL): Lplus_dev = L+ h, L_dev = L h.
 * G_dev (double [cells][2], may be NULL): G_j = 2 sum_v v_j v3 (L h + n_delta h) dv^3 with
 * n_delta = N delta per cell taken from ndelta_dev (double [cells]; required with G_dev).
 * stream: cudaStream_t or NULL for the legacy default stream.  Asynchronous. */
lbe_status lbe_apply_L(lbe_ctx* ctx, int nv, double vmax, int M, double R,
                       lbe_precision precision, int cells, const double* delta_dev,
                       const void* h_dev, void* Lplus_dev, void* L_dev,
                       const double* ndelta_dev, double* G_dev, void* stream);

/* Collision operator restricted to the parity subspace of the plate and duct solutions
 * (steps A1-A4).  The source S of Sec. 2 is odd in v3, so every CIS / SIS iterate is odd in
 * v3, and on plates also even in v2; the discrete operator commutes with those reflections.
 * parity = 1: h odd in v3 (ducts); parity = 2: h odd in v3 and even in v2 (plates).  For
 * such h the result equals lbe_apply_L's up to rounding; for other h it is not defined.
 * LBE_FP64 / LBE_DF32 / LBE_FP32: fast spectral transforms of one direction per reflection
 * orbit (a quarter or half of the directions).  LBE_BF16_REFINED: the operator as a dense
 * (nv^3/4 or nv^3/2)-square matrix at delta = 1, built once per grid from the DF32
 * transforms, applied to all cells as one tcgen05 GEMM with bfloat16 hi/lo operands and FP32
 * accumulation (relative error about 1e-5 of the scale); h, L+ h, L h are float, h 8-byte
 * aligned.  Needs
 * M >= 8.  Lplus_dev / L_dev may be NULL.  G_dev (double [cells][2], may be NULL): the
 * L-moments G_j of lbe_apply_L with n_delta from ndelta_dev (required with G_dev); the
 * tensor-core form sums them in the same pass that expands L+ h, without storing L h.
 * LBE_BF16 is accepted as a synonym of LBE_BF16_REFINED here.  Returns after the work is
 * queued on `stream` (the tensor-core form synchronises the stream). */
lbe_status lbe_apply_L_sym(lbe_ctx* ctx, int nv, double vmax, int M, double R, lbe_precision precision,
                           int parity, int cells, const double* delta_dev, const void* h_dev,
                           void* Lplus_dev, void* L_dev, const double* ndelta_dev, double* G_dev,
                           void* stream);

/* lbe_apply_L without any device allocation.  The paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory -- code recording CUDA
 * graphs or running a latency-critical loop, where cudaMalloc / cudaFree would synchronise
 * the device or is not allowed mid-capture, and host frameworks whose pooling allocator
 * owns all device memory.  It runs the same collision-operator kernels as lbe_apply_L
 * (FP64 or FP32 only; no G moments) on caller-owned inputs and outputs, with its transform
 * scratch taken from one file-scope device array of 32 MiB that every GPU loading this
 * library holds until the process exits.  Cells are processed in slices that fit that
 * array; if one cell does not fit (nv = 32 with M = 64 in FP64) the call returns
 * LBE_BAD_ARG.  The context must already hold the operator tables for (nv, vmax, M, R): an
 * earlier lbe_apply_L or lbe_solve with those parameters builds them; otherwise the call
 * returns LBE_BAD_ARG instead of allocating them.  The first call on a device looks up the
 * scratch array's device address; with lazy module loading (CUDA's default) that lookup is
 * also when the driver loads the library's module and reserves the 32 MiB, so the first
 * call can fail with LBE_OOM (or LBE_INTERNAL) when the device is full.  Make it before any
 * stream capture; later calls on that device allocate nothing.  All calls share the array
 * and its contents persist between calls; calls that overlap on the GPU race, so serialise
 * them (e.g. one stream).  Nothing in the array needs to start at zero.  The result is
 * bitwise that of lbe_apply_L (the per-cell arithmetic does not depend on how the cells are
 * sliced).  Asynchronous on `stream`. */
lbe_status lbe_apply_L_noalloc(lbe_ctx* ctx, int nv, double vmax, int M, double R,
                               lbe_precision precision, int cells, const double* delta_dev,
                               const void* h_dev, void* Lplus_dev, void* L_dev, void* stream);

/* Convergence factor of the CIS or the SIS for one Fourier mode (Sec. 2.3): a system periodic
 * in x1 with the mode exp(2 pi i x1), whose error obeys, per iteration, the CIS map
 * e <- L+(e) / (nu_eq + 2 pi i v1) (Eq. conv_iteration), or for the SIS that half step
 * followed by U3 = (-2 pi i A1 - 4 pi^2 A2) / (4 pi^2) with A1 = 2 int v1 v3 (L e + N delta e),
 * A2 = int (2 v1^2 - 1) v3 e_half, and the correction of Eq. guided.  Runs the power iteration
 * e_{k+1} = P map(e_k) / |e_k|, P the projection onto functions odd in v3 (the parity of the
 * plate and duct errors; rounding would otherwise seed even, density-type modes that the SIS
 * does not accelerate), from e0 (host, double [2][nv^3]: real part, then imaginary
 * part) with the FP64 collision operator, and writes ratios[k] = |e_{k+1}| (host, double
 * [iters]); the ratios converge to omega, the modulus of the dominant eigenvalue (the paper
 * fits U3(k) = U_inf + C exp(-lambda k), omega = exp(-lambda)).  N <= 0 selects 1.25.  The
 * start vector is the caller's, so runs are reproducible.  Synchronous on the context's
 * stream. */
lbe_status lbe_fourier_omega(lbe_ctx* ctx, int nv, double vmax, int M, double R, double delta, double N,
                             lbe_scheme scheme, int iters, const double* e0, double* ratios);

/* Solve one problem starting from a checkpoint instead of h = 0 (checkpoint / resume; the
 * SIS state is the iterate h and the flow rates of the stopping test).  h_in (host, double
 * [cells * nv^3], the layout of lbe_solve's h_out) is the starting VDF.  prev (may be NULL)
 * is the lbe_result of the run that produced h_in: its mass_flow and heat_flow start the
 * stopping test, so a solve stopped after k iterations and resumed here continues exactly
 * as the uninterrupted solve would -- the iterates, flow rates and stopping decision are
 * bitwise those of the uninterrupted run.  With prev = NULL the first change is measured
 * against the flow rates of h_in computed afresh.  LBE_FP64, LBE_FP32 and LBE_BF16 (FP32 data
 * are rounded from h_in; LBE_BF16 plates keep one value per orbit of the v2 and v3 reflections,
 * taken from h_in at v2 < 0, v3 < 0).  The refined precisions are rejected (LBE_BAD_ARG): their
 * state also holds the FP64 base point of the defect correction.  Outputs as for lbe_solve;
 * out->iters counts this call's iterations. */
lbe_status lbe_solve_from(lbe_ctx* ctx, const lbe_problem* pb, const double* h_in, const lbe_result* prev,
                          lbe_result* out, double* U3_out, double* h_out);

/* Transport sweep of one problem (steps A5-A6): solves nu_eq h + v.grad h = rhs with the
 * problem's geometry and delta.  rhs_dev, h_dev: [cells][nv^3], double for FP64 else
 * float.  mom_dev (double [cells][5], may be NULL): U3, q3, W1 = F201/4, W2 = F021/4,
 * X12 = F111/4 of the result.  Asynchronous on `stream`. */
lbe_status lbe_sweep(lbe_ctx* ctx, const lbe_problem* pb, const void* rhs_dev, void* h_dev,
                     double* mom_dev, void* stream);

/* SIS diffusion solve (step A7) on host arrays of length cells: given the half-step
 * moments Uh, W1, W2, X12 and the L-moments G1, G2 of one problem, write U3^(k+1) to
 * U_out.  Runs the device kernel and synchronises. */
lbe_status lbe_diffusion(lbe_ctx* ctx, const lbe_problem* pb, const double* Uh,
                         const double* W1, const double* W2, const double* X12,
                         const double* G1, const double* G2, double* U_out);

/* Continuous-batching service.  lbe_submit queues a problem and returns a ticket at once;
 * a service thread admits queued problems while slots and the HBM budget allow, advances
 * all admitted problems together (shared collision and sweep launches per velocity grid)
 * and retires each one as it converges.  lbe_poll reports completion (*done = 1) and
 * copies the result; a ticket can be polled until lbe_destroy.  Thread-safe. */
lbe_status lbe_submit(lbe_ctx* ctx, const lbe_problem* pb, uint64_t* ticket);
lbe_status lbe_poll(lbe_ctx* ctx, uint64_t ticket, lbe_result* out, int* done);

/* Withdraw a submitted request.  A request still queued is dropped at once; an admitted one
 * leaves the service at its next iteration boundary (its slot and cells are freed, none of
 * its kernels is interrupted).  Either way lbe_poll then reports it done with status
 * LBE_CANCELLED.  Cancelling a finished request changes nothing.  Thread-safe. */
lbe_status lbe_cancel(lbe_ctx* ctx, uint64_t ticket);

/* Maximum problems advanced together by the service (default 64). */
lbe_status lbe_set_max_active(lbe_ctx* ctx, int max_active);

/* Run the context's synchronous calls (lbe_solve, lbe_solve_batch, lbe_diffusion) on the
 * caller's CUDA stream (cudaStream_t, or NULL for the context's own stream).  The stream
 * must belong to the context's device and outlive its use. */
lbe_status lbe_set_stream(lbe_ctx* ctx, void* stream);

/* Process-wide counters since the library was loaded: kernels launched by this library,
 * bytes it copied host->device and device->host, and cells passed through the collision
 * operator (one cell = one application of L to one nv^3 vector).  With kernel timing on
 * (lbe_set_kernel_timing), every tensor-core GEMM launched by lbe_apply_L_sym, and every
 * GEMM of the mixture operator (lbe_mix_apply_L, lbe_mix_solve: FP64, double-float or on the
 * tensor cores), is bracketed by CUDA events on its stream and waited for: dense_gemm_timed
 * counts those launches and dense_gemm_ms sums their durations; and every transport-sweep
 * launch of a solve (step A5, one launch per geometry per iteration) likewise: sweep_timed,
 * sweep_ms, and sweep_bytes, the algorithmic bytes of those launches (right-hand side read
 * and h written once per cell-velocity).
 * Reading the counters waits for the timed sweeps to finish. */
typedef struct {
    uint64_t kernel_launches;
    uint64_t h2d_bytes;
    uint64_t d2h_bytes;
    uint64_t cell_l_evals;
    uint64_t dense_gemm_timed;
    double dense_gemm_ms;
    uint64_t sweep_timed;
    double sweep_ms;
    double sweep_bytes;
} lbe_stats;
lbe_status lbe_get_stats(lbe_stats* out);

/* Process-wide switch (0 = off, the default) for the event timing described above. */
lbe_status lbe_set_kernel_timing(int on);

/* The autotuner's decisions in this context, one text line each (for logs and benchmark
 * records): launch choices measured at first use -- the schedule of the 1D float transport
 * sweep per (grid, number of problems, nodes) class, and the form of the tensor-core operator's
 * GEMM (one CTA per work item, alone or in clusters, or persistent and warp-specialised) per
 * launch shape.  Every candidate computes the same bits, so the choices change speed only.  The
 * environment variable LBE_GEMM_FORM ("persistent", or a cluster size 1, 2 or 4) fixes the GEMM
 * form instead of timing it (for profilers, whose overhead distorts the timing).  buf (host, cap
 * bytes) receives a NUL-terminated string; LBE_BAD_ARG if it does not fit (the text is then
 * truncated). */
lbe_status lbe_tuning_report(lbe_ctx* ctx, char* buf, size_t cap);

/* Test hook for the bounded-wait failure path (0 = off, the default).  While on, every CTA of
 * the tensor-core GEMM first waits on a shared-memory barrier that nothing completes, with a
 * limit of about 1e5 cycles; when the limit passes the CTA raises the failure word, waits
 * (with the normal limit) for the operand copies it has issued, frees its tensor memory and
 * returns, and the call returns LBE_TIMEOUT.  The context stays usable.  Process-wide. */
lbe_status lbe_debug_expire_waits(int on);

/* ---- Binary hard-sphere mixture (Sec. 4) ------------------------------------------------
 * Species A and B: masses m_A, m_B, hard-sphere diameters d_A, d_B (collision diameter
 * (d_a + d_b) / 2), molar fractions chi_A and chi_B = 1 - chi_A.  Velocities are in units
 * of v_mA, the most probable speed of A, so f_a,eq = chi_a (r_a / pi)^(3/2) exp(-r_a |v|^2)
 * with r_a = m_a / m_A (Sec. 4, Eq. Maxwell), and
 *   L_a h = sum_b Q_ab(f_a,eq, h_b) + Q_ab(h_a, f_b,eq)        (Sec. 4, Eq. Boltzmann_lin).
 * The paper cites its spectral method for Q_ab without writing it out; this library derives
 * it from the collision integral.  With mu_b = m_b / (m_a + m_b) and x ⊥ y, the pre- and
 * post-collision velocities are v* = v + x + y, v' = v + 2 mu_b x, v*' = v + (mu_b - mu_a) x + y,
 * and hard spheres give the constant Carleman kernel d_ab^2.  The gain's kernel modes are
 *   beta_ab(l, m) = sum_p w'_p phi((2 mu_b xi_l + (mu_b - mu_a) xi_m) . e_p) psi_p(m),
 * with the single-species phi, psi, hemisphere rule, truncation R and Nyquist zeroing; equal
 * masses and diameters reproduce the single-species operator exactly.  Unless the masses are
 * equal, phi's argument mixes the two spectra, so the gain is no sum of products of
 * transforms: the library builds the operator once per (mixture, grid) as a dense FP64
 * matrix on the device (O(nv^6 M) work and about 8 nv^6 bytes of temporary device memory)
 * and applies it as an FP64 GEMM.
 * delta = p0 l / (mu v_m) with v_m = sqrt(2 kT / m), m = chi_A m_A + chi_B m_B, and mu the
 * first Chapman-Enskog approximation of the mixture viscosity (the approximation under which
 * the single-species nu_bar = 1.25 delta of Sec. 2.5 holds).
 */
typedef struct {
    double mass_ratio;  /* m_B / m_A > 0                                                       */
    double diam_ratio;  /* d_B / d_A > 0                                                       */
    double chi_A;       /* molar fraction of A, 0 < chi_A < 1                                  */
} lbe_mixture;

/* Poiseuille flow of a mixture (Sec. 4; S_a = v3 f_a,eq, X_P = -1) between plates (geom.dim = 1:
 * the half channel, 2 <= ns <= 1000 sections, grid_kind, diffuse wall, symmetry plane) or through
 * a rectangular duct (geom.dim = 2: 3 <= nx, ny <= 256 cells of [0, width] x [0, 1], diffuse
 * walls; each species' Poisson solve runs in one thread block). */
typedef struct {
    lbe_mixture mix;
    lbe_geometry geom;
    double delta;
    double N_A, N_B;     /* SIS tuning; <= 0 selects N_a = int nu_a,eq f_a,eq dv / (delta chi_a)  */
    int nv;              /* a multiple of 4, 4..32                                              */
    double vmax;
    int M;               /* power of two, 2..64                                                 */
    double R;            /* Carleman truncation radius > 0                                      */
    lbe_scheme scheme;
    double eps;          /* stop when all four flow rates change by < eps relative; 0 = never   */
    int max_iter;        /* cap on all iterations                                               */
    lbe_precision precision; /* LBE_FP64; LBE_DF32: the operator's GEMM in double-float arithmetic
                          * on the FP32 pipes (about 1e-13 of the scale from FP64), the rest FP64;
                          * LBE_BF16: the operator as a tcgen05 BF16 hi/lo GEMM with
                          * float accumulation (everything else FP64), stopping when the four
                          * changes fall below eps times the larger molecular flow rate;
                          * LBE_BF16_REFINED: such iterations down to their floor (changes below
                          * 1e-5 of that scale, or no longer shrinking for three iterations),
                          * then defect correction: an FP64-class (LBE_DF32) iteration h' = Phi(h)
                          * (its change is the FP64 stopping test), and its error
                          * e = G (e + h' - h) solved by the source-free iteration on the tensor
                          * cores; h = h' + e                                                   */
    double solid_fraction;   /* > 0 (ducts only, nx = ny): instead of the duct, the periodic unit
                          * cell of a square array of cylinders -- a centred circle of this area
                          * (below 0.78) as a staircase of solid cells, diffuse walls, periodic
                          * sides (config of Sec. 4's porous media); the sweep takes a periodic
                          * neighbour not yet swept from the previous sweep (a converged
                          * iteration satisfies the periodic scheme), and the diffusion
                          * correction acts on the fluid cells whose eight neighbours are fluid
                          * (solved by conjugate gradients), the others held at the kinetic U.
                          * Solid cells hold h = 0 and U = 0; the operator acts on the fluid
                          * cells only.  The sweep's lag makes its last half step g part of the
                          * iteration's state; LBE_BF16_REFINED's correction then runs on the
                          * pair (h, g)                                                        */
} lbe_mix_problem;

typedef struct {
    double M_A, M_B;     /* molecular flow rates M_a = sqrt(m / m_A) (1/A) int U_a (Sec. 4): plates
                          * 2 int_{-1/2}^0 U_a dx1, ducts the cell mean                          */
    double Q_A, Q_B;     /* heat flow rates, q_a = int (r_a |v|^2 - 5/2) v3 h_a dv                  */
    int iters;           /* all iterations                                                          */
    int status;
    double N_A, N_B;     /* the tuning used                                                        */
    int fp64_iters;      /* iterations with the FP64 operator                                      */
} lbe_mix_result;

/* Tables of one mixture on one grid: out4 (host, 4 doubles) receives b_AA at delta = 1 (the
 * hard-sphere strength per unit solid angle, B = b_ab |v - v*|, b_ab = b_AA d_ab^2 / d_A^2),
 * N_A, N_B (Sec. 4's N_a equation) and mu1 (units m_A = kT = d_A = 1); nu_out (host,
 * [2][nv^3] or NULL) receives nu_A, nu_B at delta = 1.  Builds (and caches) the operator. */
lbe_status lbe_mix_info(lbe_ctx* ctx, const lbe_mixture* mix, int nv, double vmax, int M, double R,
                        double* out4, double* nu_out);

/* L+_a and L_a = L+_a - delta nu_a h_a for `cells` cells (device pointers, [cells][nv^3]
 * double each, full velocity grid; LA, LB may be NULL) on `stream` (NULL: the context's).
 * Asynchronous; LBE_BAD_ARG for invalid sizes, LBE_OOM when the operator does not fit. */
lbe_status lbe_mix_apply_L(lbe_ctx* ctx, const lbe_mixture* mix, int nv, double vmax, int M, double R,
                           int cells, double delta, const double* hA, const double* hB, double* LplusA,
                           double* LA, double* LplusB, double* LB, void* stream);

/* Solve one mixture problem by the CIS or the SIS of Eqs. LBE2_true1 / LBE2_true2 (plates: the
 * equations integrated once across the half channel; ducts: one Poisson equation per species,
 * the ring of wall-adjacent cells held at the kinetic U).  On the device h keeps one value per
 * orbit of the parity group ({1, R2, R3, R2 R3} plates, {1, R3} ducts).  U_out (host,
 * [2][cells] or NULL) receives U_A, U_B of the returned h; h_out (host, [2][cells][nv^3] or
 * NULL) receives h_A, h_B; cells = ns + 1 or nx ny.
 * Returns the result's status: LBE_OK, LBE_NOT_CONVERGED (max_iter reached or eps = 0),
 * LBE_NAN (a non-finite flow rate), LBE_BAD_ARG, LBE_OOM. */
lbe_status lbe_mix_solve(lbe_ctx* ctx, const lbe_mix_problem* pb, lbe_mix_result* out, double* U_out,
                         double* h_out);

#ifdef __cplusplus
}
#endif

#endif /* LBE_H */

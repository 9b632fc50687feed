// Internal declarations of the GB300 linearized-Boltzmann library (host side).
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <complex>
#include <condition_variable>
#include <cstdint>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/lbe.h"

namespace lbe {

// ---------------------------------------------------------------------------------------
// Velocity grid and collision-operator tables (one per (nv, vmax, M, R)).
// Built on the host in double from the formulas of the discrete operator (see lbe.h):
//   mult[p]  = (psi_p + i phi_p) / nv^3   for p < M, mult[M] = G_hat / nv^3 (real)
//   ab[p]    = (w'_p A_p, w'_p B_p)       gain weights in physical space, w'_p = 2 b w_p
//   nu1      = nu_eq at delta = 1,  feq = f_eq
// Device copies in double and float.  The BF16 tensor path keeps its own operands.
// ---------------------------------------------------------------------------------------
struct HostTables {
    int nv = 0, M = 0;
    double vmax = 0, R = 0, dv = 0;
    std::vector<double> v;                  // [nv] midpoint nodes
    std::vector<double> feq, nu1;           // [nv^3]
    std::vector<double> mult;               // [(M+1)][nv^3][2]
    std::vector<double> ab;                 // [M][nv^3][2]
    double cU = 0, cq = 0;                  // sum v3^2 f_eq dv^3, sum (|v|^2-5/2) v3^2 f_eq dv^3
    int sym_reps1 = 0, sym_reps2 = 0;       // representatives per reflection group (0: unavailable)
};

void build_host_tables(HostTables& t, int nv, double vmax, int M, double R);
// pieces of the same construction (tables.cpp): phi(s) = 2 int_0^R r cos(r s) dr,
// psi(a) = 4 pi R J1(R a) / a, the separable DFT of an n^3 array (sign -1 forward, +1 inverse,
// no scaling), and the hemisphere rule (directions e[3 p + i], weights w[p] summing to 2 pi,
// ring-major order)
double carleman_phi(double s, double R);
double carleman_psi(double a, double R);
void host_dft3(std::vector<std::complex<double>>& a, int n, int sign);
void hemisphere_rule(int M, std::vector<double>& e, std::vector<double>& w);

struct TcOperands;  // tensor-core operands (fsm_dense.cu)
struct MixOp;       // binary-mixture operator (mixture.cu)

// Launch choices made by measurement at first use (the autotuner): the schedule of the 1D
// float transport sweep per (grid, problems, nodes) class.  Every choice computes the same
// bits, so tuning changes speed only.
struct Tuning {
    std::mutex mu;
    std::map<long long, int> sweep;  // key -> schedule (0 staged, 1 register ring, 2 shared ring)
    std::vector<std::string> log;    // one line per decision (lbe_tuning_report)
    // the context's side stream (if any): the tuner waits for it, so that overlapping work does
    // not distort its timings
    cudaStream_t side = nullptr;
};

struct DevTables {
    int nv = 0, M = 0;
    double vmax = 0, R = 0, dv = 0;
    double cU = 0, cq = 0;
    int sym_reps1 = 0, sym_reps2 = 0;
    // double
    double* feq_d = nullptr; double* nu1_d = nullptr; double* mult_d = nullptr; double* ab_d = nullptr;
    double* vel_d = nullptr;  // [nv] nodes
    // float
    float* feq_f = nullptr; float* nu1_f = nullptr; float* mult_f = nullptr; float* ab_f = nullptr;
    float* vel_f = nullptr;
    // per orbit of the plate parity (orbit layout, sweep.h): {v3 f_eq, v1 v3, the sum of
    // nu_eq over the orbit's four points, 0} at its representative
    float4* orb_f = nullptr;
    // double-float (hi, lo float pairs; complex tables as re.hi, re.lo, im.hi, im.lo)
    float* feq_x = nullptr; float* nu1_x = nullptr; float* mult_x = nullptr; float* ab_x = nullptr;
    TcOperands* tc = nullptr;
    Tuning* tuning = nullptr;
    size_t bytes = 0;
};

// ---------------------------------------------------------------------------------------
// Spatial description of one problem as seen by the kernels.
// ---------------------------------------------------------------------------------------
struct SweepGeom {
    int dim = 1;
    int cells = 0;          // 1D: ns+1 nodes, 2D: nx*ny
    int nx = 0, ny = 0;     // 2D
    // 1D march coefficients (double), node i in [0, n): fwd (v1 > 0) and bwd (v1 < 0)
    std::vector<double> x;                  // node coordinates (1D) / cell centres x (2D)
    std::vector<double> fa, fb, fc;         // v1 > 0 march, coefficient of h_i, h_{i-1}, h_{i-2}
    std::vector<double> ba, bb, bc;         // v1 < 0 march (h_i, h_{i+1}, h_{i+2}); last uses ghost
    std::vector<double> trap;               // 1D trapezoid weights for M = 2 int U dx
    // 2D: coefficients along a march of n cells starting at an inflow face
    std::vector<double> xa, xb, xc, ya, yb, yc;
};

void build_sweep_geom(SweepGeom& g, const lbe_problem& pb);

// ---------------------------------------------------------------------------------------
// Context.
// ---------------------------------------------------------------------------------------
struct Job {
    uint64_t ticket = 0;
    lbe_problem pb{};
    lbe_result res{};
    int done = 0;
    std::atomic<int> cancel{0};  // set by lbe_cancel; the service retires the job at its next boundary
    double t_submit = 0;  // seconds on the service clock
};

// Grow-only device workspace carved into 256-byte aligned pieces; reused across calls so
// repeated solves allocate nothing once warm.
struct Arena {
    void* base = nullptr;
    size_t cap = 0;
    size_t off = 0;
};

// process-wide counters (lbe_get_stats)
extern std::atomic<unsigned long long> g_launches, g_h2d, g_d2h, g_levals;
// optional event timing of the tensor-core GEMM (lbe_set_kernel_timing)
extern std::atomic<int> g_time_kernels;
// test hook of the GEMM's bounded waits (lbe_debug_expire_waits)
extern std::atomic<int> g_expire_waits;
void add_gemm_time(double ms);
void get_gemm_time(unsigned long long* n, double* ms);
// the same for the transport-sweep launches of the solves (false: timing off or capturing)
bool sweep_timing_begin(cudaStream_t s, cudaEvent_t* ev);
void sweep_timing_end(cudaStream_t s, cudaEvent_t* ev, double bytes);

struct Ctx {
    int device = 0;
    size_t budget = 0;
    size_t used = 0;
    std::string last_error;
    std::mutex tables_mu;
    std::map<std::string, std::unique_ptr<DevTables>> tables;
    cudaStream_t stream = nullptr;      // stream of the synchronous calls
    cudaStream_t own_stream = nullptr;  // created by lbe_create (the highest stream priority)
    // low-priority stream for work that overlaps the synchronous calls' critical path (the
    // refined solves' base evaluations), created at first use
    cudaStream_t side_stream = nullptr;
    Arena solve_arena, apply_arena;
    // binary-mixture operators by (mixture, grid, layout) (mixture.cu)
    std::map<std::string, MixOp*> mix_ops;
    Arena refine_arena[3];  // refined solves: FP64 batch, low-precision batch, work buffers
    // serving
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Job*> queue;
    std::map<uint64_t, std::unique_ptr<Job>> jobs;
    std::atomic<uint64_t> next_ticket{1};
    std::thread service;
    bool stop = false;
    bool service_started = false;
    int max_active = 64;
};

// tables
DevTables* get_tables(Ctx* c, int nv, double vmax, int M, double R, lbe_status* st);
std::string tables_key(int nv, double vmax, int M, double R);
double default_R(double vmax);

// memory accounting
lbe_status dev_alloc(Ctx* c, void** p, size_t bytes);
void dev_free(Ctx* c, void* p, size_t bytes);
lbe_status arena_reserve(Ctx* c, Arena& a, size_t bytes);  // resets the carve offset
void* arena_take(Arena& a, size_t bytes);                  // nullptr when it does not fit
void arena_release(Ctx* c, Arena& a);

// streaming multiprocessors of the current device (queried once per device); grid-stride
// kernels launch a multiple of it
int sm_count();

// status helpers
lbe_status cuda_status(Ctx* c, cudaError_t e, const char* where);
lbe_status bad_arg(Ctx* c, const std::string& what);
lbe_status validate_problem(Ctx* c, const lbe_problem& pb);

}  // namespace lbe

// The opaque handle of include/lbe.h is the context itself.
struct lbe_ctx : public lbe::Ctx {};

// C ABI (include/lbe.h): context, tables, validation, the CIS/SIS solve driver.
//
// One SIS iteration of a batch of problems that share a velocity grid (Sec. 2.2):
//   fsm (A1-A3)   L+ h, L h for the cells of every unfinished problem
//   lmoments (A4) G_j = 2 sum v_j v3 (L h + N delta h) dv^3            [SIS only]
//   sweep (A5)    h^(k+1/2) from nu h + v.grad h = L+ h + S
//   moments (A6)  U3, q3, W1, W2, X12 of h^(k+1/2)
//   sis_update (A7-A8)  diffusion correction, flow rates, convergence flags
//   correct (A8)  h^(k+1) = h^(k+1/2) + 2 dU v3 f_eq
// The flags come back to the host once per iteration; finished problems drop out of the
// active list and stop iterating.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "lbe_internal.h"
#include "sweep.h"
#include "batch.h"

namespace lbe {

lbe_status cuda_status(Ctx* c, cudaError_t e, const char* where) {
    if (e == cudaSuccess) return LBE_OK;
    if (c) c->last_error = std::string(where) + ": " + cudaGetErrorString(e);
    if (e == cudaErrorMemoryAllocation) return LBE_OOM;
    return LBE_INTERNAL;
}

int sm_count() {
    static std::atomic<int> cache[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
    int n = cache[dev].load();
    if (n > 0) return n;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 152;
    cache[dev].store(n);
    return n;
}

lbe_status bad_arg(Ctx* c, const std::string& what) {
    if (c) c->last_error = what;
    return LBE_BAD_ARG;
}

lbe_status dev_alloc(Ctx* c, void** p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) return LBE_OK;
    if (c->used + bytes > c->budget) {
        c->last_error = "HBM budget exceeded";
        return LBE_OOM;
    }
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return cuda_status(c, e, "cudaMalloc");
    }
    c->used += bytes;
    return LBE_OK;
}

void dev_free(Ctx* c, void* p, size_t bytes) {
    if (!p) return;
    cudaFree(p);
    c->used -= std::min(bytes, c->used);
}

std::atomic<unsigned long long> g_launches{0}, g_h2d{0}, g_d2h{0}, g_levals{0};
std::atomic<int> g_time_kernels{0};
std::atomic<int> g_expire_waits{0};
static std::mutex g_time_mu;
static unsigned long long g_gemm_n = 0;
static double g_gemm_ms = 0.0;
void add_gemm_time(double ms) {
    std::lock_guard<std::mutex> lk(g_time_mu);
    ++g_gemm_n;
    g_gemm_ms += ms;
}
void get_gemm_time(unsigned long long* n, double* ms) {
    std::lock_guard<std::mutex> lk(g_time_mu);
    *n = g_gemm_n;
    *ms = g_gemm_ms;
}

// Transport-sweep launches timed inside solves: events are recorded on the solve's stream and
// resolved (waited for) only when the counters are read.
struct PendingSweep {
    cudaEvent_t a, b;
    double bytes;
};
static std::vector<PendingSweep> g_sweep_pending;
static unsigned long long g_sweep_n = 0;
static double g_sweep_ms = 0.0, g_sweep_bytes = 0.0;
bool sweep_timing_begin(cudaStream_t s, cudaEvent_t* ev) {
    if (!g_time_kernels.load()) return false;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return false;
    if (cudaEventCreate(&ev[0]) != cudaSuccess) return false;
    if (cudaEventCreate(&ev[1]) != cudaSuccess) {
        cudaEventDestroy(ev[0]);
        return false;
    }
    cudaEventRecord(ev[0], s);
    return true;
}
void sweep_timing_end(cudaStream_t s, cudaEvent_t* ev, double bytes) {
    cudaEventRecord(ev[1], s);
    std::lock_guard<std::mutex> lk(g_time_mu);
    g_sweep_pending.push_back({ev[0], ev[1], bytes});
}
static void resolve_sweep_times() {
    std::lock_guard<std::mutex> lk(g_time_mu);
    for (auto& p : g_sweep_pending) {
        float ms = 0.f;
        if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
            ++g_sweep_n;
            g_sweep_ms += ms;
            g_sweep_bytes += p.bytes;
        }
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    g_sweep_pending.clear();
}

lbe_status arena_reserve(Ctx* c, Arena& a, size_t bytes) {
    a.off = 0;
    if (bytes <= a.cap) return LBE_OK;
    if (a.base) {
        cudaStreamSynchronize(c->stream);
        dev_free(c, a.base, a.cap);
        a.base = nullptr;
        a.cap = 0;
    }
    const size_t want = bytes + bytes / 8;  // headroom for slightly larger later requests
    lbe_status st = dev_alloc(c, &a.base, want);
    if (st != LBE_OK) {
        st = dev_alloc(c, &a.base, bytes);
        if (st != LBE_OK) return st;
        a.cap = bytes;
        return LBE_OK;
    }
    a.cap = want;
    return LBE_OK;
}

void* arena_take(Arena& a, size_t bytes) {
    const size_t off = (a.off + 255) & ~(size_t)255;
    if (off + bytes > a.cap) return nullptr;
    a.off = off + bytes;
    return (char*)a.base + off;
}

void arena_release(Ctx* c, Arena& a) {
    if (a.base) dev_free(c, a.base, a.cap);
    a.base = nullptr;
    a.cap = a.off = 0;
}

lbe_status validate_problem(Ctx* c, const lbe_problem& pb) {
    const auto& g = pb.geom;
    if (g.dim != 1 && g.dim != 2) return bad_arg(c, "geom.dim must be 1 or 2");
    if (g.dim == 1 && (g.ns < 2 || g.ns > 100000)) return bad_arg(c, "geom.ns must be in [2, 100000]");
    if (g.dim == 1 && g.grid_kind != 0 && g.grid_kind != 1) return bad_arg(c, "geom.grid_kind must be 0 or 1");
    if (g.dim == 2 && (g.nx < 3 || g.ny < 3 || (long)g.nx * g.ny > 1000000))
        return bad_arg(c, "geom.nx, geom.ny must be >= 3");
    if (g.dim == 2 && !(g.width > 0)) return bad_arg(c, "geom.width must be > 0");
    if (!(pb.delta >= 0) || !std::isfinite(pb.delta)) return bad_arg(c, "delta must be finite and >= 0");
    if (pb.nv != 8 && pb.nv != 16 && pb.nv != 24 && pb.nv != 32) return bad_arg(c, "nv must be 8, 16, 24 or 32");
    if (!(pb.vmax > 0) || !std::isfinite(pb.vmax)) return bad_arg(c, "vmax must be > 0");
    if (pb.M < 2 || pb.M > 64 || (pb.M & (pb.M - 1))) return bad_arg(c, "M must be a power of two in [2, 64]");
    if (pb.R > 2.0 * pb.vmax) return bad_arg(c, "R must be <= 2 vmax");
    if (pb.forcing != LBE_POISEUILLE && pb.forcing != LBE_THERMAL_TRANSPIRATION) return bad_arg(c, "bad forcing");
    if (pb.scheme != LBE_CIS && pb.scheme != LBE_SIS) return bad_arg(c, "bad scheme");
    if (pb.precision != LBE_FP64 && pb.precision != LBE_FP32 && pb.precision != LBE_BF16_REFINED &&
        pb.precision != LBE_FP32_REFINED && pb.precision != LBE_BF16)
        return bad_arg(c, "bad precision");
    if (pb.precision == LBE_BF16 && pb.M < 8) return bad_arg(c, "LBE_BF16 needs M >= 8");
    if (!(pb.eps >= 0)) return bad_arg(c, "eps must be >= 0");
    if (pb.max_iter < 1) return bad_arg(c, "max_iter must be >= 1");
    return LBE_OK;
}

// ---------------------------------------------------------------------------------------
// tables
// ---------------------------------------------------------------------------------------
std::string tables_key(int nv, double vmax, int M, double R) {
    char b[128];
    snprintf(b, sizeof b, "%d/%.17g/%d/%.17g", nv, vmax, M, R);
    return b;
}

template <typename T>
static lbe_status upload(Ctx* c, T** dst, const std::vector<T>& src, size_t* bytes) {
    lbe_status st = dev_alloc(c, (void**)dst, src.size() * sizeof(T));
    if (st != LBE_OK) return st;
    *bytes += src.size() * sizeof(T);
    return cuda_status(c, cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice),
                       "upload");
}

static std::vector<float> to_f(const std::vector<double>& a) { return std::vector<float>(a.begin(), a.end()); }
// each double as the float pair (hi, lo) with hi = fl(x), lo = fl(x - hi)
static std::vector<float> to_df(const std::vector<double>& a) {
    std::vector<float> o(2 * a.size());
    for (size_t i = 0; i < a.size(); ++i) {
        o[2 * i] = (float)a[i];
        o[2 * i + 1] = (float)(a[i] - (double)o[2 * i]);
    }
    return o;
}

DevTables* get_tables(Ctx* c, int nv, double vmax, int M, double R, lbe_status* st) {
    if (R <= 0) R = default_R(vmax);
    std::lock_guard<std::mutex> lk(c->tables_mu);
    const std::string key = tables_key(nv, vmax, M, R);
    auto it = c->tables.find(key);
    if (it != c->tables.end()) {
        *st = LBE_OK;
        return it->second.get();
    }
    HostTables h;
    build_host_tables(h, nv, vmax, M, R);
    auto t = std::make_unique<DevTables>();
    t->nv = nv;
    t->M = M;
    t->vmax = vmax;
    t->R = R;
    t->dv = h.dv;
    t->cU = h.cU;
    t->cq = h.cq;
    t->sym_reps1 = h.sym_reps1;
    t->sym_reps2 = h.sym_reps2;
    t->tuning = new Tuning();
    size_t b = 0;
    lbe_status s = LBE_OK;
    if (s == LBE_OK) s = upload(c, &t->feq_d, h.feq, &b);
    if (s == LBE_OK) s = upload(c, &t->nu1_d, h.nu1, &b);
    if (s == LBE_OK) s = upload(c, &t->mult_d, h.mult, &b);
    if (s == LBE_OK) s = upload(c, &t->ab_d, h.ab, &b);
    if (s == LBE_OK) s = upload(c, &t->vel_d, h.v, &b);
    if (s == LBE_OK) s = upload(c, &t->feq_f, to_f(h.feq), &b);
    if (s == LBE_OK) s = upload(c, &t->nu1_f, to_f(h.nu1), &b);
    if (s == LBE_OK) s = upload(c, &t->mult_f, to_f(h.mult), &b);
    if (s == LBE_OK) s = upload(c, &t->ab_f, to_f(h.ab), &b);
    if (s == LBE_OK) s = upload(c, &t->vel_f, to_f(h.v), &b);
    if (s == LBE_OK) {  // orbit constants of the plate parity (the correction step)
        const int H = nv / 2;
        std::vector<float> orb((size_t)nv * H * H * 4, 0.f);
        for (int i1 = 0; i1 < nv; ++i1)
            for (int j2 = 0; j2 < H; ++j2)
                for (int j3 = 0; j3 < H; ++j3) {
                    const long q = ((long)i1 * H + j2) * H + j3;
                    const long va = ((long)i1 * nv + j2) * nv + j3, vb = ((long)i1 * nv + nv - 1 - j2) * nv + j3;
                    const long vc = ((long)i1 * nv + j2) * nv + nv - 1 - j3;
                    const long vd = ((long)i1 * nv + nv - 1 - j2) * nv + nv - 1 - j3;
                    orb[4 * q + 0] = (float)(h.v[j3] * h.feq[va]);
                    orb[4 * q + 1] = (float)(h.v[i1] * h.v[j3]);
                    orb[4 * q + 2] = (float)(h.nu1[va] + h.nu1[vb] + h.nu1[vc] + h.nu1[vd]);
                }
        float* of = nullptr;
        s = upload(c, &of, orb, &b);
        t->orb_f = reinterpret_cast<float4*>(of);
    }
    if (s == LBE_OK) s = upload(c, &t->feq_x, to_df(h.feq), &b);
    if (s == LBE_OK) s = upload(c, &t->nu1_x, to_df(h.nu1), &b);
    if (s == LBE_OK) s = upload(c, &t->mult_x, to_df(h.mult), &b);
    if (s == LBE_OK) s = upload(c, &t->ab_x, to_df(h.ab), &b);
    t->bytes = b;
    *st = s;
    if (s != LBE_OK) {  // give back what was uploaded before the failure
        for (void* p : {(void*)t->feq_d, (void*)t->nu1_d, (void*)t->mult_d, (void*)t->ab_d, (void*)t->vel_d,
                        (void*)t->feq_f, (void*)t->nu1_f, (void*)t->mult_f, (void*)t->ab_f, (void*)t->vel_f,
                        (void*)t->orb_f, (void*)t->feq_x, (void*)t->nu1_x, (void*)t->mult_x, (void*)t->ab_x})
            if (p) cudaFree(p);
        c->used -= std::min(b, c->used);
        delete t->tuning;
        return nullptr;
    }
    DevTables* raw = t.get();
    c->tables[key] = std::move(t);
    return raw;
}

// ---------------------------------------------------------------------------------------
// geometry
// ---------------------------------------------------------------------------------------
static void backward_coeffs(double xm2, double xm1, double x0, double& a, double& b, double& cc) {
    const double h1 = x0 - xm1, h2 = xm1 - xm2;
    a = (2.0 * h1 + h2) / (h1 * (h1 + h2));
    b = -(h1 + h2) / (h1 * h2);
    cc = h1 / (h2 * (h1 + h2));
}

// march coefficients along increasing positions pos[0..n-1], pos[0] the inflow boundary
static void march_coeffs(const std::vector<double>& pos, std::vector<double>& a, std::vector<double>& b,
                         std::vector<double>& cc) {
    const size_t n = pos.size();
    a.assign(n, 0.0);
    b.assign(n, 0.0);
    cc.assign(n, 0.0);
    a[1] = 1.0 / (pos[1] - pos[0]);
    b[1] = -a[1];
    for (size_t i = 2; i < n; ++i) backward_coeffs(pos[i - 2], pos[i - 1], pos[i], a[i], b[i], cc[i]);
}

void build_sweep_geom(SweepGeom& g, const lbe_problem& pb) {
    g.dim = pb.geom.dim;
    if (g.dim == 1) {
        const int ns = pb.geom.ns, n = ns + 1;
        g.cells = n;
        g.x.resize(n);
        for (int i = 0; i < n; ++i) {
            if (pb.geom.grid_kind == 1) {
                const double s = i / (2.0 * ns);
                g.x[i] = (10.0 - 15.0 * s + 6.0 * s * s) * s * s * s - 0.5;
            } else {
                g.x[i] = -0.5 + 0.5 * i / ns;
            }
        }
        march_coeffs(g.x, g.fa, g.fb, g.fc);
        g.ba.assign(n, 0.0);
        g.bb.assign(n, 0.0);
        g.bc.assign(n, 0.0);
        for (int i = n - 2; i >= 0; --i) {
            const double y0 = -g.x[i], y1 = -g.x[i + 1];
            const double y2 = (i + 2 <= n - 1) ? -g.x[i + 2] : g.x[n - 2];  // mirror ghost
            backward_coeffs(y2, y1, y0, g.ba[i], g.bb[i], g.bc[i]);
        }
        g.trap.assign(n, 0.0);
        for (int i = 0; i + 1 < n; ++i) {
            const double w = g.x[i + 1] - g.x[i];  // M = 2 int_{-1/2}^0 U dx (trapezoid)
            g.trap[i] += w;
            g.trap[i + 1] += w;
        }
    } else {
        const int nx = pb.geom.nx, ny = pb.geom.ny;
        g.cells = nx * ny;
        g.nx = nx;
        g.ny = ny;
        const double dx = pb.geom.width / nx, dy = 1.0 / ny;
        std::vector<double> px(nx + 1), py(ny + 1), a, b, cc;
        px[0] = 0;
        py[0] = 0;
        for (int i = 0; i < nx; ++i) px[i + 1] = (i + 0.5) * dx;
        for (int j = 0; j < ny; ++j) py[j + 1] = (j + 0.5) * dy;
        march_coeffs(px, a, b, cc);
        g.xa.assign(a.begin() + 1, a.end());
        g.xb.assign(b.begin() + 1, b.end());
        g.xc.assign(cc.begin() + 1, cc.end());
        march_coeffs(py, a, b, cc);
        g.ya.assign(a.begin() + 1, a.end());
        g.yb.assign(b.begin() + 1, b.end());
        g.yc.assign(cc.begin() + 1, cc.end());
        g.trap.assign(g.cells, 1.0 / g.cells);
    }
}

// ---------------------------------------------------------------------------------------
// batch state
// ---------------------------------------------------------------------------------------
lbe_status batch_init(Batch& B, Ctx* c, const lbe_problem* pbs, int n, Arena* arena,
                      cudaStream_t stream) {
    B.c = c;
    B.arena = arena;
    B.s = stream;
    B.njobs = n;
    B.pbs.assign(pbs, pbs + n);
    const lbe_problem& p0 = pbs[0];
    lbe_status st;
    B.t = get_tables(c, p0.nv, p0.vmax, p0.M, p0.R, &st);
    if (!B.t) return st;
    B.prec = p0.precision;
    if (B.prec == LBE_BF16_REFINED || B.prec == LBE_FP32_REFINED || B.prec == LBE_BF16) B.prec = LBE_FP32;
    const int eb = B.prec == LBE_FP64 ? 8 : 4;
    const long n3 = (long)p0.nv * p0.nv * p0.nv;
    std::vector<double> coef, dcell, ndcell;
    B.geo.resize(n);
    long work = 0;
    for (int j = 0; j < n; ++j) {
        const lbe_problem& pb = pbs[j];
        build_sweep_geom(B.geo[j], pb);
        SweepGeom& g = B.geo[j];
        SweepJobDev s{};
        s.cell_off = B.cells;
        s.ncell = g.cells;
        s.nx = g.nx;
        s.ny = g.ny;
        s.forcing = pb.forcing;
        s.delta = pb.delta;
        s.coef_off = (int)coef.size();
        if (g.dim == 1) {
            for (auto* v : {&g.fa, &g.fb, &g.fc, &g.ba, &g.bb, &g.bc}) coef.insert(coef.end(), v->begin(), v->end());
        } else {
            for (auto* v : {&g.xa, &g.xb, &g.xc, &g.ya, &g.yb, &g.yc}) coef.insert(coef.end(), v->begin(), v->end());
        }
        SisJobDev q{};
        q.cell_off = B.cells;
        q.ncell = g.cells;
        q.dim = g.dim;
        q.nx = g.nx;
        q.ny = g.ny;
        q.width = pb.geom.width;
        q.scheme = pb.scheme == LBE_SIS ? 1 : 0;
        const double Nn = pb.N > 0 ? pb.N : 1.25;
        q.ndsig = Nn * pb.delta * (pb.forcing == LBE_POISEUILLE ? 1.0 : 0.0);
        q.eps = pb.eps;
        q.max_iter = pb.max_iter;
        q.coef_off = (int)coef.size();
        if (g.dim == 1) {
            {
            // the march divides by fa at every node: store 1/fa (block [1/fa | fb | fc | x])
            std::vector<double> ifa(g.fa.size());
            for (size_t i = 0; i < ifa.size(); ++i) ifa[i] = g.fa[i] != 0.0 ? 1.0 / g.fa[i] : 0.0;
            for (auto* v : {&ifa, &g.fb, &g.fc, &g.x}) coef.insert(coef.end(), v->begin(), v->end());
        }
        } else {
            const int mx = g.nx - 2, my = g.ny - 2;
            for (int p = 0; p < mx; ++p)
                for (int a = 0; a < mx; ++a) coef.push_back(std::sin(M_PI * (p + 1.0) * (a + 1.0) / (mx + 1.0)));
            for (int p = 0; p < my; ++p)
                for (int a = 0; a < my; ++a) coef.push_back(std::sin(M_PI * (p + 1.0) * (a + 1.0) / (my + 1.0)));
            const double dx = pb.geom.width / g.nx, dy = 1.0 / g.ny;
            for (int p = 0; p < mx; ++p)
                for (int r = 0; r < my; ++r) {
                    const double sx = std::sin(M_PI * (p + 1.0) / (2.0 * (mx + 1.0)));
                    const double sy = std::sin(M_PI * (r + 1.0) / (2.0 * (my + 1.0)));
                    coef.push_back(-4.0 / (dx * dx) * sx * sx - 4.0 / (dy * dy) * sy * sy);
                }
            q.work_off = work;
            work += 2L * mx * my;
        }
        q.trap_off = (int)coef.size();
        coef.insert(coef.end(), g.trap.begin(), g.trap.end());
        for (int i = 0; i < g.cells; ++i) {
            dcell.push_back(pb.delta);
            ndcell.push_back(Nn * pb.delta);
        }
        B.sj.push_back(s);
        B.ij.push_back(q);
        B.cell_off.push_back(B.cells);
        B.cells += g.cells;
    }
    const size_t vol = (size_t)B.cells * n3 * eb;
    size_t scr = fsm_cc_scratch_bytes(*B.t, (int)std::min<long>(B.cells, 1L << 30), eb, &B.chunk);
    struct Piece {
        DevBuf* b;
        size_t n;
    };
    const Piece pieces[] = {{&B.h, vol}, {&B.hh, vol}, {&B.lp, vol}, {&B.lh, vol}, {&B.scratch, scr},
                            {&B.mom, (size_t)B.cells * 5 * 8}, {&B.G, (size_t)B.cells * 2 * 8},
                            {&B.dU, (size_t)B.cells * 8}, {&B.U3, (size_t)B.cells * 8},
                            {&B.delta, (size_t)B.cells * 8}, {&B.nd, (size_t)B.cells * 8},
                            {&B.hmom, (size_t)B.cells * 2 * 8},
                            {&B.coef, coef.size() * 8}, {&B.work, (size_t)std::max<long>(work, 1) * 8},
                            {&B.sjobs, n * sizeof(SweepJobDev)}, {&B.ijobs, n * sizeof(SisJobDev)},
                            {&B.states, n * sizeof(JobState)}, {&B.act, n * sizeof(int)}};
    size_t total = 0;
    for (const Piece& q : pieces) total += (q.n + 255) & ~(size_t)255;
    if ((st = arena_reserve(c, *arena, total)) != LBE_OK) return st;
    for (const Piece& q : pieces) {
        q.b->p = arena_take(*arena, q.n);
        q.b->n = q.n;
        if (!q.b->p) return LBE_INTERNAL;
    }
    cudaStream_t s = stream;
    cudaMemsetAsync(B.h.p, 0, vol, s);  // h^0 = 0
    cudaMemsetAsync(B.hmom.p, 0, B.hmom.n, s);
    cudaMemcpyAsync(B.delta.p, dcell.data(), dcell.size() * 8, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(B.nd.p, ndcell.data(), ndcell.size() * 8, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(B.coef.p, coef.data(), coef.size() * 8, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(B.sjobs.p, B.sj.data(), n * sizeof(SweepJobDev), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(B.ijobs.p, B.ij.data(), n * sizeof(SisJobDev), cudaMemcpyHostToDevice, s);
    B.hstate.assign(n, JobState{});
    cudaMemcpyAsync(B.states.p, B.hstate.data(), n * sizeof(JobState), cudaMemcpyHostToDevice, s);
    g_h2d += (dcell.size() + ndcell.size() + coef.size()) * 8 + n * (sizeof(SweepJobDev) + sizeof(SisJobDev) +
                                                                  sizeof(JobState));
    B.active.resize(n);
    for (int j = 0; j < n; ++j) B.active[j] = j;
    return cuda_status(c, cudaStreamSynchronize(s), "batch_init");
}

// One iteration over the active jobs.  Contiguous active jobs share FSM launches.
template <typename T>
void batch_iterate(Batch& B, bool upload, bool read) {
    cudaStream_t s = B.s;
    const DevTables& t = *B.t;
    const long n3 = (long)t.nv * t.nv * t.nv;
    const int na = (int)B.active.size();
    T* h = B.h.as<T>();
    T* hh = B.hh.as<T>();
    T* lp = B.lp.as<T>();
    T* lh = B.lh.as<T>();
    // contiguous cell spans of the active jobs (by memory position), never mixing plates
    // and ducts: each problem's operator uses its own parity group (plates: odd in v3 and
    // even in v2; ducts: odd in v3), so its arithmetic does not depend on its neighbours
    struct Span {
        long c0, n;
        int dim;
    };
    std::vector<Span> spans;
    {
        std::vector<Span> r;
        for (int j : B.active) r.push_back({B.cell_off[j], (long)B.sj[j].ncell, B.geo[j].dim});
        std::sort(r.begin(), r.end(), [](const Span& a, const Span& b) { return a.c0 < b.c0; });
        for (auto& q : r) {
            if (!spans.empty() && spans.back().c0 + spans.back().n == q.c0 && spans.back().dim == q.dim)
                spans.back().n += q.n;
            else
                spans.push_back(q);
        }
    }
    bool any_sis = false;
    for (int j : B.active) any_sis |= B.pbs[j].scheme == LBE_SIS;
    for (auto& sp : spans) {
        const long c0 = sp.c0;
        const int nc = (int)sp.n;
        const int mode = sp.dim == 1 ? 2 : 1;
        // the orbit layout of this span: 1 plates (a quarter of each cell), 2 ducts (a half)
        const int ql = B.quarter() ? (sp.dim == 1 ? 1 : 2) : 0;
        const bool q = ql != 0;
        const long nq = ql == 1 ? n3 / 4 : (ql == 2 ? n3 / 2 : n3);  // values a cell holds
        if (sizeof(T) == 8 && B.base_h) {
            // L h = L_64(h_base) + L_32(h - h_base): the increment is small, so FP32 suffices
            const long o = c0 * n3, nn = (long)nc * n3;
            if (q)
                range_sub_f32_q((const double*)(h + o), B.base_h + o, B.inc_h + o, nc, n3, nq, s);
            else
                range_sub_f32((const double*)(h + o), B.base_h + o, B.inc_h + o, nn, s);
            if (B.inc_tc) {  // BF16-refined: the increment through the tensor-core operator
                const lbe_status ts = tc_apply_sym(B.c, B.t, mode, nc, B.delta.as<double>() + c0, B.inc_h + o,
                                                   B.inc_lp + o, B.inc_lh + o, s, false, nullptr, nullptr, nullptr,
                                                   q);
                if (ts != LBE_OK && B.op_status == LBE_OK) B.op_status = ts;
            } else {
                fsm_cc_apply<float>(t, nc, B.delta.as<double>() + c0, B.inc_h + o, B.inc_lp + o, B.inc_lh + o,
                                    B.inc_scratch, B.inc_chunk, s, mode);
            }
            if (q) {
                range_add_f64_q(B.base_lp + o, B.inc_lp + o, (double*)(lp + o), nc, n3, nq, s);
                range_add_f64_q(B.base_lh + o, B.inc_lh + o, (double*)(lh + o), nc, n3, nq, s);
            } else {
                range_add_f64(B.base_lp + o, B.inc_lp + o, (double*)(lp + o), nn, s);
                range_add_f64(B.base_lh + o, B.inc_lh + o, (double*)(lh + o), nn, s);
            }
        } else if (sizeof(T) == 4 && B.use_tc) {
            // L+ h and the L-moments in one pass; L h itself is not stored
            const lbe_status ts = tc_apply_sym(B.c, B.t, mode, nc, B.delta.as<double>() + c0, (const float*)(h + c0 * n3),
                                               (float*)(lp + c0 * n3), nullptr, s, false, B.nd.as<double>() + c0,
                                               B.G.as<double>() + c0 * 2, B.hmom.as<double>() + c0 * 2,
                                               q);
            if (ts != LBE_OK && B.op_status == LBE_OK) B.op_status = ts;
            continue;
        } else {
            fsm_cc_apply<T>(t, nc, B.delta.as<double>() + c0, h + c0 * n3, lp + c0 * n3, lh + c0 * n3,
                            B.scratch.p, B.chunk, s, mode);
        }
        if (any_sis)
            lmoments<T>(t, nc, lh + c0 * n3, h + c0 * n3, B.nd.as<double>() + c0, B.G.as<double>() + c0 * 2, s, ql);
    }
    // sweeps grouped by dimension
    std::vector<int> act1, act2;
    for (int j : B.active) (B.geo[j].dim == 1 ? act1 : act2).push_back(j);
    // the device active list is [act1..., act2...]
    std::vector<int> ordered(act1);
    ordered.insert(ordered.end(), act2.begin(), act2.end());
    if (upload) {
        cudaMemcpyAsync(B.act.p, ordered.data(), na * sizeof(int), cudaMemcpyHostToDevice, s);
        g_h2d += na * sizeof(int);
    }
    int* dact = B.act.as<int>();
    int mc1 = 0, mc2 = 0;  // largest coefficient block of a job (shared-memory staging)
    for (int j : act1) mc1 = std::max(mc1, 6 * B.sj[j].ncell);
    for (int j : act2) mc2 = std::max(mc2, 3 * (B.sj[j].nx + B.sj[j].ny));
    {  // optional event timing of each sweep launch (algorithmic bytes: rhs in, h out)
        long c1 = 0, c2 = 0;
        for (int j : act1) c1 += B.sj[j].ncell;
        for (int j : act2) c2 += B.sj[j].ncell;
        cudaEvent_t ev[2];
        bool tm = !act1.empty() && sweep_timing_begin(s, ev);
        const int q1 = B.quarter() ? 1 : 0;  // plates in the orbit layout: a quarter of each cell
        launch_sweep<T>(t, 1, (int)act1.size(), mc1, lp, hh, B.sjobs.as<SweepJobDev>(), dact, B.coef.as<double>(), s,
                        q1);
        if (tm) sweep_timing_end(s, ev, 2.0 * sizeof(T) * (double)c1 * (q1 ? n3 / 4 : n3));
        tm = !act2.empty() && sweep_timing_begin(s, ev);
        launch_sweep<T>(t, 2, (int)act2.size(), mc2, lp, hh, B.sjobs.as<SweepJobDev>(), dact + act1.size(),
                        B.coef.as<double>(), s, q1);  // ducts in the orbit layout: a half of each cell
        if (tm) sweep_timing_end(s, ev, 2.0 * sizeof(T) * (double)c2 * (q1 ? n3 / 2 : n3));
    }
    for (auto& sp : spans)
        launch_moments<T>(t, sp.c0, (int)sp.n, hh, B.mom.as<double>(), s, B.quarter() ? (sp.dim == 1 ? 1 : 2) : 0);
    int max_cells = 0;
    for (int j : B.active) max_cells = std::max(max_cells, B.sj[j].ncell);
    launch_sis_update(t, na, B.ijobs.as<SisJobDev>(), dact, B.mom.as<double>(), B.G.as<double>(),
                      B.coef.as<double>(), B.work.as<double>(), B.dU.as<double>(), B.U3.as<double>(),
                      B.states.as<JobState>(), s);
    launch_correct<T>(t, na, hh, h, B.dU.as<double>(), B.extra.p ? B.extra.as<T>() : nullptr,
                      B.sjobs.as<SweepJobDev>(), dact, s, B.states.as<JobState>(),
                      (sizeof(T) == 4 && B.use_tc) ? B.hmom.as<double>() : nullptr, B.nd.as<double>(),
                      B.quarter() ? 1 : 0, max_cells, act2.empty() ? 0 : 1);
    if (read) {
        cudaMemcpyAsync(B.hstate.data(), B.states.p, B.njobs * sizeof(JobState), cudaMemcpyDeviceToHost, s);
        g_d2h += B.njobs * sizeof(JobState);
    }
}

static double host_now() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// Iterations that can be queued before the next convergence check without passing any
// problem's predicted convergence: from the last two changes of each active problem (its
// contraction per iteration) the iterations it still needs, the smallest of them, at most 8.
// Queued iterations leave finished problems untouched (JobState::skip), so a wrong guess
// only costs the extra iterations of the problems still running.
static int predict_chunk(const Batch& B, int left) {
    int k = 8;
    for (int j : B.active) {
        const JobState& st = B.hstate[j];
        if (st.iters < 3) return 1;
        const SisJobDev& q = B.ij[j];
        const double dM = std::fabs(st.M - st.Mprev), dQ = std::fabs(st.Q - st.Qprev);
        const double rel = q.crit == 0 ? std::max(dM / std::fabs(st.M), dQ / std::fabs(st.Q))
                                       : std::max(dM, dQ) / std::max(std::fabs(st.M), std::fabs(st.Q));
        if (!(rel > 0) || !std::isfinite(rel) || q.eps <= 0) {
            if (q.eps > 0) return 1;
        } else {
            const double om = std::min(0.95, std::max(0.05, B.omega.size() > (size_t)j ? B.omega[j] : 0.9));
            const double need = std::log(q.eps / rel) / std::log(om);
            k = std::min(k, std::max(1, (int)std::floor(need)));
        }
        k = std::min(k, std::max(1, q.max_iter - st.iters));
    }
    return std::max(1, std::min(k, left));
}

template <typename T>
static void run_chunk(Batch& B, int K) {
    // the first iteration uploads the active list and runs uncaptured, which also warms every
    // workspace the iteration uses; the rest replay it as a CUDA graph
    batch_iterate<T>(B, true, K == 1);
    if (K == 1) return;
    const int rest = K - 1;
    bool use_graph = B.graphs_ok && rest >= 2 && B.s != nullptr && B.s != cudaStreamLegacy &&
                     B.s != cudaStreamPerThread;
    if (use_graph && (!B.graph || B.graph_key != B.active)) {
        if (B.graph) {
            cudaGraphExecDestroy(B.graph);
            B.graph = nullptr;
        }
        const unsigned long long l0 = g_launches.load(), e0 = g_levals.load();
        cudaGraph_t g = nullptr;
        bool ok = cudaStreamBeginCapture(B.s, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        if (ok) {
            batch_iterate<T>(B, false, false);
            ok = cudaStreamEndCapture(B.s, &g) == cudaSuccess && g != nullptr;
        }
        if (ok) ok = cudaGraphInstantiate(&B.graph, g, 0) == cudaSuccess;
        if (g) cudaGraphDestroy(g);
        B.graph_launches = g_launches.load() - l0;
        B.graph_levals = g_levals.load() - e0;
        g_launches -= B.graph_launches;  // counted per replay below
        g_levals -= B.graph_levals;
        if (!ok) {
            cudaGetLastError();
            if (B.graph) cudaGraphExecDestroy(B.graph);
            B.graph = nullptr;
            B.graphs_ok = false;
            B.op_status = LBE_OK;
            use_graph = false;
        } else {
            B.graph_key = B.active;
        }
    }
    if (use_graph) {
        for (int k = 0; k < rest; ++k) {
            cudaGraphLaunch(B.graph, B.s);
            g_launches += B.graph_launches;
            g_levals += B.graph_levals;
        }
        cudaMemcpyAsync(B.hstate.data(), B.states.p, B.njobs * sizeof(JobState), cudaMemcpyDeviceToHost, B.s);
        g_d2h += B.njobs * sizeof(JobState);
    } else {
        for (int k = 0; k < rest; ++k) batch_iterate<T>(B, false, k == rest - 1);
    }
}

lbe_status batch_run(Batch& B, int max_steps) {
    // a graph holds the workspace addresses of its capture; other calls between two runs may
    // have moved them, so every run captures afresh
    if (B.graph) {
        cudaGraphExecDestroy(B.graph);
        B.graph = nullptr;
    }
    B.graph_key.clear();
    int steps = 0;
    B.t_start = host_now();
    B.t_done.assign(B.njobs, 0.0);
    B.omega.assign(B.njobs, 0.9);
    std::vector<double> last(B.njobs, 0.0);
    while (!B.active.empty() && steps < max_steps) {
        const int K = predict_chunk(B, max_steps - steps);
        if (B.prec == LBE_FP64)
            run_chunk<double>(B, K);
        else
            run_chunk<float>(B, K);
        lbe_status st = cuda_status(B.c, cudaStreamSynchronize(B.s), "iterate");
        if (st == LBE_OK && B.use_tc) st = tc_check(B.c, B.t);
        if (st == LBE_OK) st = B.op_status;
        if (st != LBE_OK) return st;
        std::vector<int> keep;
        const double t = host_now();
        std::vector<int> finished;
        for (int j : B.active) {
            const JobState& js = B.hstate[j];
            // contraction per iteration from successive relative changes
            if (last[j] > 0 && js.rel > 0 && std::isfinite(js.rel))
                B.omega[j] = std::pow(js.rel / last[j], 1.0 / K);
            last[j] = js.rel;
            if (!js.done) {
                keep.push_back(j);
            } else {
                B.t_done[j] = t;
                finished.push_back(j);
            }
        }
        B.active.swap(keep);
        steps += K;
        if (B.on_done && !finished.empty()) B.on_done(finished);
    }
    const double t = host_now();
    for (int j : B.active) B.t_done[j] = t;
    if (B.on_done && !B.active.empty()) B.on_done(B.active);
    return LBE_OK;
}

template void batch_iterate<double>(Batch&, bool, bool);
template void batch_iterate<float>(Batch&, bool, bool);

void fill_result(const Batch& B, int j, lbe_result* r, double secs) {
    const JobState& s = B.hstate[j];
    r->mass_flow = s.M;
    r->heat_flow = s.Q;
    r->iters = s.iters;
    r->last_rel_change = s.rel;
    r->seconds = (j < (int)B.t_done.size() && B.t_done[j] > 0) ? B.t_done[j] - B.t_start : secs;
    r->refinements = 0;
    const lbe_problem& pb = B.pbs[j];
    if (s.nan)
        r->status = LBE_NAN;
    else if (pb.eps > 0 && s.done && s.iters < pb.max_iter)
        r->status = LBE_OK;
    else if (pb.eps > 0 && std::fabs(s.M - s.Mprev) < pb.eps * std::fabs(s.M) &&
             std::fabs(s.Q - s.Qprev) < pb.eps * std::fabs(s.Q))
        r->status = LBE_OK;
    else
        r->status = LBE_NOT_CONVERGED;
}

}  // namespace lbe

using namespace lbe;


extern "C" {

const char* lbe_status_str(lbe_status s) {
    switch (s) {
        case LBE_OK: return "ok";
        case LBE_NOT_CONVERGED: return "not converged";
        case LBE_NAN: return "non-finite flow rate";
        case LBE_BAD_ARG: return "bad argument";
        case LBE_OOM: return "out of device memory";
        case LBE_TIMEOUT: return "device wait timed out";
        case LBE_INTERNAL: return "internal CUDA error";
        case LBE_UNSUPPORTED: return "unsupported";
        case LBE_CANCELLED: return "cancelled";
    }
    return "unknown status";
}

const char* lbe_last_error(lbe_ctx* ctx) { return ctx ? ctx->last_error.c_str() : "null context"; }

lbe_status lbe_create(lbe_ctx** out, int device, size_t budget) {
    if (!out) return LBE_BAD_ARG;
    *out = nullptr;
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess || device < 0 || device >= n) return e != cudaSuccess ? LBE_INTERNAL : LBE_BAD_ARG;
    if ((e = cudaSetDevice(device)) != cudaSuccess) return LBE_INTERNAL;
    auto* c = new lbe_ctx();
    c->device = device;
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    c->budget = budget ? budget : (size_t)(0.9 * fr);
    int prio_low = 0, prio_high = 0;
    cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high);
    if (cudaStreamCreateWithPriority(&c->own_stream, cudaStreamNonBlocking, prio_high) != cudaSuccess) {
        delete c;
        return LBE_INTERNAL;
    }
    c->stream = c->own_stream;
    init_twiddles_cc();
    e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        delete c;
        return LBE_INTERNAL;
    }
    *out = c;
    return LBE_OK;
}

lbe_status lbe_destroy(lbe_ctx* ctx) {
    if (!ctx) return LBE_BAD_ARG;
    cudaSetDevice(ctx->device);
    stop_service(ctx);
    mix_release(ctx);
    for (auto& kv : ctx->tables) {
        DevTables* t = kv.second.get();
        tc_release(ctx, t);
        delete t->tuning;
        t->tuning = nullptr;
        for (void* p : {(void*)t->feq_d, (void*)t->nu1_d, (void*)t->mult_d, (void*)t->ab_d, (void*)t->vel_d,
                        (void*)t->feq_f, (void*)t->nu1_f, (void*)t->mult_f, (void*)t->ab_f, (void*)t->vel_f,
                        (void*)t->orb_f, (void*)t->feq_x, (void*)t->nu1_x, (void*)t->mult_x, (void*)t->ab_x})
            if (p) cudaFree(p);
    }
    ctx->tables.clear();
    cudaDeviceSynchronize();
    arena_release(ctx, ctx->solve_arena);
    arena_release(ctx, ctx->apply_arena);
    for (auto& a : ctx->refine_arena) arena_release(ctx, a);
    if (ctx->own_stream) cudaStreamDestroy(ctx->own_stream);
    if (ctx->side_stream) cudaStreamDestroy(ctx->side_stream);
    delete ctx;
    return LBE_OK;
}

int lbe_problem_cells(const lbe_problem* pb) {
    if (!pb) return 0;
    return pb->geom.dim == 1 ? pb->geom.ns + 1 : pb->geom.nx * pb->geom.ny;
}

// Host: the orbit layout (sweep.h) of `cells` cells from the full velocity grid -- the orbit
// representatives (i2, i3 < nv / 2); orbit_unpack_host (batch.h) is the inverse.
static void orbit_pack(int nv, long cells, const double* full, float* q, int dim) {
    const int H = nv / 2, R2 = dim == 2 ? nv : H;
    const long n3 = (long)nv * nv * nv;
    for (long c = 0; c < cells; ++c)
        for (int i1 = 0; i1 < nv; ++i1)
            for (int j2 = 0; j2 < R2; ++j2)
                for (int j3 = 0; j3 < H; ++j3)
                    q[c * n3 + ((long)i1 * R2 + j2) * H + j3] = (float)full[c * n3 + ((long)i1 * nv + j2) * nv + j3];
}
static lbe_status lbe_solve_batch_impl(lbe_ctx* ctx, const lbe_problem* pbs, int n, lbe_result* outs,
                                double* U3_out, double* h_out, const double* h_in = nullptr,
                                const lbe_result* prev = nullptr) {
    if (!ctx || !pbs || n < 1 || !outs) return bad_arg(ctx, "null argument");
    cudaSetDevice(ctx->device);
    for (int j = 0; j < n; ++j) {
        lbe_status st = validate_problem(ctx, pbs[j]);
        if (st != LBE_OK) return st;
        if (pbs[j].nv != pbs[0].nv || pbs[j].vmax != pbs[0].vmax || pbs[j].M != pbs[0].M ||
            pbs[j].R != pbs[0].R || pbs[j].precision != pbs[0].precision)
            return bad_arg(ctx, "batched problems must share nv, vmax, M, R and precision");
    }
    if (pbs[0].precision == LBE_BF16_REFINED || pbs[0].precision == LBE_FP32_REFINED)
        return refined_solve(ctx, pbs, n, outs, U3_out, h_out);
    auto t0 = std::chrono::steady_clock::now();
    Batch B;
    lbe_status st = batch_init(B, ctx, pbs, n, &ctx->solve_arena, ctx->stream);
    if (st != LBE_OK) return st;
    if (pbs[0].precision == LBE_BF16) {
        // the tensor-core operator with FP32 everything else; scale-relative stopping test
        if (B.t->sym_reps2 == 0) return bad_arg(ctx, "LBE_BF16 needs a parity-reducible direction set");
        B.use_tc = true;
        B.orbit = true;
        for (int j = 0; j < n; ++j) B.ij[j].crit = 1;
        cudaMemcpyAsync(B.ijobs.p, B.ij.data(), n * sizeof(SisJobDev), cudaMemcpyHostToDevice, ctx->stream);
        g_h2d += n * sizeof(SisJobDev);
    }
    if (h_in) {  // resume from a checkpoint (one problem)
        const long n3h = (long)pbs[0].nv * pbs[0].nv * pbs[0].nv;
        const long nn = B.cells * n3h;
        if (B.prec == LBE_FP64) {
            st = cuda_status(ctx, cudaMemcpyAsync(B.h.p, h_in, nn * 8, cudaMemcpyHostToDevice, ctx->stream),
                             "h_in copy");
        } else {
            std::vector<float> tmp(h_in, h_in + nn);
            if (B.quarter()) orbit_pack(pbs[0].nv, B.cells, h_in, tmp.data(), B.geo[0].dim);
            st = cuda_status(ctx, cudaMemcpyAsync(B.h.p, tmp.data(), nn * 4, cudaMemcpyHostToDevice, ctx->stream),
                             "h_in copy");
            if (st == LBE_OK) st = cuda_status(ctx, cudaStreamSynchronize(ctx->stream), "h_in copy");
        }
        g_h2d += nn * (B.prec == LBE_FP64 ? 8 : 4);
        if (st != LBE_OK) return st;
        if (B.use_tc) {  // the h part of the L-moments, which the correction step keeps per cell
            int zero = 0;
            cudaMemcpyAsync(B.act.p, &zero, sizeof(int), cudaMemcpyHostToDevice, ctx->stream);
            launch_correct<float>(*B.t, 1, nullptr, B.h.as<float>(), nullptr, nullptr, B.sjobs.as<SweepJobDev>(),
                                  B.act.as<int>(), ctx->stream, nullptr, B.hmom.as<double>(), B.nd.as<double>(),
                                  B.quarter() ? 1 : 0, 0, B.geo[0].dim == 2 ? 1 : 0);
        }
        if (prev) {  // the flow rates the interrupted run held
            B.hstate[0].M = prev->mass_flow;
            B.hstate[0].Q = prev->heat_flow;
            cudaMemcpyAsync(B.states.p, B.hstate.data(), sizeof(JobState), cudaMemcpyHostToDevice, ctx->stream);
            g_h2d += sizeof(JobState);
        } else {  // flow rates of h_in
            int zero = 0;
            cudaMemcpyAsync(B.act.p, &zero, sizeof(int), cudaMemcpyHostToDevice, ctx->stream);
            if (B.prec == LBE_FP64)
                launch_moments<double>(*B.t, 0, (int)B.cells, B.h.as<double>(), B.mom.as<double>(), ctx->stream);
            else
                launch_moments<float>(*B.t, 0, (int)B.cells, B.h.as<float>(), B.mom.as<double>(), ctx->stream,
                                      B.quarter() ? B.geo[0].dim : 0);
            launch_set_rates(1, B.ijobs.as<SisJobDev>(), B.act.as<int>(), B.mom.as<double>(), B.coef.as<double>(),
                             B.states.as<JobState>(), ctx->stream);
        }
    }
    int maxit = 0;
    for (int j = 0; j < n; ++j) maxit = std::max(maxit, pbs[j].max_iter);
    st = batch_run(B, maxit);
    if (st != LBE_OK) return st;
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    lbe_status worst = LBE_OK;
    for (int j = 0; j < n; ++j) {
        fill_result(B, j, &outs[j], secs);
        if (outs[j].status != LBE_OK && worst == LBE_OK) worst = (lbe_status)outs[j].status;
    }
    const long n3 = (long)pbs[0].nv * pbs[0].nv * pbs[0].nv;
    if (U3_out) {
        st = cuda_status(ctx, cudaMemcpy(U3_out, B.U3.p, B.cells * 8, cudaMemcpyDeviceToHost), "U3 copy");
        g_d2h += B.cells * 8;
    }
    if (st == LBE_OK && h_out) {
        if (B.prec == LBE_FP64) {
            st = cuda_status(ctx, cudaMemcpy(h_out, B.h.p, B.cells * n3 * 8, cudaMemcpyDeviceToHost), "h copy");
        } else {
            std::vector<float> tmp(B.cells * n3);
            st = cuda_status(ctx, cudaMemcpy(tmp.data(), B.h.p, tmp.size() * 4, cudaMemcpyDeviceToHost), "h copy");
            for (size_t i = 0; i < tmp.size(); ++i) h_out[i] = tmp[i];
            if (B.quarter())
                for (int j = 0; j < n; ++j)
                    orbit_unpack_host(pbs[0].nv, B.sj[j].ncell, tmp.data() + B.cell_off[j] * n3,
                                      h_out + B.cell_off[j] * n3, B.geo[j].dim);
        }
    }
    return st != LBE_OK ? st : worst;
}

lbe_status lbe_solve(lbe_ctx* ctx, const lbe_problem* pb, lbe_result* out, double* U3_out, double* h_out) {
    return lbe_solve_batch_impl(ctx, pb, 1, out, U3_out, h_out);
}

lbe_status lbe_solve_batch(lbe_ctx* ctx, const lbe_problem* pbs, int n, lbe_result* outs) {
    return lbe_solve_batch_impl(ctx, pbs, n, outs, nullptr, nullptr);
}

lbe_status lbe_solve_from(lbe_ctx* ctx, const lbe_problem* pb, const double* h_in, const lbe_result* prev,
                          lbe_result* out, double* U3_out, double* h_out) {
    if (!ctx || !pb || !h_in || !out) return bad_arg(ctx, "null argument");
    if (pb->precision != LBE_FP64 && pb->precision != LBE_FP32 && pb->precision != LBE_BF16)
        return bad_arg(ctx, "lbe_solve_from takes LBE_FP64, LBE_FP32 or LBE_BF16");
    if (prev && (!std::isfinite(prev->mass_flow) || !std::isfinite(prev->heat_flow)))
        return bad_arg(ctx, "prev flow rates must be finite");
    return lbe_solve_batch_impl(ctx, pb, 1, out, U3_out, h_out, h_in, prev);
}

lbe_status lbe_apply_L(lbe_ctx* ctx, int nv, double vmax, int M, double R, lbe_precision precision, int cells,
                       const double* delta_dev, const void* h_dev, void* Lplus_dev, void* L_dev,
                       const double* ndelta_dev, double* G_dev, void* stream) {
    if (!ctx) return LBE_BAD_ARG;
    if (cells < 0 || (cells > 0 && (!h_dev || !delta_dev))) return bad_arg(ctx, "null h or delta");
    if (nv != 8 && nv != 16 && nv != 24 && nv != 32) return bad_arg(ctx, "nv must be 8, 16, 24 or 32");
    if (M < 2 || M > 64 || (M & (M - 1))) return bad_arg(ctx, "M must be a power of two in [2, 64]");
    if (!(vmax > 0) || R > 2 * vmax) return bad_arg(ctx, "bad vmax or R");
    if (G_dev && !ndelta_dev) return bad_arg(ctx, "G needs ndelta");
    if (precision == LBE_BF16_REFINED || precision == LBE_BF16) {
        ctx->last_error = "the tensor-core operator acts on the parity subspace: use lbe_apply_L_sym";
        return LBE_UNSUPPORTED;
    }
    if (precision != LBE_FP64 && precision != LBE_FP32 && precision != LBE_DF32) return bad_arg(ctx, "bad precision");
    if (cells == 0) return LBE_OK;
    cudaSetDevice(ctx->device);
    lbe_status st;
    DevTables* t = get_tables(ctx, nv, vmax, M, R, &st);
    if (!t) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const bool wide = precision == LBE_FP64 || precision == LBE_DF32;  // double data
    const int eb = wide ? 8 : 4;
    int chunk = 1;
    const size_t scr = fsm_cc_scratch_bytes(*t, cells, eb, &chunk);
    const size_t vol = (size_t)cells * nv * nv * nv * eb;
    // L is needed for G; the arena holds a temporary when the caller did not ask for it
    const size_t need = ((scr + 255) & ~(size_t)255) + ((G_dev && !L_dev) ? vol : 0);
    if ((st = arena_reserve(ctx, ctx->apply_arena, need)) != LBE_OK) return st;
    void* p = arena_take(ctx->apply_arena, scr);
    void* Lo = L_dev ? L_dev : ((G_dev) ? arena_take(ctx->apply_arena, vol) : nullptr);
    if (wide) {
        st = precision == LBE_FP64
                 ? fsm_cc_apply<double>(*t, cells, delta_dev, (const double*)h_dev, (double*)Lplus_dev, (double*)Lo,
                                        p, chunk, s)
                 : fsm_df_apply(*t, cells, delta_dev, (const double*)h_dev, (double*)Lplus_dev, (double*)Lo, p,
                                chunk, s);
        if (G_dev) lmoments<double>(*t, cells, (const double*)Lo, (const double*)h_dev, ndelta_dev, G_dev, s);
    } else {
        st = fsm_cc_apply<float>(*t, cells, delta_dev, (const float*)h_dev, (float*)Lplus_dev, (float*)Lo, p,
                                 chunk, s);
        if (G_dev) lmoments<float>(*t, cells, (const float*)Lo, (const float*)h_dev, ndelta_dev, G_dev, s);
    }
    if (st != LBE_OK) return st;
    return cuda_status(ctx, cudaGetLastError(), "apply_L");
}

lbe_status lbe_apply_L_sym(lbe_ctx* ctx, int nv, double vmax, int M, double R, lbe_precision precision, int parity,
                           int cells, const double* delta_dev, const void* h_dev, void* Lplus_dev, void* L_dev,
                           const double* ndelta_dev, double* G_dev, void* stream) {
    if (!ctx) return LBE_BAD_ARG;
    if (parity != 1 && parity != 2) return bad_arg(ctx, "parity must be 1 (odd in v3) or 2 (also even in v2)");
    if (cells < 0 || (cells > 0 && (!h_dev || !delta_dev))) return bad_arg(ctx, "null h or delta");
    if (nv != 8 && nv != 16 && nv != 24 && nv != 32) return bad_arg(ctx, "nv must be 8, 16, 24 or 32");
    if (M < 8 || M > 64 || (M & (M - 1))) return bad_arg(ctx, "M must be a power of two in [8, 64]");
    if (!(vmax > 0) || R > 2 * vmax) return bad_arg(ctx, "bad vmax or R");
    if (precision == LBE_BF16) precision = LBE_BF16_REFINED;  // the same tensor-core operator
    if (precision != LBE_FP64 && precision != LBE_FP32 && precision != LBE_BF16_REFINED && precision != LBE_DF32)
        return bad_arg(ctx, "precision must be FP64, FP32, DF32, BF16 or BF16_REFINED");
    if (G_dev && !ndelta_dev) return bad_arg(ctx, "G needs ndelta");
    if (cells == 0) return LBE_OK;
    cudaSetDevice(ctx->device);
    lbe_status st;
    DevTables* t = get_tables(ctx, nv, vmax, M, R, &st);
    if (!t) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const int eb = (precision == LBE_FP64 || precision == LBE_DF32) ? 8 : 4;
    const size_t vol = (size_t)cells * nv * nv * nv * eb;
    int chunk = 1;
    const size_t scr = precision == LBE_BF16_REFINED ? 0 : fsm_cc_scratch_bytes(*t, cells, eb, &chunk);
    const size_t need = scr + 256 + (Lplus_dev ? 0 : vol + 256) + (L_dev ? 0 : vol + 256);
    if ((st = arena_reserve(ctx, ctx->apply_arena, need)) != LBE_OK) return st;
    void* p = scr ? arena_take(ctx->apply_arena, scr) : nullptr;
    void* lp = Lplus_dev ? Lplus_dev : arena_take(ctx->apply_arena, vol);
    void* lo = L_dev ? L_dev : arena_take(ctx->apply_arena, vol);
    if (precision == LBE_BF16_REFINED) {
        if ((uintptr_t)h_dev % 8 != 0) return bad_arg(ctx, "h_dev must be 8-byte aligned for the tensor-core form");
        // with G: L+ h (and L h) and the L-moments in one fused pass
        return tc_apply_sym(ctx, t, parity, cells, delta_dev, (const float*)h_dev, (float*)lp, (float*)lo, s, true,
                            ndelta_dev, G_dev);
    }
    if (precision == LBE_FP64)
        st = fsm_cc_apply<double>(*t, cells, delta_dev, (const double*)h_dev, (double*)lp, (double*)lo, p, chunk, s,
                                  parity);
    else if (precision == LBE_DF32)
        st = fsm_df_apply(*t, cells, delta_dev, (const double*)h_dev, (double*)lp, (double*)lo, p, chunk, s, parity);
    else
        st = fsm_cc_apply<float>(*t, cells, delta_dev, (const float*)h_dev, (float*)lp, (float*)lo, p, chunk, s,
                                 parity);
    if (st != LBE_OK) return st;
    if (G_dev) {
        if (eb == 8)
            lmoments<double>(*t, cells, (const double*)lo, (const double*)h_dev, ndelta_dev, G_dev, s);
        else
            lmoments<float>(*t, cells, (const float*)lo, (const float*)h_dev, ndelta_dev, G_dev, s);
    }
    return cuda_status(ctx, cudaGetLastError(), "apply_L_sym");
}

lbe_status lbe_sweep(lbe_ctx* ctx, const lbe_problem* pb, const void* rhs_dev, void* h_dev, double* mom_dev,
                     void* stream) {
    if (!ctx || !pb || !rhs_dev || !h_dev) return bad_arg(ctx, "null argument");
    lbe_status st = validate_problem(ctx, *pb);
    if (st != LBE_OK) return st;
    if (pb->precision != LBE_FP64 && pb->precision != LBE_FP32)
        return bad_arg(ctx, "sweep precision must be FP64 or FP32");
    cudaSetDevice(ctx->device);
    DevTables* t = get_tables(ctx, pb->nv, pb->vmax, pb->M, pb->R, &st);
    if (!t) return st;
    SweepGeom g;
    build_sweep_geom(g, *pb);
    std::vector<double> coef;
    if (g.dim == 1)
        for (auto* v : {&g.fa, &g.fb, &g.fc, &g.ba, &g.bb, &g.bc}) coef.insert(coef.end(), v->begin(), v->end());
    else
        for (auto* v : {&g.xa, &g.xb, &g.xc, &g.ya, &g.yb, &g.yc}) coef.insert(coef.end(), v->begin(), v->end());
    SweepJobDev j{};
    j.cell_off = 0;
    j.ncell = g.cells;
    j.nx = g.nx;
    j.ny = g.ny;
    j.coef_off = 0;
    j.forcing = pb->forcing;
    j.delta = pb->delta;
    cudaStream_t s = (cudaStream_t)stream;
    void *dc = nullptr, *dj = nullptr;
    if ((st = dev_alloc(ctx, &dc, coef.size() * 8)) != LBE_OK) return st;
    if ((st = dev_alloc(ctx, &dj, sizeof j)) != LBE_OK) {
        dev_free(ctx, dc, coef.size() * 8);
        return st;
    }
    cudaMemcpyAsync(dc, coef.data(), coef.size() * 8, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(dj, &j, sizeof j, cudaMemcpyHostToDevice, s);
    if (pb->precision == LBE_FP64) {
        launch_sweep<double>(*t, g.dim, 1, (int)coef.size(), (const double*)rhs_dev, (double*)h_dev,
                             (SweepJobDev*)dj, nullptr, (double*)dc, s);
        if (mom_dev) launch_moments<double>(*t, 0, g.cells, (const double*)h_dev, mom_dev, s);
    } else {
        launch_sweep<float>(*t, g.dim, 1, (int)coef.size(), (const float*)rhs_dev, (float*)h_dev, (SweepJobDev*)dj,
                            nullptr,
                            (double*)dc, s);
        if (mom_dev) launch_moments<float>(*t, 0, g.cells, (const float*)h_dev, mom_dev, s);
    }
    st = cuda_status(ctx, cudaStreamSynchronize(s), "sweep");
    dev_free(ctx, dc, coef.size() * 8);
    dev_free(ctx, dj, sizeof j);
    return st;
}

lbe_status lbe_diffusion(lbe_ctx* ctx, const lbe_problem* pb, const double* Uh, const double* W1, const double* W2,
                         const double* X12, const double* G1, const double* G2, double* U_out) {
    if (!ctx || !pb || !Uh || !W1 || !G1 || !U_out) return bad_arg(ctx, "null argument");
    lbe_status st = validate_problem(ctx, *pb);
    if (st != LBE_OK) return st;
    if (pb->geom.dim == 2 && (!W2 || !X12 || !G2)) return bad_arg(ctx, "2D needs W2, X12, G2");
    cudaSetDevice(ctx->device);
    lbe_problem p = *pb;
    p.scheme = LBE_SIS;
    p.precision = LBE_FP64;
    Batch B;
    if ((st = batch_init(B, ctx, &p, 1, &ctx->solve_arena, ctx->stream)) != LBE_OK) return st;
    const int n = (int)B.cells;
    std::vector<double> mom(5 * n, 0.0), G(2 * n, 0.0);
    for (int i = 0; i < n; ++i) {
        mom[5 * i + 0] = Uh[i];
        mom[5 * i + 2] = W1[i];
        mom[5 * i + 3] = W2 ? W2[i] : 0.0;
        mom[5 * i + 4] = X12 ? X12[i] : 0.0;
        G[2 * i + 0] = G1[i];
        G[2 * i + 1] = G2 ? G2[i] : 0.0;
    }
    cudaStream_t s = ctx->stream;
    cudaMemcpyAsync(B.mom.p, mom.data(), mom.size() * 8, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(B.G.p, G.data(), G.size() * 8, cudaMemcpyHostToDevice, s);
    launch_sis_update(*B.t, 1, B.ijobs.as<SisJobDev>(), nullptr, B.mom.as<double>(), B.G.as<double>(),
                      B.coef.as<double>(), B.work.as<double>(), B.dU.as<double>(), B.U3.as<double>(),
                      B.states.as<JobState>(), s);
    std::vector<double> du(n);
    cudaMemcpyAsync(du.data(), B.dU.p, n * 8, cudaMemcpyDeviceToHost, s);
    if ((st = cuda_status(ctx, cudaStreamSynchronize(s), "diffusion")) != LBE_OK) return st;
    for (int i = 0; i < n; ++i) U_out[i] = Uh[i] + du[i];
    return LBE_OK;
}

}  // extern "C"

struct lbe_batch {
    lbe_ctx* ctx = nullptr;
    lbe::Arena arena;
    lbe::Batch B;
    int maxit = 0;
};

extern "C" {

lbe_status lbe_batch_create(lbe_ctx* ctx, const lbe_problem* pbs, int n, lbe_batch** out) {
    if (!ctx || !pbs || n < 1 || !out) return bad_arg(ctx, "null argument");
    *out = nullptr;
    cudaSetDevice(ctx->device);
    for (int j = 0; j < n; ++j) {
        lbe_status st = validate_problem(ctx, pbs[j]);
        if (st != LBE_OK) return st;
        if (pbs[j].nv != pbs[0].nv || pbs[j].vmax != pbs[0].vmax || pbs[j].M != pbs[0].M ||
            pbs[j].R != pbs[0].R || pbs[j].precision != pbs[0].precision)
            return bad_arg(ctx, "batched problems must share nv, vmax, M, R and precision");
    }
    if (pbs[0].precision != LBE_FP64 && pbs[0].precision != LBE_FP32)
        return bad_arg(ctx, "resident batches take FP64 or FP32");
    auto* b = new lbe_batch();
    b->ctx = ctx;
    lbe_status st = batch_init(b->B, ctx, pbs, n, &b->arena, ctx->stream);
    if (st != LBE_OK) {
        arena_release(ctx, b->arena);
        delete b;
        return st;
    }
    for (int j = 0; j < n; ++j) b->maxit = std::max(b->maxit, pbs[j].max_iter);
    *out = b;
    return LBE_OK;
}

lbe_status lbe_batch_run(lbe_batch* b, lbe_result* outs) {
    if (!b || !outs) return LBE_BAD_ARG;
    Ctx* c = b->ctx;
    cudaSetDevice(c->device);
    Batch& B = b->B;
    B.s = c->stream;
    const long n3 = (long)B.pbs[0].nv * B.pbs[0].nv * B.pbs[0].nv;
    auto t0 = std::chrono::steady_clock::now();
    cudaMemsetAsync(B.h.p, 0, B.cells * n3 * (B.prec == LBE_FP64 ? 8 : 4), B.s);
    cudaMemsetAsync(B.hmom.p, 0, B.hmom.n, B.s);
    B.hstate.assign(B.njobs, JobState{});
    cudaMemcpyAsync(B.states.p, B.hstate.data(), B.njobs * sizeof(JobState), cudaMemcpyHostToDevice, B.s);
    g_h2d += B.njobs * sizeof(JobState);
    B.active.resize(B.njobs);
    for (int j = 0; j < B.njobs; ++j) B.active[j] = j;
    lbe_status st = batch_run(B, b->maxit);
    if (st != LBE_OK) return st;
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    lbe_status worst = LBE_OK;
    for (int j = 0; j < B.njobs; ++j) {
        fill_result(B, j, &outs[j], secs);
        if (outs[j].status != LBE_OK && worst == LBE_OK) worst = (lbe_status)outs[j].status;
    }
    return worst;
}

lbe_status lbe_batch_destroy(lbe_batch* b) {
    if (!b) return LBE_BAD_ARG;
    cudaSetDevice(b->ctx->device);
    cudaStreamSynchronize(b->ctx->stream);
    arena_release(b->ctx, b->arena);
    delete b;
    return LBE_OK;
}

lbe_status lbe_set_stream(lbe_ctx* ctx, void* stream) {
    if (!ctx) return LBE_BAD_ARG;
    ctx->stream = stream ? (cudaStream_t)stream : ctx->own_stream;
    return LBE_OK;
}

lbe_status lbe_get_stats(lbe_stats* out) {
    if (!out) return LBE_BAD_ARG;
    out->kernel_launches = g_launches.load();
    out->h2d_bytes = g_h2d.load();
    out->d2h_bytes = g_d2h.load();
    out->cell_l_evals = g_levals.load();
    unsigned long long n = 0;
    double ms = 0.0;
    get_gemm_time(&n, &ms);
    out->dense_gemm_timed = n;
    out->dense_gemm_ms = ms;
    resolve_sweep_times();
    {
        std::lock_guard<std::mutex> lk(g_time_mu);
        out->sweep_timed = g_sweep_n;
        out->sweep_ms = g_sweep_ms;
        out->sweep_bytes = g_sweep_bytes;
    }
    return LBE_OK;
}

lbe_status lbe_set_kernel_timing(int on) {
    g_time_kernels.store(on ? 1 : 0);
    return LBE_OK;
}

lbe_status lbe_tuning_report(lbe_ctx* ctx, char* buf, size_t cap) {
    if (!ctx || !buf || cap == 0) return LBE_BAD_ARG;
    std::string out;
    std::lock_guard<std::mutex> lk(ctx->tables_mu);
    for (auto& kv : ctx->tables) {
        Tuning* tu = kv.second->tuning;
        if (!tu) continue;
        std::lock_guard<std::mutex> lk2(tu->mu);
        for (auto& line : tu->log) out += line + "\n";
    }
    const size_t n = std::min(out.size(), cap - 1);
    memcpy(buf, out.data(), n);
    buf[n] = 0;
    return out.size() < cap ? LBE_OK : LBE_BAD_ARG;
}

lbe_status lbe_debug_expire_waits(int on) {
    g_expire_waits.store(on ? 1 : 0);
    return LBE_OK;
}

}  // extern "C"

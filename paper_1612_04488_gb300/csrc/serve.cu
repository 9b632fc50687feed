// Continuous-batching service behind lbe_submit / lbe_poll.
//
// Requests are grouped into buckets by (nv, vmax, M, R, arithmetic).  A bucket owns one
// resident batch whose device buffers have room for `cap_cells` cells and `slots` problems;
// a problem occupies one slot and one contiguous range of cells (first-fit pool).  The
// service thread repeats:
//   admit   queued problems into free slots / cell ranges of their bucket (the HBM budget
//           bounds the buckets that can be created);
//   iterate one SIS (or CIS) iteration of every bucket with active problems, each bucket on
//           its own stream so that the buckets' kernels overlap on the device; within a
//           bucket the collision operator and the moments run over merged cell spans of all
//           active problems and the sweeps run as one launch over the active slots;
//   retire  problems whose convergence flag is set, freeing their slot and cells.
// Every per-problem quantity is computed by per-cell or per-problem blocks in a fixed
// order, so a problem's result is bitwise the same alone and in any mix.
//
// Refined requests (LBE_FP32_REFINED, LBE_BF16_REFINED) hold a slot in the FP32 and in the
// FP64 bucket of their grid and run the defect correction of refine.cu one step at a time:
// FP32 SIS of the full problem to a change of 1e-5 of the flow-rate scale; then alternately
// one FP64 SIS iteration (residual r = Phi(h) - h and the eps test of LBE_FP64) and an FP32
// solve of the homogeneous correction equation with source r, h <- h + e.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <memory>
#include <string>
#include <vector>

#include "batch.h"
#include "lbe_internal.h"
#include "sweep.h"

namespace lbe {

namespace {

constexpr int kMaxSlotCellsX = 128;  // service geometry limits (per-slot coefficient regions)
constexpr int kMaxSlotNs = 1024;
constexpr long kBucketCells = 4096;  // cells of one bucket's pool (a request must fit in one)

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Bucket;

// A request inside the service.  phase: 0 plain (one bucket), 1 FP32 solve of the full
// problem, 2 one FP64 residual iteration, 3 FP32 correction solve.
struct SJob {
    Job* j = nullptr;
    int phase = 0;
    Bucket* F = nullptr;  // FP32 bucket (or the only bucket when plain)
    int fs = -1;
    Bucket* D = nullptr;  // FP64 bucket of a refined request
    int ds = -1;
    int outer = 0, inner = 0, refs = 0;
};

struct Bucket {
    std::string key;
    int nv = 0, M = 0, prec = LBE_FP32;
    double vmax = 0, R = 0;
    long cap_cells = 0;
    int slots = 0;
    size_t coef_per_slot = 0, work_per_slot = 0;
    cudaStream_t stream = nullptr;
    Arena arena;
    Batch B;
    std::vector<SJob*> slot_job;
    std::vector<std::pair<long, long>> free_ranges;  // (offset, length), sorted by offset
    DevBuf aux;  // FP32 buckets: additive source r; FP64 buckets: copy of h before an iteration
    // FP64 buckets of refined requests: operator of h as base (FP64, once per request) plus
    // the FP32 operator of the increment (see Batch)
    bool inc = false;
    DevBuf base_h, base_lp, base_lh, inc_h, inc_lp, inc_lh, inc_scratch;
    lbe_status failed = LBE_OK;  // an operator launch of the last iteration failed
};

size_t coef_len(const SweepGeom& g) {
    if (g.dim == 1) return 6 * (size_t)g.cells + 4 * (size_t)g.cells + g.cells;
    const size_t mx = g.nx - 2, my = g.ny - 2;
    return 3 * (size_t)g.nx + 3 * (size_t)g.ny + mx * mx + my * my + mx * my + g.cells;
}

bool take_range(Bucket& b, long n, long* off) {
    for (size_t i = 0; i < b.free_ranges.size(); ++i) {
        auto& r = b.free_ranges[i];
        if (r.second >= n) {
            *off = r.first;
            r.first += n;
            r.second -= n;
            if (r.second == 0) b.free_ranges.erase(b.free_ranges.begin() + i);
            return true;
        }
    }
    return false;
}

void give_range(Bucket& b, long off, long n) {
    b.free_ranges.push_back({off, n});
    std::sort(b.free_ranges.begin(), b.free_ranges.end());
    std::vector<std::pair<long, long>> m;
    for (auto& r : b.free_ranges) {
        if (!m.empty() && m.back().first + m.back().second == r.first)
            m.back().second += r.second;
        else
            m.push_back(r);
    }
    b.free_ranges.swap(m);
}

std::string bucket_key(const lbe_problem& pb, int prec, bool inc, bool tc) {
    char k[160];
    const double R = pb.R > 0 ? pb.R : default_R(pb.vmax);
    snprintf(k, sizeof k, "%d/%.17g/%d/%.17g/%d/%d/%d", pb.nv, pb.vmax, pb.M, R, prec, inc ? 1 : 0, tc ? 1 : 0);
    return k;
}

// Buffers of a bucket: the batch layout of batch_init, sized by capacity instead of jobs.
lbe_status bucket_create(Ctx* c, Bucket& b, const lbe_problem& pb, int prec, long cap_cells, int slots,
                         bool inc) {
    b.inc = inc;
    b.nv = pb.nv;
    b.M = pb.M;
    b.vmax = pb.vmax;
    b.R = pb.R > 0 ? pb.R : default_R(pb.vmax);
    b.prec = prec;
    b.cap_cells = cap_cells;
    b.slots = slots;
    lbe_status st;
    b.B.t = get_tables(c, pb.nv, pb.vmax, pb.M, b.R, &st);
    if (!b.B.t) return st;
    if (cudaStreamCreateWithFlags(&b.stream, cudaStreamNonBlocking) != cudaSuccess) return LBE_INTERNAL;
    Batch& B = b.B;
    B.c = c;
    B.arena = &b.arena;
    B.s = b.stream;
    B.prec = prec;
    B.njobs = slots;
    B.cells = cap_cells;
    B.pbs.assign(slots, lbe_problem{});
    B.geo.assign(slots, SweepGeom{});
    B.sj.assign(slots, SweepJobDev{});
    B.ij.assign(slots, SisJobDev{});
    B.cell_off.assign(slots, 0);
    B.hstate.assign(slots, JobState{});
    const int eb = prec == LBE_FP64 ? 8 : 4;
    const long n3 = (long)pb.nv * pb.nv * pb.nv;
    const size_t mx = kMaxSlotCellsX - 2;
    b.coef_per_slot = std::max<size_t>(11 * (kMaxSlotNs + 1), 6 * kMaxSlotCellsX + 3 * mx * mx + kMaxSlotCellsX * kMaxSlotCellsX);
    b.work_per_slot = 2 * mx * mx;
    const size_t vol = (size_t)cap_cells * n3 * eb;
    const size_t scr = fsm_cc_scratch_bytes(*B.t, (int)cap_cells, eb, &B.chunk);
    struct Piece {
        DevBuf* d;
        size_t n;
    };
    const Piece pieces[] = {{&B.h, vol}, {&B.hh, vol}, {&B.lp, vol}, {&B.lh, vol}, {&B.scratch, scr},
                            {&B.mom, (size_t)cap_cells * 5 * 8}, {&B.G, (size_t)cap_cells * 2 * 8},
                            {&B.dU, (size_t)cap_cells * 8}, {&B.U3, (size_t)cap_cells * 8},
                            {&B.delta, (size_t)cap_cells * 8}, {&B.nd, (size_t)cap_cells * 8},
                            {&B.hmom, (size_t)cap_cells * 2 * 8},
                            {&B.coef, b.coef_per_slot * slots * 8}, {&B.work, b.work_per_slot * slots * 8},
                            {&B.sjobs, slots * sizeof(SweepJobDev)}, {&B.ijobs, slots * sizeof(SisJobDev)},
                            {&B.states, slots * sizeof(JobState)}, {&B.act, slots * sizeof(int)},
                            {&b.aux, vol},
                            {&b.base_h, inc ? vol : 0}, {&b.base_lp, inc ? vol : 0}, {&b.base_lh, inc ? vol : 0},
                            {&b.inc_h, inc ? vol / 2 : 0}, {&b.inc_lp, inc ? vol / 2 : 0},
                            {&b.inc_lh, inc ? vol / 2 : 0},
                            {&b.inc_scratch, inc ? fsm_cc_scratch_bytes(*B.t, (int)cap_cells, 4, &B.inc_chunk) : 0}};
    size_t total = 0;
    for (const Piece& q : pieces) total += (q.n + 255) & ~(size_t)255;
    if ((st = arena_reserve(c, b.arena, total)) != LBE_OK) return st;
    for (const Piece& q : pieces) {
        if (q.n == 0) continue;
        q.d->p = arena_take(b.arena, q.n);
        q.d->n = q.n;
        if (!q.d->p) return LBE_INTERNAL;
    }
    if (inc) {
        B.base_h = b.base_h.as<double>();
        B.base_lp = b.base_lp.as<double>();
        B.base_lh = b.base_lh.as<double>();
        B.inc_h = b.inc_h.as<float>();
        B.inc_lp = b.inc_lp.as<float>();
        B.inc_lh = b.inc_lh.as<float>();
        B.inc_scratch = b.inc_scratch.p;
    }
    if (prec != LBE_FP64) {
        B.extra = b.aux;  // zero outside correction solves
        cudaMemsetAsync(b.aux.p, 0, vol, b.stream);
        cudaStreamSynchronize(b.stream);
    }
    b.slot_job.assign(slots, nullptr);
    b.free_ranges = {{0, cap_cells}};
    return LBE_OK;
}

void fill_cells(double* dev, long off, long n, double v, cudaStream_t s) {
    std::vector<double> tmp(n, v);
    cudaMemcpyAsync(dev + off, tmp.data(), n * 8, cudaMemcpyHostToDevice, s);
    cudaStreamSynchronize(s);  // tmp is pageable and local
    g_h2d += n * 8;
}

// Place problem pb in slot s at cell offset off with h = 0.  stage 1: FP32 solve of a
// refined request (change test against the flow-rate scale, tolerance 1e-5).
void slot_install(Bucket& b, int s, const lbe_problem& pb, long off, int phase) {
    Batch& B = b.B;
    B.pbs[s] = pb;
    SweepGeom& g = B.geo[s];
    g = SweepGeom{};
    build_sweep_geom(g, pb);
    std::vector<double> coef;
    SweepJobDev sj{};
    sj.cell_off = off;
    sj.ncell = g.cells;
    sj.nx = g.nx;
    sj.ny = g.ny;
    sj.forcing = pb.forcing;
    sj.delta = pb.delta;
    sj.coef_off = (int)(s * b.coef_per_slot);
    if (g.dim == 1)
        for (auto* v : {&g.fa, &g.fb, &g.fc, &g.ba, &g.bb, &g.bc}) coef.insert(coef.end(), v->begin(), v->end());
    else
        for (auto* v : {&g.xa, &g.xb, &g.xc, &g.ya, &g.yb, &g.yc}) coef.insert(coef.end(), v->begin(), v->end());
    SisJobDev ij{};
    ij.cell_off = off;
    ij.ncell = g.cells;
    ij.dim = g.dim;
    ij.nx = g.nx;
    ij.ny = g.ny;
    ij.width = pb.geom.width;
    ij.scheme = pb.scheme == LBE_SIS ? 1 : 0;
    const double Nn = pb.N > 0 ? pb.N : 1.25;
    ij.ndsig = Nn * pb.delta * (pb.forcing == LBE_POISEUILLE ? 1.0 : 0.0);
    ij.eps = phase == 1 ? std::max(pb.eps, 1e-5) : pb.eps;
    ij.crit = phase == 1 ? 1 : 0;
    ij.max_iter = pb.max_iter;
    ij.coef_off = (int)(s * b.coef_per_slot + coef.size());
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
        ij.work_off = (long)(s * b.work_per_slot);
    }
    ij.trap_off = (int)(s * b.coef_per_slot + coef.size());
    coef.insert(coef.end(), g.trap.begin(), g.trap.end());
    B.sj[s] = sj;
    B.ij[s] = ij;
    B.cell_off[s] = off;
    B.hstate[s] = JobState{};
    cudaStream_t st = b.stream;
    cudaMemcpyAsync(B.coef.as<double>() + s * b.coef_per_slot, coef.data(), coef.size() * 8,
                    cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(B.sjobs.as<SweepJobDev>() + s, &B.sj[s], sizeof(SweepJobDev), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(B.ijobs.as<SisJobDev>() + s, &B.ij[s], sizeof(SisJobDev), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(B.states.as<JobState>() + s, &B.hstate[s], sizeof(JobState), cudaMemcpyHostToDevice, st);
    g_h2d += coef.size() * 8 + sizeof(SweepJobDev) + sizeof(SisJobDev) + sizeof(JobState);
    fill_cells(B.delta.as<double>(), off, g.cells, pb.delta, st);
    fill_cells(B.nd.as<double>(), off, g.cells, Nn * pb.delta, st);
    const long n3 = (long)pb.nv * pb.nv * pb.nv;
    const int eb = b.prec == LBE_FP64 ? 8 : 4;
    cudaMemsetAsync((char*)B.h.p + off * n3 * eb, 0, (size_t)g.cells * n3 * eb, st);
    cudaMemsetAsync(B.hmom.as<double>() + off * 2, 0, (size_t)g.cells * 2 * 8, st);
    if (b.prec != LBE_FP64) cudaMemsetAsync((char*)b.aux.p + off * n3 * eb, 0, (size_t)g.cells * n3 * eb, st);
}

// Switch an FP32 slot to the homogeneous correction equation (or back): forcing, momentum
// term, tolerance and test, state reset, h = 0.
void slot_set_correction(Bucket& b, int s) {
    Batch& B = b.B;
    B.sj[s].forcing = kForcingNone;
    B.ij[s].ndsig = 0.0;
    B.ij[s].eps = 1e-4;
    B.ij[s].crit = 1;
    B.ij[s].max_iter = 30;
    B.hstate[s] = JobState{};
    cudaStream_t st = b.stream;
    cudaMemcpyAsync(B.sjobs.as<SweepJobDev>() + s, &B.sj[s], sizeof(SweepJobDev), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(B.ijobs.as<SisJobDev>() + s, &B.ij[s], sizeof(SisJobDev), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(B.states.as<JobState>() + s, &B.hstate[s], sizeof(JobState), cudaMemcpyHostToDevice, st);
    g_h2d += sizeof(SweepJobDev) + sizeof(SisJobDev) + sizeof(JobState);
    const long n3 = (long)b.nv * b.nv * b.nv;
    cudaMemsetAsync(B.h.as<float>() + B.cell_off[s] * n3, 0, (size_t)B.sj[s].ncell * n3 * 4, st);
    cudaMemsetAsync(B.hmom.as<double>() + B.cell_off[s] * 2, 0, (size_t)B.sj[s].ncell * 2 * 8, st);
}

struct Service {
    Ctx* c;
    std::vector<std::unique_ptr<Bucket>> buckets;
    long cap_cells_default = kBucketCells;
};

}  // namespace

static Bucket* find_bucket(Service& sv, const std::string& key) {
    for (auto& b : sv.buckets)
        if (b->key == key) return b.get();
    return nullptr;
}

// tc: BF16-refined requests -- an FP32 bucket whose collision operator is the tensor-core
// GEMM, or an FP64 increment-mode bucket whose increments go through that GEMM
static Bucket* get_bucket(Service& sv, Ctx* c, const lbe_problem& pb, int prec, bool inc, lbe_status* st,
                          bool tc = false) {
    const std::string key = bucket_key(pb, prec, inc, tc);
    Bucket* b = find_bucket(sv, key);
    *st = LBE_OK;
    if (b) return b;
    auto nb = std::make_unique<Bucket>();
    nb->key = key;
    *st = bucket_create(c, *nb, pb, prec, sv.cap_cells_default, c->max_active, inc);
    if (*st != LBE_OK) {
        if (nb->stream) cudaStreamDestroy(nb->stream);
        arena_release(c, nb->arena);
        return nullptr;
    }
    if (prec == LBE_FP64)
        nb->B.inc_tc = tc && inc;
    else
        nb->B.use_tc = nb->B.orbit = tc;
    b = nb.get();
    sv.buckets.push_back(std::move(nb));
    return b;
}

static bool reserve(Bucket* b, int cells, int* slot, long* off) {
    *slot = -1;
    for (int s = 0; s < b->slots; ++s)
        if (!b->slot_job[s]) {
            *slot = s;
            break;
        }
    if (*slot < 0 || cells > b->cap_cells) return false;
    return take_range(*b, cells, off);
}

static void release(Bucket* b, int s) {
    b->slot_job[s] = nullptr;
    give_range(*b, b->B.cell_off[s], b->B.sj[s].ncell);
}

static void finish(Ctx* c, SJob* sj, const Bucket* b, int s, double t) {
    Job* j = sj->j;
    lbe_result r{};
    fill_result(b->B, s, &r, t - j->t_submit);
    if (sj->phase != 0) {
        r.iters = sj->outer + sj->inner;
        r.refinements = sj->refs;
    }
    std::lock_guard<std::mutex> lk(c->mu);
    j->res = r;
    j->done = 1;
}

static void service_main(Ctx* c) {
    cudaSetDevice(c->device);
    Service sv{c};
    std::vector<Job*> pending;
    std::vector<std::unique_ptr<SJob>> live;
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(c->mu);
            if (live.empty() && c->queue.empty() && pending.empty()) {
                if (c->stop) break;
                c->cv.wait_for(lk, std::chrono::milliseconds(50));
                continue;
            }
            while (!c->queue.empty()) {
                pending.push_back(c->queue.front());
                c->queue.pop_front();
            }
        }
        // ---- admit, in arrival order, while slots and cells allow -----------------------
        std::vector<Job*> still;
        for (Job* j : pending) {
            if (j->cancel.load()) {  // withdrawn before admission
                std::lock_guard<std::mutex> lk(c->mu);
                j->res = lbe_result{};
                j->res.status = LBE_CANCELLED;
                j->done = 1;
                continue;
            }
            const lbe_problem& pb = j->pb;
            const bool refined = pb.precision == LBE_FP32_REFINED || pb.precision == LBE_BF16_REFINED;
            const int cells = lbe_problem_cells(&pb);
            lbe_status st;
            const bool tc = pb.precision == LBE_BF16_REFINED && pb.M >= 8;
            Bucket* F = get_bucket(sv, c, pb, refined ? LBE_FP32 : pb.precision, false, &st, tc);
            // the FP64 bucket of a BF16-refined request evaluates increments on the tensor cores too
            Bucket* D = (F && refined) ? get_bucket(sv, c, pb, LBE_FP64, true, &st, tc) : nullptr;
            if (!F || (refined && !D)) {
                if (live.empty()) {  // nothing will free memory: fail the request
                    std::lock_guard<std::mutex> lk(c->mu);
                    j->res.status = st;
                    j->done = 1;
                } else {
                    still.push_back(j);
                }
                continue;
            }
            int fs = -1, ds = -1;
            long foff = 0, doff = 0;
            if (!reserve(F, cells, &fs, &foff)) {
                still.push_back(j);
                continue;
            }
            if (refined && !reserve(D, cells, &ds, &doff)) {
                give_range(*F, foff, cells);
                still.push_back(j);
                continue;
            }
            auto sj = std::make_unique<SJob>();
            sj->j = j;
            sj->F = F;
            sj->fs = fs;
            sj->phase = refined ? 1 : 0;
            F->slot_job[fs] = sj.get();
            slot_install(*F, fs, pb, foff, refined ? 1 : 0);
            if (refined) {
                lbe_problem p64 = pb;
                p64.precision = LBE_FP64;
                sj->D = D;
                sj->ds = ds;
                D->slot_job[ds] = sj.get();
                slot_install(*D, ds, p64, doff, 0);
            }
            live.push_back(std::move(sj));
        }
        pending.swap(still);
        // ---- one iteration of every bucket's iterating problems, one stream per bucket ----
        std::vector<Bucket*> ran;
        for (auto& bp : sv.buckets) {
            Bucket& b = *bp;
            b.B.active.clear();
            for (int s = 0; s < b.slots; ++s) {
                SJob* sj = b.slot_job[s];
                if (!sj) continue;
                const bool here = (sj->phase == 0) || (sj->phase == 2 ? (sj->D == &b && sj->ds == s)
                                                                      : (sj->F == &b && sj->fs == s));
                if (here) b.B.active.push_back(s);
            }
            if (b.B.active.empty()) continue;
            if (b.prec == LBE_FP64)
                batch_iterate<double>(b.B);
            else
                batch_iterate<float>(b.B);
            ran.push_back(&b);
        }
        for (Bucket* b : ran) {
            lbe_status st = cuda_status(c, cudaStreamSynchronize(b->stream), "service iterate");
            if (st == LBE_OK && (b->B.use_tc || b->B.inc_tc)) st = tc_check(c, b->B.t);
            if (st == LBE_OK) st = b->B.op_status;
            b->B.op_status = LBE_OK;
            if (st != LBE_OK) b->failed = st;
        }
        // ---- retire finished problems, advance refined ones ------------------------------
        const double t = now_s();
        std::vector<std::unique_ptr<SJob>> keep;
        for (auto& up : live) {
            SJob* sj = up.get();
            const long n3 = (long)sj->j->pb.nv * sj->j->pb.nv * sj->j->pb.nv;
            bool done = false;
            const lbe_status bad = (sj->F && sj->F->failed != LBE_OK)   ? sj->F->failed
                                   : (sj->D && sj->D->failed != LBE_OK) ? sj->D->failed
                                                                        : LBE_OK;
            const bool cancelled = sj->j->cancel.load() != 0;
            if (bad != LBE_OK || cancelled) {  // a launch of its buckets failed, or it was withdrawn
                {
                    std::lock_guard<std::mutex> lk(c->mu);
                    sj->j->res = lbe_result{};
                    sj->j->res.status = bad != LBE_OK ? bad : LBE_CANCELLED;
                    sj->j->done = 1;
                }
                if (sj->F) release(sj->F, sj->fs);
                if (sj->D) release(sj->D, sj->ds);
                continue;
            }
            if (sj->phase == 0) {
                const JobState& js = sj->F->B.hstate[sj->fs];
                if (std::find(sj->F->B.active.begin(), sj->F->B.active.end(), sj->fs) != sj->F->B.active.end() &&
                    js.done) {
                    finish(c, sj, sj->F, sj->fs, t);
                    release(sj->F, sj->fs);
                    done = true;
                }
            } else if (sj->phase == 1 || sj->phase == 3) {
                Bucket* F = sj->F;
                Bucket* D = sj->D;
                const JobState& js = F->B.hstate[sj->fs];
                if (js.done) {
                    sj->inner += js.iters;
                    const long n = (long)F->B.sj[sj->fs].ncell * n3;
                    double* h = D->B.h.as<double>() + D->B.cell_off[sj->ds] * n3;
                    double* hold = D->aux.as<double>() + D->B.cell_off[sj->ds] * n3;
                    const float* e = F->B.h.as<float>() + F->B.cell_off[sj->fs] * n3;
                    cudaStream_t ds = D->stream;
                    // a tensor-core bucket: e in the orbit layout (plates a quarter, ducts a half)
                    const bool q = F->B.quarter();
                    const int dim = F->B.geo[sj->fs].dim;
                    const long nc = F->B.sj[sj->fs].ncell;
                    if (sj->phase == 1) {
                        if (q)
                            range_widen_q(e, h, nc, F->nv, dim, ds);
                        else
                            range_widen(e, h, n, ds);
                        // the request's one FP64 collision-operator evaluation, at h0
                        const long o = D->B.cell_off[sj->ds] * n3;
                        range_copy(h, D->base_h.as<double>() + o, n, ds);
                        fsm_df_apply(*D->B.t, D->B.sj[sj->ds].ncell, D->B.delta.as<double>() + D->B.cell_off[sj->ds],
                                             D->base_h.as<double>() + o, D->base_lp.as<double>() + o,
                                             D->base_lh.as<double>() + o, D->B.scratch.p, D->B.chunk, ds,
                                             D->B.geo[sj->ds].dim == 1 ? 2 : 1);
                        // the FP32 flow rates of h start the FP64 change test
                        D->B.hstate[sj->ds] = JobState{};
                        D->B.hstate[sj->ds].M = js.M;
                        D->B.hstate[sj->ds].Q = js.Q;
                        cudaMemcpyAsync(D->B.states.as<JobState>() + sj->ds, &D->B.hstate[sj->ds], sizeof(JobState),
                                        cudaMemcpyHostToDevice, ds);
                    } else {
                        if (q)
                            range_correct_q(hold, e, h, nc, F->nv, dim, ds);
                        else
                            range_correct(hold, e, h, n, ds);
                        ++sj->refs;
                        // flow rates of the corrected h for the next change test
                        launch_moments<double>(*D->B.t, D->B.cell_off[sj->ds], D->B.sj[sj->ds].ncell,
                                               D->B.h.as<double>(), D->B.mom.as<double>(), ds);
                        int one = sj->ds;
                        cudaMemcpyAsync(D->B.act.p, &one, sizeof(int), cudaMemcpyHostToDevice, ds);
                        launch_set_rates(1, D->B.ijobs.as<SisJobDev>(), D->B.act.as<int>(), D->B.mom.as<double>(),
                                         D->B.coef.as<double>(), D->B.states.as<JobState>(), ds);
                    }
                    range_copy(h, hold, n, ds);
                    cudaStreamSynchronize(ds);
                    sj->phase = 2;
                }
            } else if (sj->phase == 2) {
                Bucket* F = sj->F;
                Bucket* D = sj->D;
                const JobState& js = D->B.hstate[sj->ds];
                ++sj->outer;
                if (js.done || sj->outer >= sj->j->pb.max_iter) {
                    finish(c, sj, D, sj->ds, t);
                    release(D, sj->ds);
                    release(F, sj->fs);
                    done = true;
                } else {
                    const long n = (long)D->B.sj[sj->ds].ncell * n3;
                    const double* h = D->B.h.as<double>() + D->B.cell_off[sj->ds] * n3;
                    const double* hold = D->aux.as<double>() + D->B.cell_off[sj->ds] * n3;
                    float* r = F->aux.as<float>() + F->B.cell_off[sj->fs] * n3;
                    if (F->B.quarter())
                        range_residual_q(h, hold, r, D->B.sj[sj->ds].ncell, F->nv, F->B.geo[sj->fs].dim, D->stream);
                    else
                        range_residual(h, hold, r, n, D->stream);
                    cudaStreamSynchronize(D->stream);
                    slot_set_correction(*F, sj->fs);
                    cudaStreamSynchronize(F->stream);
                    sj->phase = 3;
                }
            }
            if (!done) keep.push_back(std::move(up));
        }
        live.swap(keep);
        for (auto& b : sv.buckets) b->failed = LBE_OK;  // its requests have been failed
    }
    for (auto& b : sv.buckets) {
        cudaStreamSynchronize(b->stream);
        arena_release(c, b->arena);
        cudaStreamDestroy(b->stream);
    }
}

void stop_service(Ctx* c) {
    {
        std::lock_guard<std::mutex> lk(c->mu);
        if (!c->service_started) return;
        c->stop = true;
    }
    c->cv.notify_all();
    if (c->service.joinable()) c->service.join();
    c->service_started = false;
}

}  // namespace lbe

using namespace lbe;

extern "C" {

lbe_status lbe_submit(lbe_ctx* ctx, const lbe_problem* pb, uint64_t* ticket) {
    if (!ctx || !pb || !ticket) return LBE_BAD_ARG;
    lbe_status st = validate_problem(ctx, *pb);
    if (st != LBE_OK) return st;
    if ((pb->geom.dim == 1 && pb->geom.ns > kMaxSlotNs) ||
        (pb->geom.dim == 2 && (pb->geom.nx > kMaxSlotCellsX || pb->geom.ny > kMaxSlotCellsX)))
        return bad_arg(ctx, "service geometry limit: ns <= 1024, nx, ny <= 128");
    if (lbe_problem_cells(pb) > kBucketCells)
        return bad_arg(ctx, "service limit: at most 4096 cells per request");
    auto job = std::make_unique<Job>();
    job->pb = *pb;
    job->t_submit = now_s();
    std::lock_guard<std::mutex> lk(ctx->mu);
    job->ticket = ctx->next_ticket++;
    *ticket = job->ticket;
    ctx->queue.push_back(job.get());
    ctx->jobs[job->ticket] = std::move(job);
    if (!ctx->service_started) {
        ctx->stop = false;
        ctx->service_started = true;
        ctx->service = std::thread(service_main, static_cast<Ctx*>(ctx));
    }
    ctx->cv.notify_all();
    return LBE_OK;
}

lbe_status lbe_poll(lbe_ctx* ctx, uint64_t ticket, lbe_result* out, int* done) {
    if (!ctx || !out || !done) return LBE_BAD_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    auto it = ctx->jobs.find(ticket);
    if (it == ctx->jobs.end()) return bad_arg(ctx, "unknown ticket");
    *done = it->second->done;
    if (*done) *out = it->second->res;
    return LBE_OK;
}

lbe_status lbe_cancel(lbe_ctx* ctx, uint64_t ticket) {
    if (!ctx) return LBE_BAD_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    auto it = ctx->jobs.find(ticket);
    if (it == ctx->jobs.end()) return bad_arg(ctx, "unknown ticket");
    Job* j = it->second.get();
    if (j->done) return LBE_OK;
    j->cancel.store(1);
    auto q = std::find(ctx->queue.begin(), ctx->queue.end(), j);
    if (q != ctx->queue.end()) {  // not yet seen by the service
        ctx->queue.erase(q);
        j->res = lbe_result{};
        j->res.status = LBE_CANCELLED;
        j->done = 1;
    }
    ctx->cv.notify_all();
    return LBE_OK;
}

lbe_status lbe_set_max_active(lbe_ctx* ctx, int max_active) {
    if (!ctx || max_active < 1 || max_active > 4096) return LBE_BAD_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->max_active = max_active;
    return LBE_OK;
}

}  // extern "C"

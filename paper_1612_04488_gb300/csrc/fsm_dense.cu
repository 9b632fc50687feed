// Collision operator on the parity subspace as one tcgen05 GEMM (BF16 hi/lo, FP32 accumulate).
//
// Solutions of the plate and duct problems are odd in v3 (the source S of Sec. 2 is) and, on
// plates, even in v2.  The discrete operator commutes with each coordinate reflection
// R_k: v_k -> -v_k (the midpoint grid is symmetric and the direction set is closed under every
// R_k), so it maps the functions with given signs (s1, s2, s3) under (R1, R2, R3) into
// themselves.  Plate solutions live in the two subspaces s2 = +1, s3 = -1, s1 = +-1; duct
// solutions in the four with s3 = -1.  Each subspace is fixed by the values at one point per
// orbit of the eight reflections, p = (j1 H + j2) H + j3 with j_k < H = nv/2, so on it the
// operator (at delta = 1) is an NB x NB block, NB = H^3 = nv^3/8: two blocks for plates, four
// for ducts -- a half (plates) or a quarter (ducts) of the products of one parity-subspace
// matrix.  The blocks are built once per velocity grid by applying the fast-spectral operator
// in double-float arithmetic (FP64-class) to the symmetric basis functions of every block, so
// they are the same discrete operator.  Applying them to every cell at once is the GEMM
//     Y_b[c][q] = sum_p A_b[q][p] x_b[c][p],   L+ h_c = delta_c * expand(Y_b[c], all b),
// run with A = A_hi + A_lo and x = x_hi + x_lo split into bfloat16 and the three products
// A_hi x_hi + A_lo x_hi + A_hi x_lo accumulated in FP32 tensor memory (about 2^-16 relative).
//
// Kernels: operands staged by TMA (cp.async.bulk.tensor, 64-byte swizzle, 32-deep K slices)
// through an mbarrier stage ring; tcgen05.mma (M = 128, N = BN, K = 16) into TMEM; tcgen05.ld
// read-back.  Two forms of the same per-tile arithmetic: k_dense_gemm, one CTA per work item
// (one thread issues copies and MMAs; optional cluster multicast of the operator slices), and
// k_dense_gemm_ws, one persistent CTA per SM with a copy warp, an MMA warp and four read-back
// warps over two TMEM accumulators, so that a tile's read-back overlaps the next tile's
// products.  The autotuner times the forms per launch shape and keeps the fastest of those
// that reproduce the first one bit for bit.  Every wait is bounded: on expiry the kernel
// raises an error word, drains its own copies, frees its TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"
#include "lbe_internal.h"
#include "sweep.h"

namespace lbe {

namespace {

// kBK: K depth of one stage.  The operands are stored interleaved, [row][slice][hi 32 | lo 32]
// bf16, so one 128-byte row of a TMA box carries a slice's hi and lo halves.
constexpr int kBM = 128, kBK = 32, kRowB = 4 * kBK, kHalfB = 2 * kBK;
// index of the hi half of logical column col in an interleaved row (the lo half is 32 further)
__host__ __device__ inline long ilv(long col) { return (col / kBK) * 2 * kBK + col % kBK; }
constexpr int kSmemMax = 232448;  // opt-in dynamic shared memory per block
constexpr int kTmemCols = 256;    // accumulator columns allocated (power of two >= BN)

// Pipeline depth for a BN-wide tile: as many 32-deep K stages (A_hi, A_lo, x_hi, x_lo) as
// shared memory holds (max 8).
template <int BN>
struct GemmCfg {
    static constexpr int STAGE = 2 * kBM * kBK * 2 + 2 * BN * kBK * 2;
    static constexpr int STAGES = (kSmemMax - 1280) / STAGE < 8 ? (kSmemMax - 1280) / STAGE : 8;
    static constexpr size_t SMEM = (size_t)STAGES * STAGE + 1024 + 256;
};
constexpr long long kWaitCycles = 4000000000LL;  // ~2 s at 2 GHz
constexpr long long kProbeCycles = 100000LL;     // the test hook's wait, ~50 us

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
// Bounded wait on an mbarrier phase; false when the deadline passed.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long limit = kWaitCycles) {
    const uint32_t addr = smem_u32(bar);
    const long long t0 = clock64();
    for (;;) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(addr), "r"(parity)
            : "memory");
        if (ok) return true;
        if (clock64() - t0 > limit) return false;
    }
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst)),
        "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}
// The same with an L2 cache policy (createpolicy): the operator and the operands are re-read by
// many tiles and across calls, so they are kept in L2 ahead of streaming data.
__device__ __forceinline__ void tma_load_2d_hint(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar,
                                                 uint64_t policy) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1, {%2, "
        "%3}], [%4], %5;" ::"r"(smem_u32(dst)),
        "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar)), "l"(policy)
        : "memory");
}
__device__ __forceinline__ uint64_t policy_evict_last() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
// A tile slice copied into the same shared-memory offset of every CTA in `mask` (cluster
// multicast); each destination's mbarrier at the offset of `bar` receives its bytes.
__device__ __forceinline__ void tma_load_2d_mc(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar,
                                               uint16_t mask) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.multicast::cluster [%0], [%1, {%2, "
        "%3}], [%4], %5;" ::"r"(smem_u32(dst)),
        "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar)), "h"(mask)
        : "memory");
}
// arrive, when this CTA's issued MMAs are done, on the mbarrier at the offset of `bar` in
// every CTA of `mask`
__device__ __forceinline__ void mma_commit_mc(uint64_t* bar, uint16_t mask) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
                     smem_u32(bar)),
                 "h"(mask)
                 : "memory");
}
__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\nbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// One W-column chunk of a CTA's accumulator row r: into partial slot `slot` of P, or into Y.
template <int BN, int W>
__device__ __forceinline__ void emit_chunk(const float (&v)[W], int c0, int r, int row, int col0, int slot, int Mrows,
                                           int ncols, float* __restrict__ Y, float* __restrict__ P) {
    if (slot >= 0) {
        float* pt = P + (size_t)slot * BN * kBM;
#pragma unroll
        for (int j = 0; j < W; ++j) pt[(c0 + j) * kBM + r] = v[j];
    } else if (row < Mrows) {
#pragma unroll
        for (int j = 0; j < W; ++j) {
            const int col = col0 + c0 + j;
            if (col < ncols) Y[(long)col * Mrows + row] = v[j];
        }
    }
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle (rows of 64 bf16: the hi and lo
// halves of one 32-deep K slice side by side), 8-row groups 1024 B apart.  A start address
// 32, 64 or 96 bytes into the row selects the K16 step and the half.
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)(16 >> 4) << 16;    // leading byte offset (unused by swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;  // stride byte offset
    d |= (uint64_t)1 << 46;            // descriptor version
    d |= (uint64_t)2 << 61;            // 128-byte swizzle
    return d;
}

// Instruction descriptor: kind::f16 with bf16 A and B, f32 D, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Y_z[col][row] = sum over k in K-split z of (A_hi + A_lo)[row][k] (x_hi + x_lo)[col][k], without
// the A_lo x_lo term.  A stage holds one 32-deep K slice of all four operands, so A_hi is staged
// once for its two products: per stage 16 KB of A and 2 BN x 64 B of x feed 3 x 2 x 128 x BN x 32
// flops.
// One CTA per work item: a 128 x BN output tile and a range of its K slices.  slot < 0: the
// item covers all of K and stores its tile into Y; slot >= 0: a part of a split tile, stored
// whole into partial slot `slot` of P ([slot][BN][128]) for k_gemm_fixup to add up.
// With cs > 1 the launch is a cluster of cs CTAs whose items share the row tile and the K
// range (neighbouring column tiles): each CTA copies 128 / cs rows of every A slice and
// multicasts them to all, so A crosses from L2 once per cluster; a stage is refilled only
// when every CTA of the cluster has consumed it (each CTA's MMA commit arrives on the stage's
// empty barrier in all of them).  The arithmetic is that of cs = 1.
struct GemmWork {
    int col0, row0, xrow0, kt0, kt1, slot;  // xrow0: first operand row (block b: b * cpad + col0)
};

template <int BN>
__global__ void __launch_bounds__(128, 1)
    k_dense_gemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmX, int Mrows,
                 int ncols, const GemmWork* __restrict__ work, float* __restrict__ Y, float* __restrict__ P,
                 int* __restrict__ err, int probe, int cs) {
    constexpr int A_BYTES = kBM * kRowB, X_BYTES = BN * kRowB, STAGE = A_BYTES + X_BYTES;
    constexpr int kStages = GemmCfg<BN>::STAGES;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* base = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* full = (uint64_t*)(base + kStages * STAGE);
    uint64_t* empty = full + kStages;
    uint64_t* done = empty + kStages;
    uint64_t* never = done + 1;  // completed by nothing: the test hook waits on it
    uint32_t* tmem_slot = (uint32_t*)(done + 2);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const GemmWork wk = work[blockIdx.x];
    const int col0 = wk.col0, row0 = wk.row0, xrow0 = wk.xrow0, kt0 = wk.kt0;
    const int KT = wk.kt1 - wk.kt0;
    const uint32_t rank = cs > 1 ? cluster_rank() : 0u;
    const uint16_t cmask = (uint16_t)((1u << cs) - 1u);

    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], (uint32_t)cs);
        }
        mbar_init(done, 1);
        mbar_init(never, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (cs > 1) cluster_sync_all();  // every CTA's barriers exist before any multicast lands
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    constexpr uint32_t IDESC = idesc_bf16(kBM, BN);

    __shared__ int failed;
    if (tid == 0) failed = 0;

    if (tid == 0) {
        auto issue = [&](int kt, int s) {  // slice kt of this CTA's K range into stage s
            const int x = (kt0 + kt) * 2 * kBK;  // the slice's hi | lo pair in the interleaved rows
            uint8_t* st = base + s * STAGE;
            mbar_expect_tx(&full[s], STAGE);  // the whole stage lands here, A from every CTA
            if (cs == 1) {
                tma_load_2d(st, &tmA, x, row0, &full[s]);
            } else {
                const int rows = kBM / cs, off = (int)rank * rows;  // this CTA's slice of the A rows
                tma_load_2d_mc(st + off * kRowB, &tmA, x, row0 + off, &full[s], cmask);
            }
            tma_load_2d(st + A_BYTES, &tmX, x, xrow0, &full[s]);
        };
        int issued = 0;
        for (int s = 0; s < kStages && s < KT; ++s) issue(s, s), ++issued;
        int consumed = 0;
        // test hook: a short wait that cannot succeed takes the failure path below with the
        // first stages' copies in flight
        bool ok = probe ? mbar_wait(never, 0, kProbeCycles) : true;
        for (int kt = 0; ok && kt < KT; ++kt) {
            const int s = kt % kStages;
            if (!mbar_wait(&full[s], (kt / kStages) & 1)) {
                ok = false;
                break;
            }
            ++consumed;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t ah = smem_u32(base + s * STAGE), al = ah + kHalfB, xh = ah + A_BYTES, xl = xh + kHalfB;
#pragma unroll
            for (int k = 0; k < kBK / 16; ++k) {
                const uint32_t o = 32 * k;  // 16 bf16 along K inside the row's hi or lo half
                mma_bf16(tmem, sdesc_sw128(ah + o), sdesc_sw128(xh + o), IDESC, (kt > 0 || k > 0) ? 1u : 0u);
                mma_bf16(tmem, sdesc_sw128(al + o), sdesc_sw128(xh + o), IDESC, 1u);
                mma_bf16(tmem, sdesc_sw128(ah + o), sdesc_sw128(xl + o), IDESC, 1u);
            }
            if (cs > 1)
                mma_commit_mc(&empty[s], cmask);
            else
                mma_commit(&empty[s]);
            const int nk = kt - 1 + kStages;  // refill the slot of the previous stage
            if (kt >= 1 && nk < KT) {
                const int sp = (kt - 1) % kStages;
                if (!mbar_wait(&empty[sp], ((kt - 1) / kStages) & 1)) {
                    ok = false;
                    break;
                }
                issue(nk, sp);
                ++issued;
            }
        }
        if (!ok) {
            failed = 1;
            atomicExch(err, 1);
            // drain the loads still in flight before the shared memory goes away
            for (int kt = consumed; kt < issued; ++kt) mbar_wait(&full[kt % kStages], (kt / kStages) & 1);
        }
        mma_commit(done);
    }
    __syncthreads();  // the other threads wait here, not spinning beside the issuing thread
    const bool got = mbar_wait(done, 0);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    __syncthreads();
    if (got && !failed && KT > 0) {
        const int r = warp * 32 + lane, row = row0 + r;
        for (int c0 = 0; c0 + 32 <= BN; c0 += 32) {
            float v[32];
            tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + c0, v);
            emit_chunk<BN, 32>(v, c0, r, row, col0, wk.slot, Mrows, ncols, Y, P);
        }
        if constexpr (BN % 32 == 16) {  // last 16 columns
            float v[16];
            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (BN - 16), v);
            emit_chunk<BN, 16>(v, BN - 16, r, row, col0, wk.slot, Mrows, ncols, Y, P);
        }
    } else if (tid == 0 && KT > 0) {
        atomicExch(err, 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
    if (cs > 1) cluster_sync_all();  // no CTA leaves while its peers may still signal it
}

// ---- persistent, warp-specialised form ----------------------------------------------------
// One CTA per SM runs a list of work items: the same items, each with the MMA order of
// k_dense_gemm, so Y is bitwise the same.  Warp 0 (one lane) streams the K slices of all the
// CTA's items through the stage ring; warp 1 (one lane) issues the MMAs into one of two TMEM
// accumulators, item after item; warps 2-5 read a finished accumulator back (warp w reads TMEM
// lanes 32 (w % 4) ..) while the next item accumulates in the other.  Barriers: full / empty per
// stage (copy -> MMA -> copy) and tfull / tempty per accumulator (MMA -> read-back -> MMA).
// Every wait is bounded and also ends once another role has failed (the shared abort flag); on
// failure the CTA waits for its copies and MMAs in flight before it frees TMEM and returns.
constexpr int kTmemCols2 = 512;  // two accumulators, 256 columns apart
constexpr int kPersistent = 8;   // the autotuner's code for this form (1, 2, 4: cluster sizes)

__device__ __forceinline__ bool mbar_wait_ab(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                             long long limit = kWaitCycles) {
    const uint32_t addr = smem_u32(bar);
    const long long t0 = clock64();
    for (int it = 0;; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(addr), "r"(parity)
            : "memory");
        if (ok) return true;
        if ((it & 31) == 31 && *abort_flag) return false;
        if (clock64() - t0 > limit) return false;
    }
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

template <int BN>
__global__ void __launch_bounds__(192, 1)
    k_dense_gemm_ws(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmX, int Mrows,
                    int ncols, const GemmWork* __restrict__ work, const int* __restrict__ cta_off,
                    float* __restrict__ Y, float* __restrict__ P, int* __restrict__ err, int probe) {
    constexpr int A_BYTES = kBM * kRowB, X_BYTES = BN * kRowB, STAGE = A_BYTES + X_BYTES;
    constexpr int kStages = GemmCfg<BN>::STAGES;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* base = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* full = (uint64_t*)(base + kStages * STAGE);
    uint64_t* empty = full + kStages;
    uint64_t* tfull = empty + kStages;  // [2]
    uint64_t* tempty = tfull + 2;       // [2]
    uint64_t* mdone = tempty + 2;       // every MMA the CTA issued is complete
    uint64_t* never = mdone + 1;        // completed by nothing: the test hook waits on it
    uint32_t* tmem_slot = (uint32_t*)(never + 1);
    __shared__ int abort_flag, n_issued, n_consumed;  // K slices copied / consumed (drain)
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int i0 = cta_off[blockIdx.x], i1 = cta_off[blockIdx.x + 1];
    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&tfull[a], 1);
            mbar_init(&tempty[a], 4);  // one arrival per read-back warp
        }
        mbar_init(mdone, 1);
        mbar_init(never, 1);
        abort_flag = 0;
        n_issued = 0;
        n_consumed = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kTmemCols2));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    constexpr uint32_t IDESC = idesc_bf16(kBM, BN);
    volatile int* ab = &abort_flag;

    if (warp == 0) {
        if (lane == 0) {  // producer: every K slice of every item, in order
            int g = 0;
            bool ok = true;
            const uint64_t keep = policy_evict_last();
            for (int it = i0; ok && it < i1; ++it) {
                const GemmWork wk = work[it];
                for (int kt = wk.kt0; kt < wk.kt1; ++kt, ++g) {
                    const int s = g % kStages;
                    if (g >= kStages && !mbar_wait_ab(&empty[s], ((g / kStages) - 1) & 1, ab)) {
                        ok = false;
                        break;
                    }
                    const int x = kt * 2 * kBK;  // the slice's hi | lo pair in the interleaved rows
                    uint8_t* st = base + s * STAGE;
                    mbar_expect_tx(&full[s], STAGE);
                    tma_load_2d_hint(st, &tmA, x, wk.row0, &full[s], keep);
                    tma_load_2d_hint(st + A_BYTES, &tmX, x, wk.xrow0, &full[s], keep);
                    n_issued = g + 1;
                }
            }
            if (!ok) {
                *ab = 1;
                atomicExch(err, 1);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {  // MMA issue: item n accumulates in accumulator n & 1
            int g = 0, n = 0;
            // test hook: a short wait that cannot succeed takes the failure path with the first
            // stages' copies in flight
            bool ok = probe ? mbar_wait(never, 0, kProbeCycles) : true;
            for (int it = i0; ok && it < i1; ++it, ++n) {
                const GemmWork wk = work[it];
                const int a = n & 1;
                if (n >= 2 && !mbar_wait_ab(&tempty[a], ((n >> 1) - 1) & 1, ab)) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t acc = tmem + (uint32_t)(a * 256);
                const int KT = wk.kt1 - wk.kt0;
                for (int kt = 0; kt < KT; ++kt, ++g) {
                    const int s = g % kStages;
                    if (!mbar_wait_ab(&full[s], (g / kStages) & 1, ab)) {
                        ok = false;
                        break;
                    }
                    n_consumed = g + 1;
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t ah = smem_u32(base + s * STAGE), al = ah + kHalfB, xh = ah + A_BYTES,
                                   xl = xh + kHalfB;
#pragma unroll
                    for (int k = 0; k < kBK / 16; ++k) {
                        const uint32_t o = 32 * k;
                        mma_bf16(acc, sdesc_sw128(ah + o), sdesc_sw128(xh + o), IDESC, (kt > 0 || k > 0) ? 1u : 0u);
                        mma_bf16(acc, sdesc_sw128(al + o), sdesc_sw128(xh + o), IDESC, 1u);
                        mma_bf16(acc, sdesc_sw128(ah + o), sdesc_sw128(xl + o), IDESC, 1u);
                    }
                    mma_commit(&empty[s]);
                }
                if (!ok) break;
                mma_commit(&tfull[a]);
            }
            if (!ok) {
                *ab = 1;
                atomicExch(err, 1);
            }
            mma_commit(mdone);
        }
    } else {  // read-back: warp w owns TMEM lanes (w % 4) * 32 ..
        const int q = warp & 3, r = q * 32 + lane;
        int n = 0;
        for (int it = i0; it < i1; ++it, ++n) {
            const GemmWork wk = work[it];
            const int a = n & 1;
            const bool got = __all_sync(0xffffffffu, mbar_wait_ab(&tfull[a], (n >> 1) & 1, ab));
            if (!got) {
                if (lane == 0) {
                    *ab = 1;
                    atomicExch(err, 1);
                }
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t ta = tmem + (uint32_t)(a * 256) + ((uint32_t)(q * 32) << 16);
            const int row = wk.row0 + r;
            for (int c0 = 0; c0 + 32 <= BN; c0 += 32) {
                float v[32];
                tmem_ld32(ta + c0, v);
                emit_chunk<BN, 32>(v, c0, r, row, wk.col0, wk.slot, Mrows, ncols, Y, P);
            }
            if constexpr (BN % 32 == 16) {
                float v[16];
                tmem_ld16(ta + (BN - 16), v);
                emit_chunk<BN, 16>(v, BN - 16, r, row, wk.col0, wk.slot, Mrows, ncols, Y, P);
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[a]);
        }
    }
    __syncthreads();
    if (warp == 1 && lane == 0) mbar_wait(mdone, 0);  // no MMA writes TMEM after the free
    if (tid == 0 && abort_flag)  // copies issued but never consumed land before the CTA leaves
        for (int g = n_consumed; g < n_issued; ++g) mbar_wait(&full[g % kStages], (g / kStages) & 1);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols2));
}

// ---- reflection blocks and their transposition halves ------------------------------------
// Block b has s1 = -1 when bit 0 of b is set and s2 = -1 when bit 1 is set (ducts; plates use
// b = 0, 1 with s2 = +1); s3 = -1 always.  The operator also commutes with the transposition
// T: (v1, v2) -> (v2, v1) (the cubic grid is symmetric and the direction set is closed under it:
// T maps azimuth phi to pi/2 - phi, a midpoint azimuth when their number is a multiple of 4,
// i.e. M >= 8).  T maps the blocks with s1 = s2 (b = 0, and b = 3 for ducts) into themselves,
// and there they split once more into functions even and odd under T, indexed by the unordered
// pairs (a <= b) or (a < b) of (j1, j2) times j3:
//     ts(a, b) = b (b + 1) / 2 + a,   ta(a, b) = b (b - 1) / 2 + a.
// So the GEMM runs over sub-blocks: plates {S0, A0, F1}, ducts {S0, A0, F1, F2, S3, A3} (F: a
// whole block, S / A: the even / odd half of one), (nv/2)^3 (H + 1) / (2 H) and
// (nv/2)^3 (H - 1) / (2 H) square for the halves -- three quarters of the products of the
// blocks.  Every sub-block is padded to the 128-row tile (padding rows and columns of A are
// zero); its rows start at roff in the stacked A, and its cell operands at rows k * cpad of X,
// npmax columns wide.
struct SubLayout {
    int count = 0;
    int kind[6] = {};  // 0 whole block, 1 even half, 2 odd half
    int blk[6] = {};
    int n[6] = {};     // logical size
    int np[6] = {};    // padded size
    int roff[6] = {};  // first row in the stacked A
    int soff[6] = {};  // first value in a cell's compact output (expand)
    int rows = 0, npmax = 0;
};
__host__ __device__ constexpr int pad128(int n) { return (n + 127) / 128 * 128; }
__host__ __device__ constexpr SubLayout sub_layout(int nv, int mode) {
    SubLayout L;
    const int H = nv / 2, nf = H * H * H, ns = H * (H + 1) / 2 * H, na = H * (H - 1) / 2 * H;
    const int kinds_p[3] = {1, 2, 0}, blks_p[3] = {0, 0, 1};
    const int kinds_d[6] = {1, 2, 0, 0, 1, 2}, blks_d[6] = {0, 0, 1, 2, 3, 3};
    L.count = mode == 2 ? 3 : 6;
    int r = 0, so = 0;
    for (int k = 0; k < L.count; ++k) {
        L.kind[k] = mode == 2 ? kinds_p[k] : kinds_d[k];
        L.blk[k] = mode == 2 ? blks_p[k] : blks_d[k];
        L.n[k] = L.kind[k] == 0 ? nf : (L.kind[k] == 1 ? ns : na);
        L.np[k] = pad128(L.n[k]);
        L.roff[k] = r;
        L.soff[k] = so;
        r += L.np[k];
        so += L.n[k];
        if (L.np[k] > L.npmax) L.npmax = L.np[k];
    }
    L.rows = r;
    return L;
}
__host__ __device__ constexpr int ts_idx(int a, int b) { return b * (b + 1) / 2 + a; }
__host__ __device__ constexpr int ta_idx(int a, int b) { return b * (b - 1) / 2 + a; }
// sign of block b at a velocity point in the mirror halves m1, m2, m3
__host__ __device__ inline bool blk_neg(int b, int mode, bool m1, bool m2, bool m3) {
    int neg = m3 ? 1 : 0;
    if (b & 1) neg += m1 ? 1 : 0;
    if (mode == 1 && (b & 2)) neg += m2 ? 1 : 0;
    return neg & 1;
}

// x of every sub-block (hi / lo bf16 interleaved per 32-column slice, [sub-block][cpad][2 npmax])
// from h (float).  Block
// coefficients: the signed average of h over the reflections that the parity leaves free --
// plates x_b = (h(p) +- h(R1 p)) / 2, ducts x_b = (h(p) +- h(R1 p) +- h(R2 p) +- h(R1 R2 p)) / 4;
// halves: (x_b(a, b) +- x_b(b, a)) / 2.  Each thread takes one unordered pair a <= b of (j1, j2)
// and two neighbouring j3 (H is even): float2 loads of both orders' orbit points, bf16x2
// stores.  A second loop writes the padding columns of every sub-block as zero.
// quarter: h in the orbit layout, where the points read are stored at (i1 nv / 2 + i2) nv / 2 +
// i3 (plates: i2, i3 < nv / 2) or (i1 nv + i2) nv / 2 + i3 (ducts: i3 < nv / 2).
template <int NV, int MODE>
__global__ void __launch_bounds__(256) k_gather_sub(const float* __restrict__ h, __nv_bfloat162* __restrict__ xo,
                                                    int cells, int cpad, int quarter) {
    constexpr int H = NV / 2, NBLK = MODE == 2 ? 2 : 4, NPAIR = H * (H + 1) / 2;
    const int R2 = MODE == 2 && quarter ? H : NV, R3 = quarter ? H : NV;  // i2, i3 values of the data
    constexpr SubLayout L = sub_layout(NV, MODE);
    constexpr long N3 = (long)NV * NV * NV;
    const long total = (long)cells * NPAIR * (H / 2);
    auto put = [&](int k, long c, int idx, float2 v) {  // idx even: the pair stays in one slice
        const long o = (((long)k * cpad + c) * 2 * L.npmax + ilv(idx)) / 2;
        const __nv_bfloat162 hi = __floats2bfloat162_rn(v.x, v.y);
        const float2 hf = __bfloat1622float2(hi);
        xo[o] = hi;
        xo[o + kBK / 2] = __floats2bfloat162_rn(v.x - hf.x, v.y - hf.y);
    };
    for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < total; k += (long)gridDim.x * blockDim.x) {
        const long c = k / (NPAIR * (H / 2));
        const int r = (int)(k % (NPAIR * (H / 2)));
        const int t = r / (H / 2), j3 = 2 * (r % (H / 2));
        int bb = 0;
        while ((bb + 1) * (bb + 2) / 2 <= t) ++bb;
        const int aa = t - bb * (bb + 1) / 2;  // aa <= bb
        const float* hc = h + c * N3;
        float2 x[2][NBLK];  // [order: (aa, bb), (bb, aa)][block]
#pragma unroll
        for (int o = 0; o < 2; ++o) {
            const int j1 = o ? bb : aa, j2 = o ? aa : bb;
            const float2 p0 = *reinterpret_cast<const float2*>(hc + (j1 * R2 + j2) * R3 + j3);
            const float2 p1 = *reinterpret_cast<const float2*>(hc + ((NV - 1 - j1) * R2 + j2) * R3 + j3);
            if constexpr (MODE == 2) {
                x[o][0] = make_float2(0.5f * (p0.x + p1.x), 0.5f * (p0.y + p1.y));
                x[o][1] = make_float2(0.5f * (p0.x - p1.x), 0.5f * (p0.y - p1.y));
            } else {
                const float2 p2 = *reinterpret_cast<const float2*>(hc + (j1 * R2 + (NV - 1 - j2)) * R3 + j3);
                const float2 p3 = *reinterpret_cast<const float2*>(hc + ((NV - 1 - j1) * R2 + (NV - 1 - j2)) * R3 + j3);
                const float2 s0 = make_float2(p0.x + p1.x, p0.y + p1.y), d0 = make_float2(p0.x - p1.x, p0.y - p1.y);
                const float2 s1 = make_float2(p2.x + p3.x, p2.y + p3.y), d1 = make_float2(p2.x - p3.x, p2.y - p3.y);
                x[o][0] = make_float2(0.25f * (s0.x + s1.x), 0.25f * (s0.y + s1.y));
                x[o][1] = make_float2(0.25f * (d0.x + d1.x), 0.25f * (d0.y + d1.y));
                x[o][2] = make_float2(0.25f * (s0.x - s1.x), 0.25f * (s0.y - s1.y));
                x[o][3] = make_float2(0.25f * (d0.x - d1.x), 0.25f * (d0.y - d1.y));
            }
        }
#pragma unroll
        for (int q = 0; q < L.count; ++q) {
            const int b = L.blk[q];
            if (L.kind[q] == 0) {
                put(q, c, (aa * H + bb) * H + j3, x[0][b]);
                if (aa != bb) put(q, c, (bb * H + aa) * H + j3, x[1][b]);
            } else if (L.kind[q] == 1) {
                const float2 v = aa == bb ? x[0][b]
                                          : make_float2(0.5f * (x[0][b].x + x[1][b].x), 0.5f * (x[0][b].y + x[1][b].y));
                put(q, c, ts_idx(aa, bb) * H + j3, v);
            } else if (aa != bb) {
                put(q, c, ta_idx(aa, bb) * H + j3,
                    make_float2(0.5f * (x[0][b].x - x[1][b].x), 0.5f * (x[0][b].y - x[1][b].y)));
            }
        }
    }
    // padding columns
    int npad = 0;
#pragma unroll
    for (int q = 0; q < L.count; ++q) npad += (L.np[q] - L.n[q]) / 2;
    const long ptotal = (long)cells * npad;
    const __nv_bfloat162 z = __floats2bfloat162_rn(0.f, 0.f);
    for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < ptotal; k += (long)gridDim.x * blockDim.x) {
        const long c = k / npad;
        int r = (int)(k % npad), q = 0;
        while (r >= (L.np[q] - L.n[q]) / 2) {
            r -= (L.np[q] - L.n[q]) / 2;
            ++q;
        }
        const long o = (((long)q * cpad + c) * 2 * L.npmax + ilv(L.n[q] + 2 * r)) / 2;
        xo[o] = z;
        xo[o + kBK / 2] = z;
    }
}

// L+ h = delta s3 sum_b s_b y_b for every velocity point of a cell, y_b from the block's whole
// output or from its two halves (y_b(j1, j2) = Ys(a, b) +- Ya(a, b), + for j1 <= j2);
// optionally L h = L+ h - delta nu h, and optionally the SIS L-moments
// G_j = 2 sum_v v_j v3 (L h + N delta h) dv^3 (j = 1, 2) in the same pass, without storing L h.
// With hm (the h part of G summed when h was written, see launch_correct) and no L h wanted,
// G_j = 2 sum_v v_j v3 L+ h dv^3 + hm_j and h is not read at all.
// One block of 8 NV threads per cell stages the cell's sub-block outputs in shared memory.
template <int NV, int MODE>
__global__ void __launch_bounds__(8 * NV) k_expand_sub(const float* __restrict__ Y, const float* __restrict__ h,
                                                       const float* __restrict__ nu1, const float* __restrict__ vel,
                                                       const double* __restrict__ delta, const double* __restrict__ nd,
                                                       float* __restrict__ Lplus, float* __restrict__ Lout,
                                                       double* __restrict__ G, double dv3,
                                                       const double* __restrict__ hm) {
    extern __shared__ float sY[];
    __shared__ dfloat redx[32 * 2];
    constexpr int H = NV / 2, NBLK = MODE == 2 ? 2 : 4;
    constexpr SubLayout L = sub_layout(NV, MODE);
    constexpr long n3 = (long)NV * NV * NV;
    const long c = blockIdx.x;
    const float* yc = Y + c * (long)L.rows;
#pragma unroll
    for (int q = 0; q < L.count; ++q)
        for (int k = threadIdx.x; k < L.n[q]; k += blockDim.x) sY[L.soff[q] + k] = yc[L.roff[q] + k];
    __syncthreads();
    const float d = (float)delta[c];
    const float ndc = G ? (float)nd[c] : 0.f;
    const int i3 = threadIdx.x % NV, r0 = threadIdx.x / NV;
    const bool m3 = i3 >= H;
    const int j3 = m3 ? NV - 1 - i3 : i3;
    const float v3 = vel[i3];
    float a0 = 0.f, c0 = 0.f, a1 = 0.f, c1 = 0.f;  // compensated sums of v1 t and v2 t
    auto kahan = [](float& sum, float& comp, float x) {
        const float y = x - comp;
        const float t = sum + y;
        comp = (t - sum) - y;
        sum = t;
    };
    for (int i1 = 0; i1 < NV; ++i1) {
        const float v1 = vel[i1];
        const bool m1 = i1 >= H;
        const int j1 = m1 ? NV - 1 - i1 : i1;
#pragma unroll
        for (int k = 0; k < NV / 8; ++k) {
            const int i2 = r0 + 8 * k;
            const bool m2 = i2 >= H;
            const int j2 = m2 ? NV - 1 - i2 : i2;
            const int aa = j1 <= j2 ? j1 : j2, bb = j1 <= j2 ? j2 : j1;
            float yb[NBLK];
#pragma unroll
            for (int q = 0; q < L.count; ++q) {
                const int b = L.blk[q];
                if (L.kind[q] == 0) {
                    yb[b] = sY[L.soff[q] + (j1 * H + j2) * H + j3];
                } else if (L.kind[q] == 1) {
                    yb[b] = sY[L.soff[q] + ts_idx(aa, bb) * H + j3];
                } else if (aa != bb) {
                    const float ya = sY[L.soff[q] + ta_idx(aa, bb) * H + j3];
                    yb[b] += j1 < j2 ? ya : -ya;
                }
            }
            float y = 0.f;
#pragma unroll
            for (int b = 0; b < NBLK; ++b) y += blk_neg(b, MODE, m1, m2, false) ? -yb[b] : yb[b];
            const int v = (i1 * NV + i2) * NV + i3;
            const long g = c * n3 + v;
            const float lp = (m3 ? -d : d) * y;
            Lplus[g] = lp;
            if (hm && !Lout) {
                if (G) {
                    const float t = lp * v3;
                    kahan(a0, c0, v1 * t);
                    kahan(a1, c1, vel[i2] * t);
                }
            } else if (Lout || G) {
                const float hv = h[g];
                const float lo = lp - d * nu1[v] * hv;
                if (Lout) Lout[g] = lo;
                if (G) {
                    const float t = (lo + ndc * hv) * v3;
                    kahan(a0, c0, v1 * t);
                    kahan(a1, c1, vel[i2] * t);
                }
            }
        }
    }
    if (!G) return;
    dfloat sm[2] = {df_fast2sum(a0, -c0), df_fast2sum(a1, -c1)};  // reduced in double-float
    block_reduce_df<2>(sm, redx);
    if (threadIdx.x == 0) {
        const bool add = hm && !Lout;
        G[2 * c + 0] = 2.0 * (double)sm[0] * dv3 + (add ? hm[2 * c + 0] : 0.0);
        G[2 * c + 1] = 2.0 * (double)sm[1] * dv3 + (add ? hm[2 * c + 1] : 0.0);
    }
}

// The plate expand in the orbit layout: L+ h at the stored quarter only (i2, i3 < nv / 2, where
// the R2 and R3 signs are +1), optionally L h = L+ h - delta nu h (h in the orbit layout), and
// optionally G_1 = 2 sum_v v1 v3 L+ h dv^3 + hm_1 as four times the quarter's sum (v1 v3 L+ h is
// even under R2 and R3); G_2's summand is odd under R2, so G_2 = hm_2.  The per-point arithmetic
// is that of k_expand_sub.
template <int NV>
__global__ void __launch_bounds__(256) k_expand_q(const float* __restrict__ Y, const float* __restrict__ vel,
                                                     const double* __restrict__ delta, float* __restrict__ Lplus,
                                                     double* __restrict__ G, double dv3,
                                                     const double* __restrict__ hm, const float* __restrict__ h,
                                                     const float* __restrict__ nu1, float* __restrict__ Lout) {
    extern __shared__ __align__(16) float sY[];
    __shared__ dfloat redx[32 * 2];
    constexpr int H = NV / 2;
    constexpr SubLayout L = sub_layout(NV, 2);  // S0, A0 (block 0), F1 (block 1)
    constexpr long n3 = (long)NV * NV * NV;
    const long c = blockIdx.x;
    const float* yc = Y + c * (long)L.rows;
    // the cell's sub-block outputs into shared memory, 16 bytes per asynchronous copy, all in
    // flight at once (every sub-block's length and offsets are multiples of 4 floats)
#pragma unroll
    for (int q = 0; q < L.count; ++q)
        for (int k = 4 * threadIdx.x; k < L.n[q]; k += 4 * blockDim.x)
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(sY + L.soff[q] + k)),
                         "l"(yc + L.roff[q] + k)
                         : "memory");
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;" ::: "memory");
    __syncthreads();
    const float d = (float)delta[c];
    float a0 = 0.f, c0 = 0.f;  // compensated sum of v1 v3 L+ h
    for (int p = threadIdx.x; p < NV * H * H; p += blockDim.x) {
        const int i1 = p / (H * H), j2 = (p / H) % H, j3 = p % H;
        const bool m1 = i1 >= H;
        const int j1 = m1 ? NV - 1 - i1 : i1;
        const int aa = j1 <= j2 ? j1 : j2, bb = j1 <= j2 ? j2 : j1;
        float y0 = sY[L.soff[0] + ts_idx(aa, bb) * H + j3];
        if (aa != bb) {
            const float ya = sY[L.soff[1] + ta_idx(aa, bb) * H + j3];
            y0 += j1 < j2 ? ya : -ya;
        }
        const float y1 = sY[L.soff[2] + (j1 * H + j2) * H + j3];
        const float lp = d * (m1 ? y0 - y1 : y0 + y1);
        Lplus[c * n3 + p] = lp;
        if (Lout) Lout[c * n3 + p] = lp - d * nu1[(i1 * NV + j2) * NV + j3] * h[c * n3 + p];
        if (G) {
            const float t = lp * vel[j3];
            const float x = vel[i1] * t - c0;
            const float u = a0 + x;
            c0 = (u - a0) - x;
            a0 = u;
        }
    }
    if (!G) return;
    dfloat sm[2] = {df_fast2sum(a0, -c0), dfloat(0)};
    block_reduce_df<2>(sm, redx);
    if (threadIdx.x == 0) {
        G[2 * c + 0] = 8.0 * (double)sm[0] * dv3 + hm[2 * c + 0];
        G[2 * c + 1] = hm[2 * c + 1];
    }
}

// The duct expand in the orbit layout: L+ h at the stored half only (i3 < nv / 2, where the R3
// sign is +1), optionally L h = L+ h - delta nu h (h in the orbit layout), and optionally
// G_j = 2 sum_v v_j v3 L+ h dv^3 + hm_j as twice the half's sum (v_j v3 L+ h is even under R3).
// The per-point arithmetic is that of k_expand_sub.
template <int NV>
__global__ void __launch_bounds__(256) k_expand_h(const float* __restrict__ Y, const float* __restrict__ vel,
                                                  const double* __restrict__ delta, float* __restrict__ Lplus,
                                                  double* __restrict__ G, double dv3,
                                                  const double* __restrict__ hm, const float* __restrict__ h,
                                                  const float* __restrict__ nu1, float* __restrict__ Lout) {
    extern __shared__ __align__(16) float sY[];
    __shared__ dfloat redx[32 * 2];
    constexpr int H = NV / 2;
    constexpr SubLayout L = sub_layout(NV, 1);  // S0, A0 (block 0), F1, F2, S3, A3 (block 3)
    constexpr long n3 = (long)NV * NV * NV;
    const long c = blockIdx.x;
    const float* yc = Y + c * (long)L.rows;
#pragma unroll
    for (int q = 0; q < L.count; ++q)
        for (int k = 4 * threadIdx.x; k < L.n[q]; k += 4 * blockDim.x)
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(sY + L.soff[q] + k)),
                         "l"(yc + L.roff[q] + k)
                         : "memory");
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;" ::: "memory");
    __syncthreads();
    const float d = (float)delta[c];
    float a0 = 0.f, c0 = 0.f, a1 = 0.f, c1 = 0.f;  // compensated sums of v1 v3 L+ h, v2 v3 L+ h
    auto kahan = [](float& sum, float& comp, float x) {
        const float y = x - comp;
        const float t = sum + y;
        comp = (t - sum) - y;
        sum = t;
    };
    for (int p = threadIdx.x; p < NV * NV * H; p += blockDim.x) {
        const int i1 = p / (NV * H), i2 = (p / H) % NV, j3 = p % H;
        const bool m1 = i1 >= H, m2 = i2 >= H;
        const int j1 = m1 ? NV - 1 - i1 : i1, j2 = m2 ? NV - 1 - i2 : i2;
        const int aa = j1 <= j2 ? j1 : j2, bb = j1 <= j2 ? j2 : j1;
        float yb[4];
#pragma unroll
        for (int q = 0; q < L.count; ++q) {
            const int b = L.blk[q];
            if (L.kind[q] == 0) {
                yb[b] = sY[L.soff[q] + (j1 * H + j2) * H + j3];
            } else if (L.kind[q] == 1) {
                yb[b] = sY[L.soff[q] + ts_idx(aa, bb) * H + j3];
            } else if (aa != bb) {
                const float ya = sY[L.soff[q] + ta_idx(aa, bb) * H + j3];
                yb[b] += j1 < j2 ? ya : -ya;
            }
        }
        float y = 0.f;
#pragma unroll
        for (int b = 0; b < 4; ++b) y += blk_neg(b, 1, m1, m2, false) ? -yb[b] : yb[b];
        const float lp = d * y;
        Lplus[c * n3 + p] = lp;
        if (Lout) Lout[c * n3 + p] = lp - d * nu1[(i1 * NV + i2) * NV + j3] * h[c * n3 + p];
        if (G) {
            const float t = lp * vel[j3];
            kahan(a0, c0, vel[i1] * t);
            kahan(a1, c1, vel[i2] * t);
        }
    }
    if (!G) return;
    dfloat sm[2] = {df_fast2sum(a0, -c0), df_fast2sum(a1, -c1)};
    block_reduce_df<2>(sm, redx);
    if (threadIdx.x == 0) {
        G[2 * c + 0] = 4.0 * (double)sm[0] * dv3 + hm[2 * c + 0];
        G[2 * c + 1] = 4.0 * (double)sm[1] * dv3 + hm[2 * c + 1];
    }
}

template <int NV>
void launch_expand_h(int cells, const float* Y, const float* vel, const double* delta, float* Lplus, double* G,
                     double dv3, const double* hm, const float* h, const float* nu1, float* Lout, cudaStream_t s) {
    static std::once_flag once;
    constexpr int H = NV / 2;
    const int smem = 4 * H * H * H * 4;
    std::call_once(once, [smem] {
        cudaFuncSetAttribute(k_expand_h<NV>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    });
    k_expand_h<NV><<<cells, 256, smem, s>>>(Y, vel, delta, Lplus, G, dv3, hm, h, nu1, Lout);
}

template <int NV, int MODE>
void launch_gather(int cells, int cpad, const float* h, __nv_bfloat162* x, cudaStream_t s, int quarter) {
    k_gather_sub<NV, MODE><<<8 * sm_count(), 256, 0, s>>>(h, x, cells, cpad, quarter);
}

template <int NV>
void launch_expand_q(int cells, const float* Y, const float* vel, const double* delta, float* Lplus, double* G,
                     double dv3, const double* hm, const float* h, const float* nu1, float* Lout, cudaStream_t s) {
    static std::once_flag once;
    constexpr int H = NV / 2;
    const int smem = 2 * H * H * H * 4;
    std::call_once(once, [smem] {
        cudaFuncSetAttribute(k_expand_q<NV>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    });
    constexpr int pts = NV * H * H, threads = pts >= 256 ? 256 : (pts + 31) / 32 * 32;
    k_expand_q<NV><<<cells, threads, smem, s>>>(Y, vel, delta, Lplus, G, dv3, hm, h, nu1, Lout);
}

template <int NV, int MODE>
void launch_expand(int cells, const float* Y, const float* h, const float* nu1, const float* vel, const double* delta,
                   const double* nd, float* Lplus, float* Lout, double* G, double dv3, const double* hm,
                   cudaStream_t s) {
    static std::once_flag once;
    constexpr int H = NV / 2;
    const int smem = (MODE == 2 ? 2 : 4) * H * H * H * 4;
    std::call_once(once, [smem] {
        cudaFuncSetAttribute(k_expand_sub<NV, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    });
    k_expand_sub<NV, MODE><<<cells, 8 * NV, smem, s>>>(Y, h, nu1, vel, delta, nd, Lplus, Lout, G, dv3, hm);
}

// Column col of sub-block q: its canonical (a, b, j3) -- (j1, j2, j3) of a whole block, or the
// unordered pair of a half.
__host__ __device__ inline void sub_column(const SubLayout& L, int q, int col, int H, int* pa, int* pb, int* p3) {
    *p3 = col % H;
    const int t = col / H;
    if (L.kind[q] == 0) {
        *pa = t / H;
        *pb = t % H;
        return;
    }
    int b = L.kind[q] == 1 ? 0 : 1;
    if (L.kind[q] == 1)
        while ((b + 1) * (b + 2) / 2 <= t) ++b;
    else
        while ((b + 1) * b / 2 <= t) ++b;
    *pb = b;
    *pa = t - (L.kind[q] == 1 ? b * (b + 1) / 2 : b * (b - 1) / 2);
}

// Basis functions for the global columns g0 .. g0 + nbas - 1 (sub-block by sub-block): the
// block-b function of the orbit of (a, b, j3) (value s3 s_b on its eight points), for a half
// plus (even) or minus (odd) that of (b, a, j3).
__global__ void k_basis_sub(double* __restrict__ h, int g0, int nbas, int nv, int mode) {
    const SubLayout L = sub_layout(nv, mode);
    const int H = nv / 2;
    const long n3 = (long)nv * nv * nv;
    const long total = (long)nbas * n3;
    for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < total; k += (long)gridDim.x * blockDim.x) {
        int gi = g0 + (int)(k / n3), q = 0;
        while (gi >= L.n[q]) gi -= L.n[q++];
        int pa, pb, p3;
        sub_column(L, q, gi, H, &pa, &pb, &p3);
        const int v = (int)(k % n3);
        const int i1 = v / (nv * nv), i2 = (v / nv) % nv, i3 = v % nv;
        const bool m1 = i1 >= H, m2 = i2 >= H, m3 = i3 >= H;
        const int j1 = m1 ? nv - 1 - i1 : i1, j2 = m2 ? nv - 1 - i2 : i2, j3 = m3 ? nv - 1 - i3 : i3;
        double val = 0.0;
        if (j3 == p3) {
            const double sg = blk_neg(L.blk[q], mode, m1, m2, m3) ? -1.0 : 1.0;
            if (j1 == pa && j2 == pb) val += sg;
            if (L.kind[q] != 0 && pa != pb && j1 == pb && j2 == pa) val += L.kind[q] == 1 ? sg : -sg;
        }
        h[k] = val;
    }
}

// Columns g0 .. g0 + nbas - 1 of the stacked sub-blocks (row-major [rows][2 npmax], hi / lo
// bf16 interleaved per 32-column slice) from L+ e at the representative point of each output
// row.
__global__ void k_store_sub(const double* __restrict__ Lp, __nv_bfloat16* __restrict__ A, int g0, int nbas,
                            int nv, int mode) {
    const SubLayout L = sub_layout(nv, mode);
    const int H = nv / 2;
    const long n3 = (long)nv * nv * nv;
    int nmax = 0;
    for (int q = 0; q < L.count; ++q) nmax = L.n[q] > nmax ? L.n[q] : nmax;
    const long total = (long)nbas * nmax;
    for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < total; k += (long)gridDim.x * blockDim.x) {
        const long bb = k / nmax;  // basis function of this chunk
        const int row = (int)(k % nmax);
        int col = g0 + (int)bb, q = 0;
        while (col >= L.n[q]) col -= L.n[q++];
        if (row >= L.n[q]) continue;
        int qa, qb, q3;
        sub_column(L, q, row, H, &qa, &qb, &q3);
        const double a = Lp[bb * n3 + (qa * nv + qb) * nv + q3];
        const __nv_bfloat16 hi = __float2bfloat16_rn((float)a);
        const long idx = (long)(L.roff[q] + row) * 2 * L.npmax + ilv(col);
        A[idx] = hi;
        A[idx + 32] = __float2bfloat16_rn((float)(a - (double)__bfloat162float(hi)));
    }
}

PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    });
    return fn;
}

// Tensor map of an interleaved operand [rows][2 cols] bf16 (cols: its logical width): boxes of
// one 32-deep slice's hi | lo pair (128 bytes) by box_rows, 128-byte swizzle.
bool make_map(CUtensorMap* m, const void* ptr, long rows, long cols, int box_rows) {
    auto enc = get_encode();
    if (!enc) return false;
    cuuint64_t dims[2] = {(cuuint64_t)(2 * cols), (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)cols * 4};
    cuuint32_t box[2] = {(cuuint32_t)(2 * kBK), (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}


// Column tile for a call: the cells split evenly over ceil(cells / 256) tiles, rounded up to
// the next instantiated width (808 cells: 4 x 208 = 832 columns instead of 4 x 256).
constexpr int kWidths[] = {64, 128, 160, 192, 208, 224, 256};
int pick_bn(int cells) {
    const int nct = (cells + 255) / 256, per = (cells + nct - 1) / nct;
    for (int w : kWidths)
        if (w >= per) return w;
    return 256;
}

// A split tile: its S parts sit in partial slots slot0 .. slot0 + S - 1.
struct GemmFix {
    int col0, row0, slot0, nparts;
};

// Y tile = sum of its parts, added in slot order (deterministic).  blockIdx.y picks the split
// tile; each thread adds four consecutive rows of one column (float4: the tile's rows start at
// a multiple of 128 and Nr is a multiple of 128, so the four rows are in range together).
template <int BN>
__global__ void __launch_bounds__(256) k_gemm_fixup(const GemmFix* __restrict__ fix, const float* __restrict__ P,
                                                    float* __restrict__ Y, int Mrows, int ncols) {
    // launched as a programmatic dependent of the GEMM: scheduled while the GEMM drains, it
    // waits here until the GEMM's partial tiles are complete
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const GemmFix f = fix[blockIdx.y];
    const int q = blockIdx.x * blockDim.x + threadIdx.x;  // float4 index within the tile
    if (q >= BN * kBM / 4) return;
    const int c = (4 * q) / kBM, r = (4 * q) % kBM;
    const int col = f.col0 + c;
    if (col >= ncols) return;
    const float4* p4 = reinterpret_cast<const float4*>(P);
    const size_t per = (size_t)BN * kBM / 4;
    float4 acc = p4[(size_t)f.slot0 * per + q];
    for (int p = 1; p < f.nparts; ++p) {
        const float4 v = p4[(size_t)(f.slot0 + p) * per + q];
        acc.x += v.x;
        acc.y += v.y;
        acc.z += v.z;
        acc.w += v.w;
    }
    *reinterpret_cast<float4*>(Y + (long)col * Mrows + f.row0 + r) = acc;
}

// Work list of one launch shape.  Tiles go in groups of G neighbouring column tiles of one
// row tile (G = 4, 2 or 1, whichever divides the column tiles), deepest sub-blocks first.  With
// T tiles on P SMs, the groups within the first floor(T / P) * P tiles run whole (entire
// waves); each remaining tile is split into S K-ranges, so the last partial wave becomes S
// times as many shorter items (S = 4 for a tail, up to 4 when there are fewer tiles than SMs,
// keeping at least 4 K slices per item).  The G members of a group (and of each of its K
// parts) are consecutive items with the same row tile and K range, so any cluster size that
// divides G can take them together; the items, and so the arithmetic, do not depend on it.
struct GemmPlan {
    std::vector<GemmWork> work;     // cluster order: the group's members consecutive per K part
    std::vector<GemmWork> work_t;   // tile order: each tile's K parts consecutive (cluster size 1)
    std::vector<GemmWork> work_p;   // persistent form: the items of CTA b at cta_off[b] ..
    std::vector<int> cta_off;
    std::vector<GemmFix> fix;
    int slots = 0;
    int group = 1;
};

// The persistent form's item lists: the items, longest first, each to the CTA with the least
// work so far (K slices plus 2 for the item's read-back), ties to the lower CTA; a CTA runs its
// items in the order received.
void assign_persistent(GemmPlan& pl, int P) {
    const int nitems = (int)pl.work_t.size(), np = std::max(1, std::min(P, nitems));
    std::vector<int> order(nitems);
    for (int i = 0; i < nitems; ++i) order[i] = i;
    auto len = [&](int i) { return pl.work_t[i].kt1 - pl.work_t[i].kt0; };
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return len(a) > len(b); });
    std::vector<long> load(np, 0);
    std::vector<std::vector<int>> lists(np);
    for (int i : order) {
        int b = 0;
        for (int c = 1; c < np; ++c)
            if (load[c] < load[b]) b = c;
        lists[b].push_back(i);
        load[b] += len(i) + 2;
    }
    pl.work_p.clear();
    pl.cta_off.assign(1, 0);
    for (int b = 0; b < np; ++b) {
        for (int i : lists[b]) pl.work_p.push_back(pl.work_t[i]);
        pl.cta_off.push_back((int)pl.work_p.size());
    }
}

GemmPlan make_plan(int cells, int bn, const SubLayout& L, int P) {
    GemmPlan pl;
    const int nct = (cells + bn - 1) / bn, cpad = nct * bn;
    const int G = nct % 4 == 0 ? 4 : (nct % 2 == 0 ? 2 : 1);
    pl.group = G;
    const int nrt = L.rows / kBM, T = nct * nrt;
    struct Group {
        int row0, q, kt, cg;
    };
    std::vector<Group> groups;
    for (int rt = 0; rt < nrt; ++rt) {
        const int row0 = rt * kBM;
        int q = 0;
        while (q + 1 < L.count && row0 >= L.roff[q + 1]) ++q;
        for (int cg = 0; cg < nct / G; ++cg) groups.push_back({row0, q, L.np[q] / kBK, cg});
    }
    std::stable_sort(groups.begin(), groups.end(), [](const Group& a, const Group& b) { return a.kt > b.kt; });
    int W, S;
    int ktmin = 1 << 30;
    for (int q = 0; q < L.count; ++q) ktmin = std::min(ktmin, L.np[q] / kBK);
    if (T >= P) {
        // the split of the tail tiles whose items the persistent form's longest-first
        // assignment balances best (largest CTA load in K slices, 2 per item for its read-back)
        W = T / P * P;
        S = 4;
        long best = -1;
        for (int sc = 2; sc <= 4; ++sc) {
            if (ktmin / sc < 4) break;
            std::vector<int> len;
            for (int gi = 0; gi < (int)groups.size(); ++gi)
                for (int m = 0; m < G; ++m) {
                    const int kt = groups[gi].kt;
                    if (gi < W / G) {
                        len.push_back(kt);
                    } else {
                        for (int p = 0; p < sc; ++p) len.push_back(kt * (p + 1) / sc - kt * p / sc);
                    }
                }
            std::sort(len.begin(), len.end(), std::greater<int>());
            std::vector<long> load(std::min<size_t>(P, len.size()), 0);
            for (int l : len) *std::min_element(load.begin(), load.end()) += l + 2;
            const long mx = *std::max_element(load.begin(), load.end());
            if (best < 0 || mx < best) {
                best = mx;
                S = sc;
            }
        }
    } else {
        W = 0;
        S = std::max(1, std::min(4, P / T));
    }
    while (S > 1 && ktmin / S < 4) --S;
    const int Wg = S == 1 ? (int)groups.size() : W / G;  // whole groups
    for (int gi = 0; gi < (int)groups.size(); ++gi) {
        const Group& u = groups[gi];
        if (gi < Wg) {
            for (int m = 0; m < G; ++m) {
                const int col0 = (u.cg * G + m) * bn;
                pl.work.push_back({col0, u.row0, u.q * cpad + col0, 0, u.kt, -1});
                pl.work_t.push_back(pl.work.back());
            }
            continue;
        }
        const int base = pl.slots;  // tile m's parts sit in slots base + m S .. base + m S + S - 1
        for (int p = 0; p < S; ++p)
            for (int m = 0; m < G; ++m) {
                const int col0 = (u.cg * G + m) * bn;
                pl.work.push_back({col0, u.row0, u.q * cpad + col0, u.kt * p / S, u.kt * (p + 1) / S, base + m * S + p});
            }
        for (int m = 0; m < G; ++m)
            for (int p = 0; p < S; ++p) {
                const int col0 = (u.cg * G + m) * bn;
                pl.work_t.push_back({col0, u.row0, u.q * cpad + col0, u.kt * p / S, u.kt * (p + 1) / S, base + m * S + p});
            }
        for (int m = 0; m < G; ++m) pl.fix.push_back({(u.cg * G + m) * bn, u.row0, base + m * S, S});
        pl.slots += G * S;
    }
    assign_persistent(pl, P);
    return pl;
}

// Number of positions where the float arrays a and b differ bitwise (atomic count).
__global__ void k_count_diff(const float* __restrict__ a, const float* __restrict__ b, long n, int* __restrict__ out) {
    int c = 0;
    for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < n; k += (long)gridDim.x * blockDim.x)
        c += __float_as_uint(a[k]) != __float_as_uint(b[k]) ? 1 : 0;
    if (c) atomicAdd(out, c);
}

// The fix-up of the split tiles, launched with programmatic stream serialization behind the GEMM.
template <int BN>
void launch_fixup(int nfix, const GemmFix* fix, float* P, float* Y, int nr, int cells, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((BN * kBM / 4 + 255) / 256, nfix);
    cfg.blockDim = dim3(256);
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    if (cudaLaunchKernelEx(&cfg, k_gemm_fixup<BN>, (const GemmFix*)fix, (const float*)P, Y, nr, cells) != cudaSuccess) {
        cudaGetLastError();  // without the attribute: an ordinary launch
        k_gemm_fixup<BN><<<cfg.gridDim, 256, 0, s>>>(fix, P, Y, nr, cells);
    }
}

// The persistent form over nprog CTAs and, when fix is set, the fix-up of the split tiles.
template <int BN>
cudaError_t launch_gemm_ws(const CUtensorMap& a0, const CUtensorMap& b0, int nr, int cells, int nprog,
                           const GemmWork* work,
                           const int* cta_off, int nfix, const GemmFix* fix, float* Y, float* P, int* err, int probe,
                           cudaStream_t s) {
    static std::once_flag once;
    std::call_once(once, [] {
        cudaFuncSetAttribute(k_dense_gemm_ws<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)GemmCfg<BN>::SMEM);
    });
    k_dense_gemm_ws<BN><<<nprog, 192, GemmCfg<BN>::SMEM, s>>>(a0, b0, nr, cells, work, cta_off, Y, P, err,
                                                              probe);
    if (nfix > 0) launch_fixup<BN>(nfix, fix, P, Y, nr, cells, s);
    return cudaGetLastError();
}

// The GEMM (cluster size cs; cs = 1 an ordinary launch) and, when fix is set, the fix-up of
// the split tiles.  Returns the launch error.
template <int BN>
cudaError_t launch_gemm(const CUtensorMap& a0, const CUtensorMap& b0,
                        int nr, int cells, int nwork, const GemmWork* work, int nfix, const GemmFix* fix, float* Y,
                        float* P, int* err, int probe, int cs, cudaStream_t s) {
    static std::once_flag once;
    std::call_once(once, [] {
        cudaFuncSetAttribute(k_dense_gemm<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)GemmCfg<BN>::SMEM);
    });
    if (cs == 1) {
        k_dense_gemm<BN><<<nwork, 128, GemmCfg<BN>::SMEM, s>>>(a0, b0, nr, cells, work, Y, P, err, probe, 1);
    } else {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(nwork);
        cfg.blockDim = dim3(128);
        cfg.dynamicSmemBytes = GemmCfg<BN>::SMEM;
        cfg.stream = s;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = (unsigned)cs;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        const cudaError_t e =
            cudaLaunchKernelEx(&cfg, k_dense_gemm<BN>, a0, b0, nr, cells, work, Y, P, err, probe, cs);
        if (e != cudaSuccess) return e;
    }
    if (nfix > 0) launch_fixup<BN>(nfix, fix, P, Y, nr, cells, s);
    return cudaGetLastError();
}

}  // namespace

// Sub-blocks of one (tables, parity mode): A_hi / A_lo stacked [L.rows][L.npmax].
struct DenseOp {
    int mode = 0, nv = 0;
    SubLayout L;
    __nv_bfloat16* A = nullptr;  // hi / lo interleaved per 32-column slice, [rows][2 npmax]
    CUtensorMap mA[3];           // boxes of 128, 64 and 32 rows (cluster sizes 1, 2 and 4)
    size_t bytes = 0;
};

// Work list of one launch shape on the device (built once per (cells, BN, Nr)).
struct DevPlan {
    GemmWork* work = nullptr;    // cluster order
    GemmWork* work_t = nullptr;  // tile order (cluster size 1)
    GemmWork* work_p = nullptr;  // persistent form: items by CTA
    int* cta_off = nullptr;
    int nprog = 0;
    GemmFix* fix = nullptr;
    int nwork = 0, nfix = 0, slots = 0;
    int group = 1;  // column tiles per group (the largest cluster the items allow)
    int cs = 0;     // form chosen by the autotuner: cluster size 1, 2, 4, or kPersistent (0: not yet)
};

struct TcOperands {
    std::mutex mu;
    DenseOp op[3];  // by mode
    std::map<long long, DevPlan> plans;
    // cluster size chosen per launch class (rows, tile width, column-tile group): tuned once
    std::map<long long, int> cs_choice;
    // per-call workspace (grow-only), one per stream: callers on different streams (the
    // service's buckets) run concurrently and must not share operands or partial tiles
    std::map<cudaStream_t, Arena> ws;
    int* err_dev = nullptr;   // bounded-wait failure word of the GEMM (sticky until read)
    int* err_host = nullptr;  // pinned copy, valid after the stream's next synchronisation
};

static lbe_status build_dense(Ctx* c, DevTables* t, DenseOp& d, int mode, cudaStream_t s) {
    const int nv = t->nv;
    d.mode = mode;
    d.nv = nv;
    d.L = sub_layout(nv, mode);
    int nbas = 0;  // basis functions: every sub-block's columns
    for (int q = 0; q < d.L.count; ++q) nbas += d.L.n[q];
    const size_t abytes = (size_t)d.L.rows * 2 * d.L.npmax * 2;  // hi and lo
    lbe_status st = dev_alloc(c, (void**)&d.A, abytes);
    if (st != LBE_OK) return st;
    d.bytes = abytes;
    cudaMemsetAsync(d.A, 0, abytes, s);  // padding rows and columns stay zero
    // basis chunks through the double-float fast-spectral operator (delta = 1)
    const long n3 = (long)nv * nv * nv;
    const int nb = (int)std::min<long>(nbas, std::max<long>(1, (256L << 20) / (n3 * 8)));
    int chunk = 1;
    const size_t scr = fsm_cc_scratch_bytes(*t, nb, 8, &chunk);
    void *hb = nullptr, *lp = nullptr, *lo = nullptr, *sc = nullptr, *dl = nullptr;
    const size_t vb = (size_t)nb * n3 * 8;
    st = dev_alloc(c, &hb, vb);
    if (st == LBE_OK) st = dev_alloc(c, &lp, vb);
    if (st == LBE_OK) st = dev_alloc(c, &lo, vb);
    if (st == LBE_OK) st = dev_alloc(c, &sc, scr);
    if (st == LBE_OK) st = dev_alloc(c, &dl, (size_t)nb * 8);
    if (st == LBE_OK) {
        std::vector<double> ones(nb, 1.0);
        cudaMemcpyAsync(dl, ones.data(), nb * 8, cudaMemcpyHostToDevice, s);
        for (int g0 = 0; g0 < nbas && st == LBE_OK; g0 += nb) {
            const int b = std::min(nb, nbas - g0);
            k_basis_sub<<<8 * sm_count(), 256, 0, s>>>((double*)hb, g0, b, nv, mode);
            st = fsm_df_apply(*t, b, (const double*)dl, (const double*)hb, (double*)lp, (double*)lo, sc, chunk, s,
                              mode);
            k_store_sub<<<8 * sm_count(), 256, 0, s>>>((const double*)lp, d.A, g0, b, nv, mode);
            g_launches += 2;
        }
        if (st == LBE_OK) st = cuda_status(c, cudaStreamSynchronize(s), "dense operator build");
    }
    dev_free(c, hb, vb);
    dev_free(c, lp, vb);
    dev_free(c, lo, vb);
    dev_free(c, sc, scr);
    dev_free(c, dl, (size_t)nb * 8);
    if (st != LBE_OK) return st;
    bool maps = true;
    for (int k = 0; k < 3; ++k)
        maps = maps && make_map(&d.mA[k], d.A, d.L.rows, d.L.npmax, kBM >> k);
    if (!maps) {
        c->last_error = "cuTensorMapEncodeTiled unavailable or failed";
        return LBE_INTERNAL;
    }
    return LBE_OK;
}

// The GEMM of a stacked-sub-block operator d: Y ([cells][d.L.rows], FP32, in T's workspace
// for stream s) = the sub-blocks times the cell operand, which `fill(x2, cpad)` writes into the
// hi / lo interleaved buffer [d.L.count][cpad][2 npmax] (rows cells .. cpad are zeroed here).
// The work plans, the workspace and the form chosen by the autotuner are kept in T; with timed,
// ev[0] / ev[1] bracket the launch.
static lbe_status tc_gemm(Ctx* c, TcOperands& T, DenseOp& d, Tuning* tuning, int cells, cudaStream_t s, bool timed,
                          cudaEvent_t* ev, const std::function<void(__nv_bfloat162*, int)>& fill, float** Yout) {
    lbe_status st;
    if (!T.err_dev) {
        if ((st = dev_alloc(c, (void**)&T.err_dev, 256)) != LBE_OK) return st;
        if (cudaMallocHost((void**)&T.err_host, sizeof(int)) != cudaSuccess) {
            c->last_error = "pinned host word for the tensor-core operator";
            return LBE_OOM;
        }
        *T.err_host = 0;
        cudaMemsetAsync(T.err_dev, 0, sizeof(int), s);
    }
    const int nsub = d.L.count, npmax = d.L.npmax;
    const int mrows = d.L.rows;  // rows of the stacked sub-blocks (and of Y per cell)
    const int bn = pick_bn(cells);
    const long cpad = (cells + bn - 1) / bn * bn;  // whole TMA boxes, zero padding rows
    const long long pkey = ((long long)cells << 32) | ((long long)bn << 20) | mrows;
    auto pit = T.plans.find(pkey);
    if (pit == T.plans.end()) {
        const GemmPlan pl = make_plan(cells, bn, d.L, sm_count());
        DevPlan dp;
        dp.nwork = (int)pl.work.size();
        dp.nfix = (int)pl.fix.size();
        dp.slots = pl.slots;
        dp.group = pl.group;
        if ((st = dev_alloc(c, (void**)&dp.work, pl.work.size() * sizeof(GemmWork))) != LBE_OK) return st;
        if ((st = dev_alloc(c, (void**)&dp.work_t, pl.work_t.size() * sizeof(GemmWork))) != LBE_OK) return st;
        cudaMemcpyAsync(dp.work_t, pl.work_t.data(), pl.work_t.size() * sizeof(GemmWork), cudaMemcpyHostToDevice, s);
        if (dp.nfix && (st = dev_alloc(c, (void**)&dp.fix, pl.fix.size() * sizeof(GemmFix))) != LBE_OK) return st;
        cudaMemcpyAsync(dp.work, pl.work.data(), pl.work.size() * sizeof(GemmWork), cudaMemcpyHostToDevice, s);
        if (dp.nfix) cudaMemcpyAsync(dp.fix, pl.fix.data(), pl.fix.size() * sizeof(GemmFix), cudaMemcpyHostToDevice, s);
        dp.nprog = (int)pl.cta_off.size() - 1;
        if ((st = dev_alloc(c, (void**)&dp.work_p, pl.work_p.size() * sizeof(GemmWork))) != LBE_OK) return st;
        if ((st = dev_alloc(c, (void**)&dp.cta_off, pl.cta_off.size() * sizeof(int))) != LBE_OK) return st;
        cudaMemcpyAsync(dp.work_p, pl.work_p.data(), pl.work_p.size() * sizeof(GemmWork), cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(dp.cta_off, pl.cta_off.data(), pl.cta_off.size() * sizeof(int), cudaMemcpyHostToDevice, s);
        cudaStreamSynchronize(s);  // the host vectors go out of scope
        pit = T.plans.emplace(pkey, dp).first;
    }
    DevPlan& plan = pit->second;
    const size_t xb = (size_t)nsub * cpad * npmax * 2, yb = (size_t)cells * mrows * 4;
    const size_t pb = (size_t)plan.slots * bn * kBM * 4;
    Arena& ws = T.ws[s];
    if ((st = arena_reserve(c, ws, 2 * xb + yb + pb + 4 * 256)) != LBE_OK) return st;
    auto* xhl = (__nv_bfloat16*)arena_take(ws, 2 * xb);  // hi / lo interleaved per slice
    auto* Y = (float*)arena_take(ws, yb);
    auto* Pp = pb ? (float*)arena_take(ws, pb) : nullptr;
    if (cpad > cells)
        for (int q = 0; q < nsub; ++q) {
            const size_t o = ((size_t)q * cpad + cells) * 2 * npmax, n = (size_t)(cpad - cells) * 2 * npmax * 2;
            cudaMemsetAsync(xhl + o, 0, n, s);
        }
    CUtensorMap mX;
    if (!make_map(&mX, xhl, nsub * cpad, npmax, bn)) {
        c->last_error = "cuTensorMapEncodeTiled failed for the cell operand";
        return LBE_INTERNAL;
    }
    fill(reinterpret_cast<__nv_bfloat162*>(xhl), (int)cpad);
    const int probe = g_expire_waits.load();
    auto gemm = [&](int cs, bool with_fix) -> cudaError_t {
        const int k = cs == 4 ? 2 : (cs == 2 ? 1 : 0);
        const int nf = with_fix ? plan.nfix : 0;
        if (cs == kPersistent) switch (bn) {
#define LBE_WS(W)                                                                                                 \
    case W:                                                                                                       \
        return launch_gemm_ws<W>(d.mA[0], mX, mrows, cells, plan.nprog, plan.work_p, plan.cta_off, \
                                 nf, plan.fix, Y, Pp, T.err_dev, probe, s);
                LBE_WS(64)
                LBE_WS(128)
                LBE_WS(160)
                LBE_WS(192)
                LBE_WS(208)
                LBE_WS(224)
                default: LBE_WS(256)
#undef LBE_WS
            }
        switch (bn) {
            case 64: return launch_gemm<64>(d.mA[k], mX, mrows, cells, plan.nwork, cs == 1 ? plan.work_t : plan.work, nf, plan.fix, Y, Pp, T.err_dev, probe, cs, s);
            case 128: return launch_gemm<128>(d.mA[k], mX, mrows, cells, plan.nwork, cs == 1 ? plan.work_t : plan.work, nf, plan.fix, Y, Pp, T.err_dev, probe, cs, s);
            case 160: return launch_gemm<160>(d.mA[k], mX, mrows, cells, plan.nwork, cs == 1 ? plan.work_t : plan.work, nf, plan.fix, Y, Pp, T.err_dev, probe, cs, s);
            case 192: return launch_gemm<192>(d.mA[k], mX, mrows, cells, plan.nwork, cs == 1 ? plan.work_t : plan.work, nf, plan.fix, Y, Pp, T.err_dev, probe, cs, s);
            case 208: return launch_gemm<208>(d.mA[k], mX, mrows, cells, plan.nwork, cs == 1 ? plan.work_t : plan.work, nf, plan.fix, Y, Pp, T.err_dev, probe, cs, s);
            case 224: return launch_gemm<224>(d.mA[k], mX, mrows, cells, plan.nwork, cs == 1 ? plan.work_t : plan.work, nf, plan.fix, Y, Pp, T.err_dev, probe, cs, s);
            default: return launch_gemm<256>(d.mA[k], mX, mrows, cells, plan.nwork, cs == 1 ? plan.work_t : plan.work, nf, plan.fix, Y, Pp, T.err_dev, probe, cs, s);
        }
    };
    const long long cs_key = ((long long)mrows << 20) | ((long long)bn << 8) | plan.group;
    if (plan.cs == 0) {
        auto it = T.cs_choice.find(cs_key);
        if (it != T.cs_choice.end()) plan.cs = it->second;
    }
    if (plan.cs == 0) {
        // LBE_GEMM_FORM fixes the form instead of timing them (for profilers, whose own overhead
        // distorts the timing): "persistent", or a cluster size 1, 2 or 4 the work list allows
        static const char* forced = std::getenv("LBE_GEMM_FORM");
        if (forced) {
            const std::string f(forced);
            int want = f == "persistent" ? kPersistent : (f == "1" || f == "2" || f == "4" ? std::stoi(f) : 0);
            if (want > 1 && want != kPersistent && plan.group % want != 0) want = 0;
            if (want) plan.cs = want;
        }
    }
    if (plan.cs == 0) {
        // autotuner: each cluster size the work list allows, twice in turn (every one computes
        // the same Y); a size that cannot launch is skipped
        cudaStreamCaptureStatus cs_ = cudaStreamCaptureStatusNone;
        const bool capturing = cudaStreamIsCapturing(s, &cs_) != cudaSuccess || cs_ != cudaStreamCaptureStatusNone;
        std::vector<int> cand{1, kPersistent};
        for (int c : {2, 4})
            if (plan.group % c == 0) cand.push_back(c);
        if (capturing || probe) {
            // no timing inside a graph capture (or under the test hook): the persistent form,
            // the fastest on every shape measured, whose items are those of every other form
        } else {
            // every candidate runs with the fix-up and must reproduce the cluster-1 result bit
            // for bit (they share the work list); one that does not is never chosen
            // work overlapping on the context's side stream would distort the timings
            if (c->side_stream && c->side_stream != s) cudaStreamSynchronize(c->side_stream);
            std::vector<float> best(cand.size(), 1e30f);
            float* yref = nullptr;
            int* ndiff = nullptr;
            const size_t ny = (size_t)cells * mrows;
            const bool verify = dev_alloc(c, (void**)&yref, ny * 4) == LBE_OK &&
                                dev_alloc(c, (void**)&ndiff, 256) == LBE_OK;
            cudaEvent_t e0, e1;
            cudaEventCreate(&e0);
            cudaEventCreate(&e1);
            for (int rep = 0; rep < 2; ++rep)
                for (size_t i = 0; i < cand.size(); ++i) {
                    if (best[i] >= 2e30f) continue;
                    cudaEventRecord(e0, s);
                    if (gemm(cand[i], true) != cudaSuccess) {
                        cudaGetLastError();
                        best[i] = 3e30f;
                        continue;
                    }
                    cudaEventRecord(e1, s);
                    cudaEventSynchronize(e1);
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, e0, e1);
                    int werr = 0;  // a bounded wait expired: drop the candidate, clear the word
                    cudaMemcpy(&werr, T.err_dev, sizeof(int), cudaMemcpyDeviceToHost);
                    if (werr) {
                        cudaMemset(T.err_dev, 0, sizeof(int));
                        best[i] = 5e30f;
                        continue;
                    }
                    if (verify && rep == 0) {
                        if (i == 0) {
                            cudaMemcpyAsync(yref, Y, ny * 4, cudaMemcpyDeviceToDevice, s);
                        } else {
                            int nd = 0;
                            cudaMemsetAsync(ndiff, 0, sizeof(int), s);
                            k_count_diff<<<4 * sm_count(), 256, 0, s>>>(yref, Y, (long)ny, ndiff);
                            cudaMemcpyAsync(&nd, ndiff, sizeof(int), cudaMemcpyDeviceToHost, s);
                            cudaStreamSynchronize(s);
                            if (nd != 0) {
                                best[i] = 4e30f;
                                continue;
                            }
                        }
                    }
                    best[i] = std::min(best[i], ms);
                }
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            if (yref) dev_free(c, yref, ny * 4);
            if (ndiff) dev_free(c, ndiff, 256);
            size_t bi = 0;
            for (size_t i = 1; i < cand.size(); ++i)
                if (best[i] < best[bi]) bi = i;
            plan.cs = cand[bi];
            T.cs_choice[cs_key] = plan.cs;
            if (tuning) {
                char line[256];
                auto name = [](int c, char* b, size_t n) {
                    if (c == kPersistent)
                        snprintf(b, n, "persistent");
                    else
                        snprintf(b, n, "cluster %d", c);
                };
                char nm[32];
                name(plan.cs, nm, sizeof nm);
                int n = snprintf(line, sizeof line, "dense_gemm<%d> cells=%d rows=%d: %s (", bn, cells, mrows, nm);
                for (size_t i = 0; i < cand.size() && n < (int)sizeof line; ++i) {
                    name(cand[i], nm, sizeof nm);
                    n += best[i] < 1e29f ? snprintf(line + n, sizeof line - n, "%s%s %.1f us", i ? ", " : "", nm,
                                                    1000.0f * best[i])
                                         : snprintf(line + n, sizeof line - n, "%s%s %s", i ? ", " : "", nm,
                                                    best[i] >= 5e30f   ? "wait expired"
                                                    : best[i] >= 4e30f ? "differed"
                                                                       : "did not launch");
                }
                if (n < (int)sizeof line) snprintf(line + n, sizeof line - n, ")");
                std::lock_guard<std::mutex> lk2(tuning->mu);
                tuning->log.push_back(line);
            }
        }
    }
    {
        if (timed) cudaEventRecord(ev[0], s);
        const cudaError_t ge = gemm(plan.cs > 0 ? plan.cs : kPersistent, true);
        if (ge != cudaSuccess) return cuda_status(c, ge, "dense operator GEMM launch");
    }
    if (timed) cudaEventRecord(ev[1], s);
    *Yout = Y;
    return LBE_OK;
}

// L+ h and L h on the parity subspace with the dense tensor-core operator (float in / out).
// sync = false leaves the stream running: the GEMM's failure word is copied to pinned host
// memory behind it and tc_check reads it after the caller's own synchronisation.
lbe_status tc_apply_sym(Ctx* c, DevTables* t, int mode, int cells, const double* delta, const float* h, float* Lplus,
                        float* Lout, cudaStream_t s, bool sync, const double* nd, double* G, const double* hm,
                        bool quarter) {
    if (mode != 1 && mode != 2) return LBE_BAD_ARG;
    if (quarter && G && (!hm || Lout)) return LBE_BAD_ARG;
    if (cells <= 0) return LBE_OK;
    if (!t->tc) t->tc = new TcOperands();
    TcOperands& T = *t->tc;
    std::lock_guard<std::mutex> lk(T.mu);
    DenseOp& d = T.op[mode];
    lbe_status st;
    if (!d.A && (st = build_dense(c, t, d, mode, s)) != LBE_OK) return st;
    // optional event timing of the GEMM alone (public synchronous calls only)
    cudaEvent_t ev[2] = {nullptr, nullptr};
    const bool timed = sync && g_time_kernels.load() != 0 && cudaEventCreate(&ev[0]) == cudaSuccess &&
                       cudaEventCreate(&ev[1]) == cudaSuccess;
    float* Y = nullptr;
    const int nv = t->nv;
    st = tc_gemm(c, T, d, t->tuning, cells, s, timed, ev, [&](__nv_bfloat162* x2, int cp) {
    {
        const bool p2 = mode == 2;
        const int qf = quarter ? 1 : 0;
        switch (nv) {
            case 8: (p2 ? launch_gather<8, 2> : launch_gather<8, 1>)(cells, cp, h, x2, s, qf); break;
            case 16: (p2 ? launch_gather<16, 2> : launch_gather<16, 1>)(cells, cp, h, x2, s, qf); break;
            case 24: (p2 ? launch_gather<24, 2> : launch_gather<24, 1>)(cells, cp, h, x2, s, qf); break;
            default: (p2 ? launch_gather<32, 2> : launch_gather<32, 1>)(cells, cp, h, x2, s, qf); break;
        }
    }
    }, &Y);
    if (st != LBE_OK) {
        if (ev[0]) cudaEventDestroy(ev[0]);
        if (ev[1]) cudaEventDestroy(ev[1]);
        return st;
    }
    {  // L+ h (L h when asked for) and, with G, the SIS L-moments in one pass
        const float* nu1 = t->nu1_f;
        const float* vel = t->vel_f;
        const double dv3 = t->dv * t->dv * t->dv;
        const bool p2 = mode == 2;
        if (quarter && !p2) switch (nv) {
                case 8: launch_expand_h<8>(cells, Y, vel, delta, Lplus, G, dv3, hm, h, nu1, Lout, s); break;
                case 16: launch_expand_h<16>(cells, Y, vel, delta, Lplus, G, dv3, hm, h, nu1, Lout, s); break;
                case 24: launch_expand_h<24>(cells, Y, vel, delta, Lplus, G, dv3, hm, h, nu1, Lout, s); break;
                default: launch_expand_h<32>(cells, Y, vel, delta, Lplus, G, dv3, hm, h, nu1, Lout, s); break;
            }
        else if (quarter) switch (nv) {
                case 8: launch_expand_q<8>(cells, Y, vel, delta, Lplus, G, dv3, hm, h, nu1, Lout, s); break;
                case 16: launch_expand_q<16>(cells, Y, vel, delta, Lplus, G, dv3, hm, h, nu1, Lout, s); break;
                case 24: launch_expand_q<24>(cells, Y, vel, delta, Lplus, G, dv3, hm, h, nu1, Lout, s); break;
                default: launch_expand_q<32>(cells, Y, vel, delta, Lplus, G, dv3, hm, h, nu1, Lout, s); break;
            }
        else switch (nv) {
            case 8: (p2 ? launch_expand<8, 2> : launch_expand<8, 1>)(cells, Y, h, nu1, vel, delta, nd, Lplus, Lout, G, dv3, hm, s); break;
            case 16: (p2 ? launch_expand<16, 2> : launch_expand<16, 1>)(cells, Y, h, nu1, vel, delta, nd, Lplus, Lout, G, dv3, hm, s); break;
            case 24: (p2 ? launch_expand<24, 2> : launch_expand<24, 1>)(cells, Y, h, nu1, vel, delta, nd, Lplus, Lout, G, dv3, hm, s); break;
            default: (p2 ? launch_expand<32, 2> : launch_expand<32, 1>)(cells, Y, h, nu1, vel, delta, nd, Lplus, Lout, G, dv3, hm, s); break;
        }
    }
    g_launches += 3;
    g_levals += cells;
    cudaMemcpyAsync(T.err_host, T.err_dev, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (!sync) return cuda_status(c, cudaGetLastError(), "dense operator launch");
    st = cuda_status(c, cudaStreamSynchronize(s), "dense operator");
    if (ev[0]) {
        float ms = 0.f;
        if (timed && st == LBE_OK && cudaEventElapsedTime(&ms, ev[0], ev[1]) == cudaSuccess) add_gemm_time(ms);
        cudaEventDestroy(ev[0]);
        if (ev[1]) cudaEventDestroy(ev[1]);
    }
    return st != LBE_OK ? st : tc_check(c, t);
}

// Reads (and clears) the GEMM's failure word; valid once the stream has been synchronised.
lbe_status tc_check(Ctx* c, DevTables* t) {
    if (!t->tc || !t->tc->err_host || !*t->tc->err_host) return LBE_OK;
    *t->tc->err_host = 0;
    cudaMemset(t->tc->err_dev, 0, sizeof(int));
    c->last_error = "tensor-core operator: a bounded wait expired";
    return LBE_TIMEOUT;
}

// Frees the plans, workspaces and failure words of T (not its operators).
static void release_operands(Ctx* c, TcOperands& T) {
    for (auto& kv : T.ws) arena_release(c, kv.second);
    for (auto& kv : T.plans) {
        dev_free(c, kv.second.work, kv.second.nwork * sizeof(GemmWork));
        dev_free(c, kv.second.work_t, kv.second.nwork * sizeof(GemmWork));
        if (kv.second.fix) dev_free(c, kv.second.fix, kv.second.nfix * sizeof(GemmFix));
        dev_free(c, kv.second.work_p, kv.second.nwork * sizeof(GemmWork));
        dev_free(c, kv.second.cta_off, (kv.second.nprog + 1) * sizeof(int));
    }
    dev_free(c, T.err_dev, 256);
    if (T.err_host) cudaFreeHost(T.err_host);
    T.err_dev = nullptr;
    T.err_host = nullptr;
}

void tc_release(Ctx* c, DevTables* t) {
    if (!t->tc) return;
    for (auto& d : t->tc->op) {
        dev_free(c, d.A, d.bytes);
    }
    release_operands(c, *t->tc);
    delete t->tc;
    t->tc = nullptr;
}

// ---- the binary-mixture operator on the tensor cores (mixture.cu) ----------------------------
// The dense FP64 mixture matrix ([n][n] row-major, n = both species' unknowns per cell) as one
// sub-block of n rows and columns, padded to the 128-row tile, in BF16 hi / lo; the cell
// operand is both species' h of a cell, hi / lo, padded with zeros.
struct MixTc {
    TcOperands T;
    DenseOp d;
};

namespace {

__global__ void k_mix_store_bf16(const double* __restrict__ L, int n, int np, __nv_bfloat16* __restrict__ A) {
    const long total = (long)n * n;
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
        const long r = t / n, col = t - r * n;
        const double a = L[t];
        const __nv_bfloat16 hi = __float2bfloat16_rn((float)a);
        const long idx = r * 2 * np + ilv(col);
        A[idx] = hi;
        A[idx + kBK] = __float2bfloat16_rn((float)(a - (double)__bfloat162float(hi)));
    }
}

// x2: [cells][np] columns as hi / lo pairs (k even): column k < nr is h_A[c cs + k], nr <= k < 2 nr
// is h_B[c cs + k - nr], the rest zero; c = map[n] for GEMM column n when a cell list is given
__global__ void k_mix_gather(const double* __restrict__ hA, const double* __restrict__ hB, long cs, int nr, int np,
                             int cells, __nv_bfloat162* __restrict__ x2, const int* __restrict__ map) {
    const int half = np / 2;
    const long total = (long)cells * half;
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
        const long c = t / half, src = map ? map[c] : c;
        const int k = 2 * (int)(t - c * half);
        double v[2];
        for (int u = 0; u < 2; ++u) {
            const int kk = k + u;
            v[u] = kk < nr ? hA[src * cs + kk] : (kk < 2 * nr ? hB[src * cs + kk - nr] : 0.0);
        }
        const __nv_bfloat16 h0 = __float2bfloat16_rn((float)v[0]), h1 = __float2bfloat16_rn((float)v[1]);
        const __nv_bfloat16 l0 = __float2bfloat16_rn((float)(v[0] - (double)__bfloat162float(h0)));
        const __nv_bfloat16 l1 = __float2bfloat16_rn((float)(v[1] - (double)__bfloat162float(h1)));
        const long o = (c * 2 * np + ilv(k)) / 2;
        x2[o] = __halves2bfloat162(h0, h1);
        x2[o + kBK / 2] = __halves2bfloat162(l0, l1);
    }
}

// y_a[c cs + j] = scale Y[n mrows + a nr + j], c = n or map[n]
template <typename T>
__global__ void k_mix_readback(const float* __restrict__ Y, int mrows, int nr, int cells, long cs, double scale,
                               T* __restrict__ yA, T* __restrict__ yB, const int* __restrict__ map) {
    const long total = (long)cells * 2 * nr;
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
        const long c = t / (2 * nr), dst = map ? map[c] : c;
        const int r = (int)(t - c * 2 * nr);
        (r < nr ? yA : yB)[dst * cs + (r < nr ? r : r - nr)] = (T)(scale * (double)Y[c * mrows + r]);
    }
}

}  // namespace

lbe_status mix_tc_build(Ctx* c, const double* L, int n, MixTc** out, cudaStream_t s) {
    MixTc* m = new MixTc();
    DenseOp& d = m->d;
    d.mode = 0;
    d.L.count = 1;
    d.L.kind[0] = 0;
    d.L.n[0] = n;
    d.L.np[0] = pad128(n);
    d.L.rows = d.L.np[0];
    d.L.npmax = d.L.np[0];
    const size_t abytes = (size_t)d.L.rows * 2 * d.L.npmax * 2;
    lbe_status st = dev_alloc(c, (void**)&d.A, abytes);
    if (st != LBE_OK) {
        delete m;
        return st;
    }
    d.bytes = abytes;
    cudaMemsetAsync(d.A, 0, abytes, s);
    k_mix_store_bf16<<<8 * sm_count(), 256, 0, s>>>(L, n, d.L.npmax, d.A);
    g_launches += 1;
    st = cuda_status(c, cudaStreamSynchronize(s), "mixture tensor-core operator");
    bool maps = st == LBE_OK;
    for (int k = 0; k < 3 && maps; ++k) maps = make_map(&d.mA[k], d.A, d.L.rows, d.L.npmax, kBM >> k);
    if (st == LBE_OK && !maps) {
        c->last_error = "cuTensorMapEncodeTiled unavailable or failed";
        st = LBE_INTERNAL;
    }
    if (st != LBE_OK) {
        mix_tc_release(c, m);
        return st;
    }
    *out = m;
    return LBE_OK;
}

lbe_status mix_tc_apply(Ctx* c, MixTc* m, int cells, const double* hA, const double* hB, long cs, int nr,
                        double scale, void* yA, void* yB, bool f32, cudaStream_t s, const int* map) {
    std::lock_guard<std::mutex> lk(m->T.mu);
    float* Y = nullptr;
    const int np = m->d.L.npmax;
    // with kernel timing on, the GEMM is bracketed by events and waited for (lbe_get_stats)
    cudaEvent_t ev[2] = {nullptr, nullptr};
    const bool timed = g_time_kernels.load() != 0 && cudaEventCreate(&ev[0]) == cudaSuccess &&
                       cudaEventCreate(&ev[1]) == cudaSuccess;
    lbe_status st = tc_gemm(c, m->T, m->d, nullptr, cells, s, timed, ev, [&](__nv_bfloat162* x2, int) {
        const long tot = (long)cells * (np / 2);
        k_mix_gather<<<(int)std::min<long>((tot + 255) / 256, 32L * sm_count()), 256, 0, s>>>(hA, hB, cs, nr, np,
                                                                                              cells, x2, map);
    }, &Y);
    if (ev[0]) {
        float ms = 0.f;
        if (timed && st == LBE_OK && cudaEventSynchronize(ev[1]) == cudaSuccess &&
            cudaEventElapsedTime(&ms, ev[0], ev[1]) == cudaSuccess)
            add_gemm_time(ms);
        cudaEventDestroy(ev[0]);
        if (ev[1]) cudaEventDestroy(ev[1]);
    }
    if (st != LBE_OK) return st;
    const long tot = (long)cells * 2 * nr;
    const int gr = (int)std::min<long>((tot + 255) / 256, 32L * sm_count());
    if (f32)
        k_mix_readback<float><<<gr, 256, 0, s>>>(Y, m->d.L.rows, nr, cells, cs, scale, (float*)yA, (float*)yB, map);
    else
        k_mix_readback<double><<<gr, 256, 0, s>>>(Y, m->d.L.rows, nr, cells, cs, scale, (double*)yA, (double*)yB,
                                                  map);
    g_launches += 3;
    cudaMemcpyAsync(m->T.err_host, m->T.err_dev, sizeof(int), cudaMemcpyDeviceToHost, s);
    return cuda_status(c, cudaGetLastError(), "mixture tensor-core operator");
}

lbe_status mix_tc_check(Ctx* c, MixTc* m) {
    if (!m->T.err_host || !*m->T.err_host) return LBE_OK;
    *m->T.err_host = 0;
    cudaMemset(m->T.err_dev, 0, sizeof(int));
    c->last_error = "mixture tensor-core operator: a bounded wait expired";
    return LBE_TIMEOUT;
}

void mix_tc_release(Ctx* c, MixTc* m) {
    if (!m) return;
    dev_free(c, m->d.A, m->d.bytes);
    release_operands(c, m->T);
    delete m;
}

}  // namespace lbe

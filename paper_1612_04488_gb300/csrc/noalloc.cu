// lbe_apply_L_noalloc: the collision operator (the same CUDA-core kernels as lbe_apply_L)
// for callers that must not allocate device memory.
//
// Who needs it: code that records CUDA graphs or runs inside a latency-critical loop, where
// a cudaMalloc / cudaFree would synchronise the device or be illegal in the middle of a
// captured region, and host frameworks whose own pooling allocator owns every device byte
// and forbids a library from allocating behind its back.  Such callers pass inputs and
// outputs they already own; the transform scratch comes from one file-scope device array
// of fixed size instead of the context's workspace.
//
// Limits and contract:
//   - The scratch array holds kNoAllocScratchBytes (32 MiB) on every device where this
//     library's module is loaded, for the life of the process.
//   - Cells are processed in slices that fit the array; a request whose single cell does
//     not fit (e.g. nv = 32, M = 64 in FP64) is rejected with LBE_BAD_ARG.
//   - The operator tables must already exist in the context (an earlier lbe_apply_L or
//     lbe_solve with the same nv, vmax, M, R built them); this entry point never builds
//     them, because building allocates.
//   - The first call on a device looks up the array's device address with that device
//     current (cudaGetSymbolAddress) and caches it; make that first call before any
//     stream capture.
//   - All calls share the one array: calls whose launches overlap on the GPU race.  Every
//     scratch element is written before it is read, so nothing has to start at zero.
#include <cstdio>
#include <mutex>
#include <string>

#include "lbe_internal.h"
#include "sweep.h"

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_setup_mu;
void* g_scratch_addr[kMaxDevices] = {};

}  // namespace

using namespace lbe;

extern "C" lbe_status lbe_apply_L_noalloc(lbe_ctx* ctx, int nv, double vmax, int M, double R,
                                          lbe_precision precision, int cells, const double* delta_dev,
                                          const void* h_dev, void* Lplus_dev, void* L_dev, void* stream) {
    Ctx* c = ctx;
    if (!c) return LBE_BAD_ARG;
    if (cells < 0 || (cells > 0 && (!h_dev || !delta_dev))) return bad_arg(c, "null h or delta");
    if (nv != 8 && nv != 16 && nv != 24 && nv != 32) return bad_arg(c, "nv must be 8, 16, 24 or 32");
    if (M < 2 || M > 64 || (M & (M - 1))) return bad_arg(c, "M must be a power of two in [2, 64]");
    if (!(vmax > 0) || R > 2 * vmax) return bad_arg(c, "bad vmax or R");
    if (precision != LBE_FP64 && precision != LBE_FP32)
        return bad_arg(c, "lbe_apply_L_noalloc takes LBE_FP64 or LBE_FP32");
    if (c->device < 0 || c->device >= kMaxDevices) return bad_arg(c, "device index out of range");
    const size_t eb = precision == LBE_FP64 ? 8 : 4;
    const size_t n3 = (size_t)nv * nv * nv;
    const size_t per_cell = n3 * 2 * eb * (size_t)(M + 2);  // H + Y (M + 1 transforms) of one cell
    if (per_cell > kNoAllocScratchBytes) {
        char msg[256];
        snprintf(msg, sizeof msg,
                 "one cell needs %zu bytes of transform scratch, more than the %zu-byte no-alloc maximum",
                 per_cell, kNoAllocScratchBytes);
        return bad_arg(c, msg);
    }
    if (cells == 0) return LBE_OK;
    if (R <= 0) R = default_R(vmax);
    DevTables* t = nullptr;
    {
        std::lock_guard<std::mutex> lk(c->tables_mu);
        auto it = c->tables.find(tables_key(nv, vmax, M, R));
        if (it != c->tables.end()) t = it->second.get();
    }
    if (!t)
        return bad_arg(c, "operator tables for these (nv, vmax, M, R) are not built in this context; "
                          "call lbe_apply_L or lbe_solve with them once first");
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return cuda_status(c, e, "cudaSetDevice");
    void* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_setup_mu);
        if (!g_scratch_addr[c->device]) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess) return cuda_status(c, e, "cudaGetSymbolAddress(no-alloc scratch)");
            g_scratch_addr[c->device] = p;
        }
        scratch = g_scratch_addr[c->device];
    }
    int slice = (int)(kNoAllocScratchBytes / per_cell);
    if (slice > 64) slice = 64;  // the transform chunk of fsm_cc_apply
    cudaStream_t s = (cudaStream_t)stream;
    for (int c0 = 0; c0 < cells; c0 += slice) {
        const int k = cells - c0 < slice ? cells - c0 : slice;
        lbe_status st;
        if (precision == LBE_FP64) {
            st = fsm_cc_apply<double>(*t, k, delta_dev + c0, (const double*)h_dev + c0 * n3,
                                      Lplus_dev ? (double*)Lplus_dev + c0 * n3 : nullptr,
                                      L_dev ? (double*)L_dev + c0 * n3 : nullptr, scratch, k, s);
        } else {
            st = fsm_cc_apply<float>(*t, k, delta_dev + c0, (const float*)h_dev + c0 * n3,
                                     Lplus_dev ? (float*)Lplus_dev + c0 * n3 : nullptr,
                                     L_dev ? (float*)L_dev + c0 * n3 : nullptr, scratch, k, s);
        }
        if (st != LBE_OK) return st;
    }
    return cuda_status(c, cudaGetLastError(), "apply_L_noalloc");
}

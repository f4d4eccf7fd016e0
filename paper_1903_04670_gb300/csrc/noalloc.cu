// dgfs_collide_noalloc: the FP64 collision operator evaluated without any
// device allocation.
//
// Who needs it: callers that are not allowed to allocate device memory when
// they evaluate the operator, for example code that runs under a host
// framework which owns the whole device-memory budget and forbids its plugins
// to call cudaMalloc, or latency-critical loops where an allocation (which may
// synchronise the device) is not acceptable.  The plan's tables still come
// from dgfs_plan_create, which such callers run once at start-up; this entry
// point then takes its scratch memory from a fixed array that is part of the
// loaded library instead of the plan's workspace.
//
// The scratch array below is a file-scope __device__ array: every GPU that
// loads this library holds its kNoAllocScratchBytes until the process exits.
// Host code cannot use the array's name as a device address, so the device
// address is looked up with cudaGetSymbolAddress once per device, with that
// device current, on the first call made on that device.  The address belongs
// to the device's context: after cudaDeviceReset the library's module is
// loaded again in a new context and the array may sit elsewhere, so the
// cached address is keyed on the context's unique id and looked up again when
// the current context is a different one.
#include <cuda.h>  // driver types only; the entry points are resolved through the runtime

#include <cstdio>
#include <mutex>

#include "dgfs_internal.h"

namespace dgfs {
namespace {

constexpr size_t kNoAllocScratchBytes = 32u << 20;  // 32 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_setup_mutex;
void *g_scratch_addr[kMaxDevices] = {nullptr};
unsigned long long g_scratch_ctx[kMaxDevices] = {0};  // context id the address belongs to

typedef CUresult (*CtxGetCurrentFn)(CUcontext *);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long *);

// Unique id of the calling thread's current context (never reused within a
// process), or 0 when the driver cannot report it.  Caller holds the mutex.
unsigned long long current_context_id()
{
    static bool resolved = false;
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    if (!resolved) {
        resolved = true;
        cudaDriverEntryPointQueryResult q1 = cudaDriverEntryPointSymbolNotFound, q2 = q1;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", reinterpret_cast<void **>(&get_current), 12000,
                                             cudaEnableDefault, &q1) != cudaSuccess ||
            q1 != cudaDriverEntryPointSuccess)
            get_current = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", reinterpret_cast<void **>(&get_id), 12000,
                                             cudaEnableDefault, &q2) != cudaSuccess ||
            q2 != cudaDriverEntryPointSuccess)
            get_id = nullptr;
    }
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (get_current && get_id && get_current(&ctx) == CUDA_SUCCESS && ctx && get_id(ctx, &id) == CUDA_SUCCESS)
        return id;
    return 0;
}

// Device address of the scratch array on `device` (which must be current).
dgfs_status scratch_address(int device, void **out)
{
    if (device < 0 || device >= kMaxDevices) {
        set_error("dgfs_collide_noalloc: device ordinal out of range");
        return DGFS_EINVAL;
    }
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    const unsigned long long ctx = current_context_id();
    if (!g_scratch_addr[device] || ctx == 0 || ctx != g_scratch_ctx[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return cuda_status(e, "cudaGetSymbolAddress(noalloc scratch)");
        g_scratch_addr[device] = p;
        g_scratch_ctx[device] = ctx;
    }
    *out = g_scratch_addr[device];
    return DGFS_OK;
}

}  // namespace
}  // namespace dgfs

using namespace dgfs;

extern "C" dgfs_status dgfs_collide_noalloc(dgfs_plan plan, int P, const void *f_dev, void *Q_dev, void *stream)
{
    if (!plan || !f_dev || !Q_dev || P < 1) {
        set_error("dgfs_collide_noalloc: bad plan, pointer or P");
        return DGFS_EINVAL;
    }
    if (plan->prec != DGFS_FP64 || plan->hermitian) {
        set_error("dgfs_collide_noalloc: only DGFS_FP64 plans in the literal form are supported");
        return DGFS_EUNSUPPORTED;
    }
    // largest number of evaluations per pass whose scratch fits the array
    int chunk = 0;
    for (int c = P; c >= 1; --c)
        if (fp64_scratch_bytes(plan, P, c) <= kNoAllocScratchBytes) {
            chunk = c;
            break;
        }
    if (chunk == 0) {
        char msg[256];
        std::snprintf(msg, sizeof(msg),
                      "dgfs_collide_noalloc: P = %d needs %zu bytes of scratch even one evaluation at a time; "
                      "the static scratch holds %zu bytes",
                      P, fp64_scratch_bytes(plan, P, 1), kNoAllocScratchBytes);
        set_error(msg);
        return DGFS_EINVAL;
    }
    dgfs_status st = plan_entry_check(plan);  // makes the plan's device current
    if (st != DGFS_OK) return st;
    void *scratch = nullptr;
    st = scratch_address(plan->device, &scratch);
    if (st != DGFS_OK) return st;
    // Every buffer in the scratch is written before it is read, so nothing is
    // cleared between calls.
    return fp64_collide_ws(plan, P, f_dev, Q_dev, scratch, P, chunk, reinterpret_cast<cudaStream_t>(stream));
}

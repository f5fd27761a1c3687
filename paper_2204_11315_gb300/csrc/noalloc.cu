// noalloc.cu -- oocs_incore_run_noalloc: the in-core run for callers that
// cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: a plugin running inside a host
// application whose allocator owns the whole device memory pool, or a
// latency-critical loop where cudaMalloc / cudaFree would synchronise the
// device.  oocs_incore_run needs one grid-sized scratch field (the ping-pong
// partner of the time steps); this variant takes it from a file-scope static
// device array instead, so the caller passes only inputs and outputs.
//
// The array lives in every GPU that loads this library, until the process
// exits.  Host code must not pass the array's name to a kernel (on the host it
// is only a stand-in for the device symbol); the device address is looked up
// with cudaGetSymbolAddress once per device and context, and passed on.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>

#include "../../include/oocs.h"
#include "capi_internal.h"

namespace {

// library-owned scratch of oocs_incore_run_noalloc (shared by every call)
static __device__ __align__(256) float g_noalloc_scratch[OOCS_NOALLOC_MAX_VALUES];

struct DeviceScratch {
    int device;
    CUcontext ctx;  // the context the address belongs to
    float *ptr;
};

std::mutex g_mu;
DeviceScratch g_known[256];
int g_nknown = 0;

// cuCtxGetCurrent, taken from the driver through the runtime (no link to libcuda)
using CtxGetCurrentFn = CUresult (*)(CUcontext *);

CtxGetCurrentFn ctx_get_current()
{
    static CtxGetCurrentFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        cudaDriverEntryPointQueryResult q;
        void *p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<CtxGetCurrentFn>(p);
    });
    return fn;
}

// Device address of the scratch array in the current device's current
// context; looked up on the first call made in that (device, context) pair,
// then cached.  The context is part of the key because cudaDeviceReset ends
// the primary context: the runtime then loads this module again in a new one,
// where the array may have another address.
oocs_status scratch_on_current_device(float **out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        oocs::set_last_error(std::string("cudaGetDevice: ") + cudaGetErrorString(e));
        return OOCS_ERR_CUDA;
    }
    CtxGetCurrentFn get = ctx_get_current();
    if (!get) {
        oocs::set_last_error("cuCtxGetCurrent is not available from the driver");
        return OOCS_ERR_CUDA;
    }
    CUcontext ctx = nullptr;  // null before the runtime has made the context current
    if (get(&ctx) != CUDA_SUCCESS)
        ctx = nullptr;
    std::lock_guard<std::mutex> lock(g_mu);
    for (int i = 0; i < g_nknown && ctx; ++i)
        if (g_known[i].device == dev && g_known[i].ctx == ctx) {
            *out = g_known[i].ptr;
            return OOCS_OK;
        }
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);  // also makes the primary context current
    if (e != cudaSuccess || !p) {
        oocs::set_last_error(std::string("cudaGetSymbolAddress(no-allocation scratch): ") +
                             cudaGetErrorString(e));
        return OOCS_ERR_CUDA;
    }
    if (get(&ctx) != CUDA_SUCCESS || !ctx) {
        oocs::set_last_error("cuCtxGetCurrent: no current context for the no-allocation scratch");
        return OOCS_ERR_CUDA;
    }
    // a device seen before with another context: replace its entry
    int slot = -1;
    for (int i = 0; i < g_nknown; ++i)
        if (g_known[i].device == dev)
            slot = i;
    if (slot < 0 && g_nknown < 256)
        slot = g_nknown++;
    if (slot >= 0)
        g_known[slot] = {dev, ctx, static_cast<float *>(p)};
    *out = static_cast<float *>(p);
    return OOCS_OK;
}

}  // namespace

extern "C" oocs_status oocs_incore_run_noalloc(const oocs_desc *desc, float *u, float *u_prev,
                                               const float *m, int32_t nsteps, int64_t t0,
                                               const int64_t *src_xyz, const float *w, int32_t nw,
                                               void *stream)
try {
    if (!desc) {
        oocs::set_last_error("desc is NULL");
        return OOCS_ERR_INVALID_ARG;
    }
    const uint64_t cap = OOCS_NOALLOC_MAX_VALUES;
    const bool dims_ok = desc->nx > 0 && desc->ny > 0 && desc->nz > 0 &&
                         (uint64_t)desc->nx <= cap && (uint64_t)desc->ny <= cap / (uint64_t)desc->nx &&
                         (uint64_t)desc->nz <= cap / ((uint64_t)desc->nx * (uint64_t)desc->ny);
    if (!dims_ok) {
        oocs::set_last_error("grid of " + std::to_string(desc->nx) + " x " + std::to_string(desc->ny) +
                             " x " + std::to_string(desc->nz) +
                             " values exceeds the no-allocation scratch of " + std::to_string(cap) +
                             " values (OOCS_NOALLOC_MAX_VALUES)");
        return OOCS_ERR_INVALID_ARG;
    }
    float *scratch = nullptr;
    oocs_status s = scratch_on_current_device(&scratch);
    if (s != OOCS_OK)
        return s;
    return oocs_incore_run(desc, u, u_prev, m, scratch, nsteps, t0, src_xyz, w, nw, stream);
} catch (...) {
    return oocs::exception_status(nullptr);
}

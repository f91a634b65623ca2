// mc_run_static: mc_run for callers that cannot hand the library a device
// workspace (declared in include/mcmie.h).
//
// Some callers cannot call cudaMalloc at the point where they run the walk:
// for example a host application that owns all device memory through its own
// allocator and gives plug-ins only the buffers they read and write, or a
// caller on a latency-critical thread where an allocation may synchronise the
// device. This entry point takes only inputs and outputs; the scratch the
// walk needs (its photon counter) lives in a fixed array in this library's
// device memory instead of a caller workspace.
//
//  * The array is a file-scope static __device__ buffer of
//    MC_STATIC_SCRATCH_BYTES bytes. Every GPU that loads the library holds it
//    until the process exits. A camera whose workspace would not fit is
//    rejected with MC_ERR_NOMEM before anything is launched.
//  * The array's device address is looked up with cudaGetSymbolAddress
//    (with the device current) and cached per device together with the id
//    of the CUDA context it belongs to. A call in another context of that
//    device (after cudaDeviceReset, or when a host tears its context down and
//    builds a new one) finds the id changed and looks the address up again;
//    only such a look-up may load the library's module on the device, so the
//    first call in each context should come before any stream capture.
//  * All calls share the one array, which keeps what the last call left in it.
//    mc_run clears the counter on the stream before every launch, so
//    consecutive calls are independent, but calls whose work overlaps on the
//    GPU (different streams, or different host threads) race on the counter
//    and must be serialised by the caller.
//  * Nothing here calls cudaMalloc, cudaFree or an allocating library routine.
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/mcmie.h"

namespace {

static __device__ __align__(256) unsigned char g_scratch[MC_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_lock;
struct Cached {
    unsigned long long ctx_id;   // id of the context the address belongs to
    void *addr;                  // device address of g_scratch there (null: none yet)
};
Cached g_cache[kMaxDevices] = {};

// The CUDA driver API's context queries, reached through the runtime (no
// link to libcuda): current context and its process-unique id.
typedef CUresult (*CtxGetCurrentFn)(CUcontext *);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long *);

bool context_id(unsigned long long *id)
{
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<CtxGetCurrentFn>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<CtxGetIdFn>(f);
    });
    if (!get_current || !get_id) return false;
    CUcontext ctx = nullptr;
    if (get_current(&ctx) != CUDA_SUCCESS || !ctx) return false;
    return get_id(ctx, id) == CUDA_SUCCESS;
}

// Device address of g_scratch in the current device's current context.
mc_status scratch_address(void **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MC_ERR_CUDA;
    std::lock_guard<std::mutex> guard(g_lock);
    Cached &c = g_cache[dev];
    unsigned long long id = 0;
    if (c.addr && context_id(&id) && c.ctx_id == id) {
        *out = c.addr;
        return MC_OK;
    }
    // first call in this context (the look-up also makes the runtime's
    // context current on this thread if no context is yet)
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return MC_ERR_CUDA;
    if (!context_id(&id)) return MC_ERR_CUDA;
    c.addr = p;
    c.ctx_id = id;
    *out = p;
    return MC_OK;
}

}  // namespace

extern "C" mc_status mc_run_static(const mc_medium *medium, const mc_geometry *geom,
                                   const mc_camera *camera, const mc_run_params *run,
                                   int64_t *d_image, int64_t *d_radial, int64_t *d_totals,
                                   uint32_t *d_error, void *stream)
{
    const size_t need = mc_workspace_bytes(camera);
    if (need == 0) return MC_ERR_ARG;
    if (need > sizeof(g_scratch)) return MC_ERR_NOMEM;
    void *scratch = nullptr;
    mc_status s = scratch_address(&scratch);
    if (s != MC_OK) return s;
    mc_tallies t;
    t.d_image = d_image;
    t.d_radial = d_radial;
    t.d_totals = d_totals;
    t.d_error = d_error;
    t.d_work = scratch;
    t.work_bytes = sizeof(g_scratch);
    return mc_run(medium, geom, camera, run, &t, stream);
}

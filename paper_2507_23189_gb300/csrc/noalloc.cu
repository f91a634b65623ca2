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
//  * The first call on each device looks the array's device address up with
//    cudaGetSymbolAddress (with that device current) and caches it; make that
//    first call before any stream capture.
//  * All calls share the one array, which keeps what the last call left in it.
//    mc_run clears the counter on the stream before every launch, so
//    consecutive calls are independent, but calls whose work overlaps on the
//    GPU (different streams, or different host threads) race on the counter
//    and must be serialised by the caller.
//  * Nothing here calls cudaMalloc, cudaFree or an allocating library routine.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/mcmie.h"

namespace {

static __device__ __align__(256) unsigned char g_scratch[MC_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_lock;
void *g_addr[kMaxDevices] = {};

// Device address of g_scratch on the current device (looked up once).
mc_status scratch_address(void **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MC_ERR_CUDA;
    std::lock_guard<std::mutex> guard(g_lock);
    if (!g_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return MC_ERR_CUDA;
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
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

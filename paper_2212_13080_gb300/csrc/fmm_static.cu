// fmm_eval_static: one evaluation whose scratch memory is a file-scope static
// device array instead of a caller-provided workspace.
//
// Some callers cannot call cudaMalloc (or any allocator) when they evaluate:
// a plugin inside a host application whose device memory is all owned by the
// host's own allocator or pool, real-time integrators that must not allocate
// inside the time step (an allocation can stall for milliseconds or fail under
// fragmentation), and embedded deployments that fix their device memory at
// start-up.  For systems small enough to fit, this entry point lets them
// evaluate with a plan created at set-up and their own input and output
// arrays only.
#include <mutex>

#include "fmm_internal.cuh"

// Scratch of fmm_eval_static: FMM_STATIC_WORKSPACE_BYTES on every GPU that loads
// the library, held until the process exits.  Host code must not use this name
// as a device address: it needs the address cudaGetSymbolAddress returns.
static __device__ __align__(256) unsigned char g_static_workspace[FMM_STATIC_WORKSPACE_BYTES];

namespace {
const int kMaxDevices = 64;
void *g_static_addr[kMaxDevices];  // device address of the array, per device
std::mutex g_static_mutex;
}  // namespace

namespace fmm {
// Once per device, with that device current: the array's device address.
int static_workspace_address(void **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return FMM_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_static_mutex);
    if (!g_static_addr[dev]) {
        void *ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_static_workspace) != cudaSuccess || !ptr) return FMM_ERR_CUDA;
        g_static_addr[dev] = ptr;
    }
    *out = g_static_addr[dev];
    return FMM_OK;
}
}  // namespace fmm

extern "C" int fmm_eval_static(fmm_plan_t plan, int64_t n, const float *pos, const float *q,
                               void *potential, double *energy, void *forces, void *stream) {
    if (!plan) return FMM_ERR_ARG;
    // the plan's tables live on the device it was created on: the scratch must too
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return FMM_ERR_CUDA;
    if (dev != fmm::plan_device(plan)) return FMM_ERR_ARG;
    size_t need = 0;
    int rc = fmm_workspace_size(plan, n, &need);
    if (rc != FMM_OK) return rc;
    if (need > (size_t)FMM_STATIC_WORKSPACE_BYTES) return FMM_ERR_WORKSPACE;
    void *ws = nullptr;
    rc = fmm::static_workspace_address(&ws);
    if (rc != FMM_OK) return rc;
    // fmm_eval clears every part of the workspace that must start at zero, and
    // allocates nothing.
    return fmm_eval(plan, n, pos, q, potential, energy, forces, ws,
                    (size_t)FMM_STATIC_WORKSPACE_BYTES, stream);
}

// cg_run_noalloc: the stepping call for callers that cannot allocate device
// memory at run time.  Such callers exist: code that runs while a stream is
// being captured into a CUDA graph (allocation is not allowed there), hosts
// whose device memory is owned by their own pool allocator and must not see
// outside cudaMalloc calls, and real-time loops that forbid allocation after
// start-up.  They build the plan at set-up time and step with this call,
// which takes its scratch from a fixed, statically allocated device array
// instead of a caller-provided workspace.
#include <atomic>
#include <cstdint>
#include <cstdio>

#include "cardiac_gb300.h"
#include "cg_internal.h"

#define CG_API extern "C" __attribute__((visibility("default")))

namespace {

constexpr size_t NOALLOC_SCRATCH_BYTES = 32u << 20;    // 32 MiB
constexpr int MAX_DEVICES = 64;

// The scratch itself.  It is part of the library's device image, so every
// GPU that loads the library holds these 32 MiB until the process exits.
static __device__ __align__(256) unsigned char g_scratch[NOALLOC_SCRATCH_BYTES];

// Device address of g_scratch per device, looked up once per device.  In
// host code the name g_scratch is only a host-side stand-in, so the address
// must come from cudaGetSymbolAddress, called with that device current.
// Atomic entries: host threads making their first call on a device at the
// same time may both look the address up; each stores the same value.
std::atomic<void *> g_scratch_ptr[MAX_DEVICES] = {};

}  // namespace

CG_API cg_status cg_run_noalloc(cg_plan plan, const double *z_in, double *z_out, int64_t n_steps,
                                uint32_t *status_dev, void *stream)
{
    if (!plan) return cgk::set_last_error(CG_EINVAL, "plan is NULL");
    size_t need = 0;
    cg_status st = cg_workspace_size(plan, &need);
    if (st != CG_OK) return st;
    if (need > NOALLOC_SCRATCH_BYTES) {
        char msg[160];
        snprintf(msg, sizeof msg, "cg_run_noalloc: plan needs %zu bytes of scratch, the static scratch holds %zu",
                 need, NOALLOC_SCRATCH_BYTES);
        return cgk::set_last_error(CG_EINVAL, msg);
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES)
        return cgk::set_last_error(CG_ECUDA, "cg_run_noalloc: no usable current device");
    void *ws = g_scratch_ptr[dev].load(std::memory_order_acquire);
    if (ws == nullptr) {
        const cudaError_t e = cudaGetSymbolAddress(&ws, g_scratch);
        if (e != cudaSuccess || ws == nullptr)
            return cgk::set_last_error(CG_ECUDA, "cg_run_noalloc: cudaGetSymbolAddress of the static scratch failed");
        g_scratch_ptr[dev].store(ws, std::memory_order_release);
    }
    st = cg_run(plan, z_in, z_out, n_steps, ws, stream);
    if (st != CG_OK || status_dev == nullptr) return st;
    const cudaError_t e = cudaMemcpyAsync(status_dev, ws, sizeof(uint32_t), cudaMemcpyDeviceToDevice,
                                          reinterpret_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? CG_OK : cgk::set_last_error(CG_ECUDA, "cg_run_noalloc: status copy failed");
}

// pat_forward_noalloc: the forward operator with its scratch in a static
// device array instead of a caller-allocated workspace.
//
// Who needs it: a caller that cannot allocate device memory when it runs the
// forward model, for instance an acquisition or scanner process whose device
// memory budget is fixed when it starts, or a host program where another
// allocator owns all device memory; cudaMalloc can also synchronise the
// device, which a latency-critical loop cannot afford.  Such a caller still
// creates the plan beforehand and passes its own input and output buffers.
//
// The scratch is the file-scope array below, PAT_NOALLOC_SCRATCH_BYTES
// (16 MiB) per device: every GPU that loads this library holds it until the
// process exits.  Host code cannot use the array's name as a device address
// (on the host it names a stand-in object), so the first call on each device
// looks the address up with cudaGetSymbolAddress while that device is
// current and caches it; that first call should therefore come before any
// stream capture.  All calls share the one array, which keeps the contents
// of the last call; calls whose work overlaps on the GPU race on it.
#include <cuda_runtime.h>

#include <mutex>

#include "pat_internal.h"

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[PAT_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

// Device address of g_noalloc_scratch on the current device (looked up once per device).
int scratch_address(void** out) {
    int dev = -1;
    PAT_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        pat::set_error("pat_forward_noalloc: device index %d out of range", dev);
        return PAT_EINVAL;
    }
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return pat::cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return PAT_OK;
}

}  // namespace

extern "C" int pat_forward_noalloc(pat_plan p, const float* c, const float* p0, float* y, void* stream) {
    if (!p || !c || !p0 || !y) {
        pat::set_error("pat_forward_noalloc: null argument");
        return PAT_EINVAL;
    }
    if (p->ws_fwd > size_t(PAT_NOALLOC_SCRATCH_BYTES)) {
        pat::set_error("pat_forward_noalloc: this plan needs %zu bytes of scratch but the static scratch holds %d "
                       "bytes (reduce K or the grid, or use pat_forward with a workspace)",
                       p->ws_fwd, PAT_NOALLOC_SCRATCH_BYTES);
        return PAT_EINVAL;
    }
    int dev = -1;
    PAT_CUDA(cudaGetDevice(&dev));
    if (dev != p->device) {
        pat::set_error("pat_forward_noalloc: the plan's device (%d) must be current, not %d", p->device, dev);
        return PAT_EINVAL;
    }
    void* scratch = nullptr;
    int rc = scratch_address(&scratch);
    if (rc != PAT_OK) return rc;
    // the forward sweep writes every scratch region it reads before reading it,
    // so nothing left by an earlier call needs clearing
    pat::Ws w = pat::resolve(p, scratch, false);
    rc = pat::forward_sweep(p, c, p0, y, w, false, static_cast<cudaStream_t>(stream));
    if (rc != PAT_OK) return rc;
    p->hist_valid_ws = nullptr;
    return PAT_OK;
}

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
// (on the host it names a stand-in object), so every call looks the address
// up with cudaGetSymbolAddress in the context that is current.  The address
// is not cached: after cudaDeviceReset (or when the primary context is
// released and created again) the module is loaded anew and the array may
// sit elsewhere, and a cached address would then point at freed memory.  The
// first call in a context loads the module (set-up); make it before any
// stream capture.  All calls share the one array, which keeps the contents of
// the last call; calls whose work overlaps on the GPU race on it.
#include <cuda_runtime.h>

#include "pat_internal.h"

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[PAT_NOALLOC_SCRATCH_BYTES];

// Device address of g_noalloc_scratch in the current context.
int scratch_address(void** out) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return pat::cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
    *out = p;
    return PAT_OK;
}

// The plan's device must be current.
int check_device(const pat_plan_s* p, const char* who) {
    int dev = -1;
    PAT_CUDA(cudaGetDevice(&dev));
    if (dev != p->device) {
        pat::set_error("%s: the plan's device (%d) must be current, not %d", who, p->device, dev);
        return PAT_EINVAL;
    }
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
    int rc = check_device(p, "pat_forward_noalloc");
    if (rc != PAT_OK) return rc;
    void* scratch = nullptr;
    rc = scratch_address(&scratch);
    if (rc != PAT_OK) return rc;
    // the forward sweep writes every scratch region it reads before reading it,
    // so nothing left by an earlier call needs clearing
    pat::Ws w = pat::resolve(p, scratch, false);
    rc = pat::forward_sweep(p, c, p0, y, w, false, static_cast<cudaStream_t>(stream));
    if (rc != PAT_OK) return rc;
    p->hist_valid_ws = nullptr;
    return PAT_OK;
}

// Status word of the last pat_forward_noalloc of this plan: the bounded-wait bit that the
// staged row passes set in the scratch's flag region, and the bounds bit of the debug build.
extern "C" int pat_forward_noalloc_status(pat_plan p, int* h_flag, void* stream) {
    if (!p || !h_flag) {
        pat::set_error("pat_forward_noalloc_status: null argument");
        return PAT_EINVAL;
    }
    int rc = check_device(p, "pat_forward_noalloc_status");
    if (rc != PAT_OK) return rc;
    void* scratch = nullptr;
    rc = scratch_address(&scratch);
    if (rc != PAT_OK) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int f[2] = {0, 0};
    PAT_CUDA(cudaMemcpyAsync(f, static_cast<const char*>(scratch) + p->o_flag, 2 * sizeof(int),
                             cudaMemcpyDeviceToHost, st));
    PAT_CUDA(cudaStreamSynchronize(st));
    *h_flag = f[1] & (PAT_STATUS_WAIT | PAT_STATUS_QUEUE | PAT_STATUS_BOUNDS);
    return PAT_OK;
}

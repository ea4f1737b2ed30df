// Self-tests of the bounded waits: the mbarrier wait of the staged row passes (one
// CTA waits for a phase that nothing completes: no arrival, no copy in flight) and the
// dependency wait of the persistent sweep (one CTA waits for a work item that no CTA
// completes).  Each gives up after the given time and reports it in the status word,
// as a pass whose copies never land or whose producer never finishes would.  Also the
// self-test of the debug build's bounds check (an index one past the end of an array
// that has a spare element, so the guarded store is in bounds in either build).
#include <cuda_runtime.h>

#include "dcheck.cuh"
#include "kfixed.cuh"
#include "pat_internal.h"

namespace pat {
namespace {

__global__ void k_selftest_wait(int* status, unsigned long long limit_ns) {
    __shared__ uint64_t mb;
    if (threadIdx.x == 0) mbar_init(&mb, 1);   // one arrival expected, none comes
    __syncthreads();
    mbar_wait(&mb, 0, status, limit_ns);
}

// queue: [0] tickets, [1] abort flag, [2] items done of data set 0 (all zero: nothing done)
__global__ void k_selftest_queue(int* queue, int* status, unsigned long long limit_ns) {
    QueueCtx ctx{0, 0, 1, 1, queue, status, nullptr, nullptr, limit_ns};
    ctx.input_ready();   // waits for one item of data set 0 that nothing produces
}

__global__ void k_selftest_bounds(int* status) {
    __shared__ float buf[3];
    const int i = 2;   // one past the end of the checked range [0, 2)
    if (in_range(i, 2, status)) buf[i] = 1.f;
    __syncthreads();
}

}  // namespace
}  // namespace pat

using namespace pat;

extern "C" int pat_debug_bounds(void) { return kDebugBounds ? 1 : 0; }

extern "C" int pat_selftest_bounds(int* d_status, void* stream) {
    if (!d_status) { set_error("pat_selftest_bounds: null status"); return PAT_EINVAL; }
    count_launch();
    k_selftest_bounds<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(d_status);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PAT_OK : cuda_fail(e, "k_selftest_bounds");
}

extern "C" int pat_selftest_wait(int* d_status, unsigned timeout_us, void* stream) {
    if (!d_status) { set_error("pat_selftest_wait: null status"); return PAT_EINVAL; }
    if (timeout_us == 0 || timeout_us > 1000000u) {
        set_error("pat_selftest_wait: timeout_us must be in 1..1000000");
        return PAT_EINVAL;
    }
    count_launch();
    k_selftest_wait<<<1, 64, 0, static_cast<cudaStream_t>(stream)>>>(d_status, 1000ull * timeout_us);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PAT_OK : cuda_fail(e, "k_selftest_wait");
}

extern "C" int pat_selftest_queue(int* d_queue, int* d_status, unsigned timeout_us, void* stream) {
    if (!d_queue || !d_status) { set_error("pat_selftest_queue: null pointer"); return PAT_EINVAL; }
    if (timeout_us == 0 || timeout_us > 1000000u) {
        set_error("pat_selftest_queue: timeout_us must be in 1..1000000");
        return PAT_EINVAL;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    PAT_CUDA(cudaMemsetAsync(d_queue, 0, 3 * sizeof(int), st));
    count_launch();
    k_selftest_queue<<<1, 64, 0, st>>>(d_queue, d_status, 1000ull * timeout_us);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PAT_OK : cuda_fail(e, "k_selftest_queue");
}

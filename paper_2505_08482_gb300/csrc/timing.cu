// Launch counting and optional per-kernel-class timing with CUDA events
// recorded on the launching stream (used by the benchmark's roofline).
#include <cuda_runtime.h>

#include <atomic>
#include <vector>

#include "pat_internal.h"

namespace pat {

namespace {
struct Timing {
    int cls = 0;
    int used = 0;
    int every = 1;    // time every n-th launch of the class
    long long seen = 0;
    bool open = false;
    std::vector<cudaEvent_t> t0, t1;
};
Timing g_t;
std::atomic<unsigned long long> g_launches{0};   // batched solves may launch from several threads
}  // namespace

void count_launch() { ++g_launches; }
void add_launches(unsigned long long n) { g_launches += n; }
unsigned long long launches_so_far() { return g_launches.load(); }

void prof_begin(int cls, cudaStream_t st) {
    ++g_launches;
    if (g_t.cls != cls) return;
    g_t.open = (g_t.seen++ % g_t.every) == 0 && g_t.used < int(g_t.t0.size());
    if (g_t.open) cudaEventRecord(g_t.t0[g_t.used], st);
}

void prof_end(int cls, cudaStream_t st) {
    if (g_t.cls == cls && g_t.open) {
        cudaEventRecord(g_t.t1[g_t.used], st);
        ++g_t.used;
        g_t.open = false;
    }
}

}  // namespace pat

using namespace pat;

extern "C" unsigned long long pat_kernel_launches(void) { return g_launches.load(); }

extern "C" int pat_timing_enable(int cls, int max_launches, int every) {
    for (cudaEvent_t e : g_t.t0) cudaEventDestroy(e);
    for (cudaEvent_t e : g_t.t1) cudaEventDestroy(e);
    g_t.t0.clear();
    g_t.t1.clear();
    g_t.used = 0;
    g_t.cls = 0;
    g_t.seen = 0;
    g_t.open = false;
    g_t.every = every < 1 ? 1 : every;
    if (cls <= 0 || max_launches <= 0) return PAT_OK;
    if (cls > PAT_K_LAST) { set_error("pat_timing_enable: unknown kernel class %d", cls); return PAT_EINVAL; }
    g_t.t0.resize(max_launches);
    g_t.t1.resize(max_launches);
    for (int i = 0; i < max_launches; ++i) {
        PAT_CUDA(cudaEventCreate(&g_t.t0[i]));
        PAT_CUDA(cudaEventCreate(&g_t.t1[i]));
    }
    g_t.cls = cls;
    return PAT_OK;
}

extern "C" int pat_timing_read(double* total_ms, long long* launches) {
    if (!total_ms || !launches) { set_error("pat_timing_read: null argument"); return PAT_EINVAL; }
    double tot = 0.0;
    if (g_t.used > 0) PAT_CUDA(cudaEventSynchronize(g_t.t1[g_t.used - 1]));
    for (int i = 0; i < g_t.used; ++i) {
        float ms = 0.f;
        PAT_CUDA(cudaEventElapsedTime(&ms, g_t.t0[i], g_t.t1[i]));
        tot += ms;
    }
    *total_ms = tot;
    *launches = g_t.used;
    g_t.used = 0;
    return PAT_OK;
}

// Internal declarations of the k-space solver library: plan, workspace
// layout and kernel launchers.
#pragma once

#include <cuda_runtime.h>

#include <array>
#include <cstddef>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/pat.h"
#include "fft.cuh"

namespace pat {

struct FixedOps;
struct SweepOps;
struct ClusterOps;

// NVTX range on the host timeline for the lifetime of the object (profilers show the library's
// calls, sweeps and multigrid levels by name; without a profiler attached it costs a branch)
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};
void set_error(const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* where);

#define PAT_CUDA(call)                                           \
    do {                                                         \
        cudaError_t e_ = (call);                                 \
        if (e_ != cudaSuccess) return ::pat::cuda_fail(e_, #call); \
    } while (0)

// Device tables of one plan (all built in FP64 on the host, stored FP32).
struct Tables {
    float2* tw;        // [ng] exp(-2 pi i q / ng)
    float* kappa_t;    // [hc][ng] kappa(kx, ky) at kx * ng + ky
    float2* fx;        // [hc] i kx exp(+i kx dx/2)   (x factor of G; D uses -conj)
    float2* fy;        // [ng] i ky exp(+i ky dx/2)   (y factor of G; D uses -conj)
    float* a_cell;     // [ng] PML factor at cell centres
    float* a_stag;     // [ng] PML factor at +1/2 cell
    int* srow;         // [ng+1] CSR row pointer of sensor stencil entries
    int2* sent;        // [nent] (sensor m, column ix) per entry
    float4* sentw;     // [nent] (w_x0, w_x1, w_y, row) per entry
    int* kinst;        // [K] instance of each data set
    int* kfirst;       // [ninst+1] first data set of each instance
};

// Workspace regions (device pointers resolved from the caller's base).
struct Ws {
    float* ux; float* uy; float* rx; float* ry;   // forward state [K][ng][ng] each (contiguous)
    float* cg;                                    // c on the grid [ninst][ng][ng]
    float2* A; float2* B;                         // spectra [K][ng][hc]
    double* J; double* part; int* flag;           // objective per instance, partial sums [K][32], flag
    int* queue;                                   // persistent sweep: tickets, abort flag, done per data set
    // gradient only
    float* ckpt;                                  // [nseg-1][4][K][ng][ng]
    float* hist;                                  // [2][K][s_eff][ng][ng] pressure history (two segments)
    float* ubx; float* uby; float* rbx; float* rby;  // adjoint state [K][ng][ng]
    float2* A2; float2* B2;                       // adjoint spectra
    float* cbar;                                  // [K][n][n]
    float* resid;                                 // [K][nt][m]
    float* ypred;                                 // [K][nt][m]
};

constexpr int kPartials = 256;
constexpr int kResidBlocks = 32;   // residual partial sums per data set

}  // namespace pat

struct pat_plan_s {
    pat_grid g;
    int n, P, ng, hc, hp, K, nt, m, s, s_eff, nseg;   // hp: spectrum row pitch (hc rounded up to 4)
    int ninst;         // instances sharing the grid; K counts the data sets of all of them
    pat::FftDesc fft;
    const pat::FixedOps* fast;   // fixed-size passes for this grid side (nullptr: generic Stockham)
    const pat::SweepOps* sweep;  // persistent forward sweep of this grid side (nullptr: none)
    bool persistent;             // forward sweeps run as one persistent launch
    const pat::ClusterOps* clops;   // cluster-resident stepping of this grid side (nullptr: none)
    bool cluster;                // forward sweeps and segment recomputes run cluster-resident
    int variant;       // -1 generic, else index of the fixed-size tile variant
    int R;             // rows per CTA in row passes (even)
    int C;             // spectral columns per CTA in column passes
    size_t smem_row, smem_col;
    void* dev;         // one device allocation for the tables
    pat::Tables t;
    int nent;
    size_t ws_fwd, ws_grad;
    // layout offsets (bytes)
    size_t o_state, o_cg, o_A, o_B, o_J, o_part, o_flag, o_queue;
    size_t o_ckpt, o_hist, o_adj, o_A2, o_B2, o_cbar, o_resid, o_ypred;
    // host bookkeeping: the workspace whose history holds the last segment
    const void* hist_valid_ws;
    int device;
    // captured CUDA graphs of whole calls, keyed by call kind, buffers and variant;
    // at most kMaxGraphs are kept, the least recently replayed one is dropped first
    static constexpr size_t kMaxGraphs = 16;
    struct Graph {
        int kind, variant;
        std::array<const void*, 10> key;
        size_t ws_bytes;
        cudaGraphExec_t exec;
        unsigned long long launches;
        unsigned long long last_use;
    };
    bool use_graphs;
    std::vector<Graph> graphs;
    unsigned long long graph_clock;
    // second stream and events of the reverse sweep (recompute overlapped with the adjoint)
    cudaStream_t side;
    cudaEvent_t ev_start, ev_rec[2], ev_adj[2];
};

namespace pat {

Ws resolve(const pat_plan_s* p, void* base, bool grad);

// pressure history buffer of segment j (segments alternate between two buffers)
inline float* hist_of(const pat_plan_s* p, const Ws& w, int j) {
    return w.hist + size_t(j & 1) * p->K * p->s_eff * p->ng * p->ng;
}

// launch accounting / optional event timing of one kernel class (timing.cu)
void count_launch();
void add_launches(unsigned long long n);
unsigned long long launches_so_far();
void prof_begin(int cls, cudaStream_t st);
void prof_end(int cls, cudaStream_t st);

// ---- kernel launchers (kernels.cu) ----
struct Launch {
    const pat_plan_s* p;
    cudaStream_t st;
    bool solo = false;        // no other stream of this call runs beside it (the forward sweep)
    bool recompute = false;   // the segment recompute, which runs beside the adjoint
};

int configure_kernels(pat_plan_s* p);
bool radix_schedule(int n, FftDesc* fd);   // radix 4/5/3/2 schedule of a 5-smooth length
int check_launch(const char* what);   // PAT_OK or the pending launch error
int select_variant(pat_plan_s* p, int variant);

// forward
int launch_medium(const Launch& L, const float* c_dom, float* cg);
// row pass producing rho and p (mode 0 regular, 1 init from p0, 2 restore)
int launch_row_rho(const Launch& L, const Ws& w, int mode, const float* p0, float* y, int tstep,
                   float* hist, int hist_slot);
int launch_row_u(const Launch& L, const Ws& w, int init);
// the whole forward sweep (initial pass and nt-1 steps) as one persistent launch; checkpoints
// every s steps into ckpt (null: none), pressure history of levels >= last0 into hist (null: none)
int launch_forward_persistent(const Launch& L, const Ws& w, const float* p0, float* y, float* hist, int last0,
                              float* ckpt);
// column passes: mode 0 = one input (A) -> (MX A, MY A) into (A, B)
//                mode 1 = (A, B) -> (MX A, MY B); mode 2 = (A, B) -> MX A + MY B into A
// op 0: G multipliers, op 1: D multipliers
int launch_col(const Launch& L, float2* A, float2* B, int mode, int op, float scale);
// adjoint
int launch_row_adj_rho(const Launch& L, const Ws& w, int first, const float* resid, int tstep,
                       const float* hist, int hist_slot);
int launch_row_adj_u(const Launch& L, const Ws& w);
int launch_row_adj_final1(const Launch& L, const Ws& w, int first, const float* resid, float* grad_p0);
int launch_row_adj_final2(const Launch& L, const Ws& w, const float* p0, float* grad_p0);
int launch_reduce_cbar(const Launch& L, const Ws& w, float* grad_c);
int launch_residual(const Launch& L, const Ws& w, const float* ypred, const float* ymeas,
                    const float* wts, float* resid, double* J_out);

// cluster-resident forward steps n0 .. n1-1 (kcluster.cuh): from p0 (init, n0 = 0) or from the
// state [4][K][ng][ng] at level n0; traces into y (or null), pressure history of levels
// >= hist_base into hist (or null), checkpoints every s levels into ckpt (or null), the final
// state into state_out (or null)
int launch_forward_cluster(const Launch& L, const Ws& w, const float* p0, const float* state, int n0, int n1,
                           float* y, float* hist, int hist_base, float* ckpt, float* state_out);

// ---- api.cu internals ----
// Forward sweep into y [K][nt][m] with workspace regions w (checkpoints kept if keep).
int forward_sweep(pat_plan_s* p, const float* c, const float* p0, float* y, const Ws& w, bool keep,
                  cudaStream_t st);
// used by the reconstruction driver:
// J only (forward sweep + residual) into *J_dev; workspace of PAT_WS_GRADIENT size.
int objective(pat_plan_s* p, const float* c, const float* p0, const float* ymeas, const float* wts, double* J_dev,
              void* ws, size_t ws_bytes, cudaStream_t st);

}  // namespace pat

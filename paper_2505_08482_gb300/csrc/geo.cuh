// Per-plan constants of the kernels and the half-spectrum packing helpers
// shared by the generic (Stockham) and the fixed-size (two-level) passes.
#pragma once

#include <cuda_runtime.h>

#include "pat_internal.h"

namespace pat {

// Per-plan constants passed by value.
struct Geo {
    int ng, hc, hp, n, P, K, nt, m, s_eff;   // hp: row pitch of a spectrum (>= hc)
    FftDesc fft;
    const float2* tw;
    const float* kappa_t;
    const float2* fx;
    const float2* fy;
    const float* a_cell;
    const float* a_stag;
    const int* srow;
    const int2* sent;
    const float4* sentw;
    const int* kinst;    // instance of each data set (selects its c)
    int* status;         // workspace status word of bounded waits (nullptr: not reported)
};

inline Geo geo(const pat_plan_s* p) {
    Geo g;
    g.ng = p->ng; g.hc = p->hc; g.hp = p->hp; g.n = p->n; g.P = p->P; g.K = p->K; g.nt = p->nt; g.m = p->m;
    g.s_eff = p->s_eff;
    g.fft = p->fft;
    g.tw = p->t.tw; g.kappa_t = p->t.kappa_t; g.fx = p->t.fx; g.fy = p->t.fy;
    g.a_cell = p->t.a_cell; g.a_stag = p->t.a_stag;
    g.srow = p->t.srow; g.sent = p->t.sent; g.sentw = p->t.sentw;
    g.kinst = p->t.kinst;
    g.status = nullptr;
    return g;
}

// Programmatic dependent launch: wait until the preceding kernel of the stream
// has completed and its writes are visible (a no-op without the launch
// attribute), then let the next kernel be scheduled.  A kernel may read data
// written two or more kernels earlier before the wait, but data written by the
// immediately preceding kernel only after it.
__device__ __forceinline__ void pdl_wait_then_release() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// c of data set k's instance on the grid
__device__ __forceinline__ const float* medium_of(const Geo& g, const float* cg, int k) {
    return cg + size_t(g.kinst[k]) * g.ng * g.ng;
}

__device__ __forceinline__ void load_twiddles(float2* tw, const Geo& g) {
    for (int i = threadIdx.x; i < g.ng; i += blockDim.x) tw[i] = g.tw[i];
}

// z[j][.] = full spectrum of a_j + i b_j from the half spectra a_j, b_j
// (bins 0 and Ng/2 keep their real parts only: the rows are real).
__device__ __forceinline__ void put_c2r(float2* zrow, int ng, int kx, float2 a, float2 b) {
    if (kx == 0 || 2 * kx == ng) {
        a.y = 0.f;
        b.y = 0.f;
    }
    zrow[kx] = make_float2(a.x - b.y, a.y + b.x);
    if (kx > 0 && 2 * kx < ng) zrow[ng - kx] = make_float2(a.x + b.y, b.x - a.y);
}

// Split the FFT of a + i b into the half spectra of a and b at bin kx.
__device__ __forceinline__ void get_r2c(const float2* zrow, int ng, int kx, float2& A, float2& B) {
    const float2 zk = zrow[kx];
    const float2 zm = zrow[kx == 0 ? 0 : ng - kx];
    A = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
    B = make_float2(0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x));
}

}  // namespace pat

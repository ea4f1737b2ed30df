// Row and column passes of the k-space pseudospectral scheme (forward and
// discrete adjoint), plus the small medium / residual / reduction kernels.
//
// A time step of the forward solve (Sec. 2.1, split-field staggered k-space
// leapfrog) is four passes over the K data sets:
//   col  G   : row spectrum of p  -> FFT_y -> (G_x, G_y multipliers) -> IFFT_y
//   row  U   : C2R of both derivatives, PML velocity update, R2C of (u_x, u_y)
//   col  D   : FFT_y -> (D_x, D_y multipliers) -> IFFT_y
//   row  RHO : C2R, PML density update, p = c^2 (rho_x + rho_y), sensor
//              gather, optional pressure history, R2C of p for the next step.
// Spectra are stored row-major [K][Ng][Ng/2+1] (x half spectrum, y full).
// Two real rows are transformed with one complex FFT (z = a + i b); the
// 1/Ng^2 normalisation and the dt, rho0 factors are folded into the
// k-space multipliers of the column pass.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <mutex>

#include "pat_internal.h"
#include "geo.cuh"
#include "dcheck.cuh"
#include "kfixed.cuh"
#include "kcluster.cuh"

namespace pat {

// ---------------------------------------------------------------------------
// forward: row pass producing rho^{n+1}, p^{n+1}
//   mode 0: C2R of (A, B) = (dt rho0 D_x u_x, dt rho0 D_y u_y), PML update
//   mode 1: initial condition from p0 (rho = p0 / (2 c^2))
//   mode 2: p from the stored rho (restart from a checkpoint)
// then: sensor gather into y[k][tstep][:] (if y), history (if hist), R2C of p -> A.
__global__ void __launch_bounds__(256) k_row_rho(Geo g, float2* __restrict__ A, const float2* __restrict__ B,
                                                 float* __restrict__ rx, float* __restrict__ ry,
                                                 const float* __restrict__ cg, int mode,
                                                 const float* __restrict__ p0, float* __restrict__ y, int tstep,
                                                 float* __restrict__ hist, int hist_slot, int R) {
    extern __shared__ float2 sm[];
    const int ng = g.ng, hc = g.hc;
    const int k = blockIdx.y;
    const int y0 = blockIdx.x * R;
    const int nr = min(R, ng - y0);
    const int hslot = hist ? in_range_or_zero(hist_slot, g.s_eff, g.status) : 0;
    float2* tw = sm;
    float2* z = sm + ng;
    float2* w = z + R * ng;
    load_twiddles(tw, g);
    const size_t kf = size_t(k) * ng * ng;
    cg = medium_of(g, cg, k);
    float* pr;
    float2* freeb;
    if (mode == 0) {
        for (int i = threadIdx.x; i < nr * hc; i += blockDim.x) {
            const int r = i / hc, kx = i - r * hc;
            const size_t gi = (size_t(k) * ng + y0 + r) * g.hp + kx;
            put_c2r(z + r * ng, ng, kx, A[gi], B[gi]);
        }
        __syncthreads();
        float2* res = fft_smem<true>(z, w, nr, ng, g.fft, tw);
        float2* oth = (res == z) ? w : z;
        pr = reinterpret_cast<float*>(oth);
        for (int i = threadIdx.x; i < nr * ng; i += blockDim.x) {
            const int r = i / ng, x = i - r * ng, yy = y0 + r;
            const size_t o = kf + size_t(yy) * ng + x;
            const float2 gv = res[i];
            const float acx = g.a_cell[x], acy = g.a_cell[yy];
            const float rxn = acx * (acx * rx[o] - gv.x);
            const float ryn = acy * (acy * ry[o] - gv.y);
            rx[o] = rxn;
            ry[o] = ryn;
            const float c = cg[size_t(yy) * ng + x];
            const float pv = c * c * (rxn + ryn);
            pr[i] = pv;
            if (hist) hist[(size_t(k) * g.s_eff + hslot) * ng * ng + size_t(yy) * ng + x] = pv;
        }
        freeb = res;
    } else {
        __syncthreads();
        pr = reinterpret_cast<float*>(w);
        for (int i = threadIdx.x; i < nr * ng; i += blockDim.x) {
            const int r = i / ng, x = i - r * ng, yy = y0 + r;
            const size_t o = kf + size_t(yy) * ng + x;
            const float c = cg[size_t(yy) * ng + x];
            float pv;
            if (mode == 1) {
                const int xd = x - g.P, yd = yy - g.P;
                pv = (xd >= 0 && xd < g.n && yd >= 0 && yd < g.n) ? p0[(size_t(k) * g.n + yd) * g.n + xd] : 0.f;
                const float rv = pv / (2.f * c * c);
                rx[o] = rv;
                ry[o] = rv;
            } else {
                pv = c * c * (rx[o] + ry[o]);
            }
            pr[i] = pv;
            if (hist) hist[(size_t(k) * g.s_eff + hslot) * ng * ng + size_t(yy) * ng + x] = pv;
        }
        freeb = z;
    }
    __syncthreads();
    if (y) {
        const int e0 = g.srow[y0], e1 = g.srow[y0 + nr];
        for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
            const int2 se = g.sent[e];
            const float4 sw = g.sentw[e];
            const int r = int(sw.w) - y0;
            if (!(in_range(r, nr, g.status) && in_range(se.y + 1, ng, g.status) && in_range(se.x, g.m, g.status) &&
                  in_range(tstep, g.nt, g.status)))
                continue;
            const float v = sw.z * (sw.x * pr[r * ng + se.y] + sw.y * pr[r * ng + se.y + 1]);
            // at most two adds (rows iy, iy+1) onto a zeroed sample: order-independent
            atomicAdd(&y[(size_t(k) * g.nt + tstep) * g.m + se.x], v);
        }
    }
    const int np = nr / 2;
    for (int i = threadIdx.x; i < np * ng; i += blockDim.x) {
        const int j = i / ng, x = i - j * ng;
        freeb[i] = make_float2(pr[(2 * j) * ng + x], pr[(2 * j + 1) * ng + x]);
    }
    __syncthreads();
    float2* res2 = fft_smem<false>(freeb, reinterpret_cast<float2*>(pr), np, ng, g.fft, tw);
    for (int i = threadIdx.x; i < np * hc; i += blockDim.x) {
        const int j = i / hc, kx = i - j * hc;
        float2 a, b;
        get_r2c(res2 + j * ng, ng, kx, a, b);
        A[(size_t(k) * ng + y0 + 2 * j) * g.hp + kx] = a;
        A[(size_t(k) * ng + y0 + 2 * j + 1) * g.hp + kx] = b;
    }
}

// forward: row pass producing u^{n+1/2} from (A, B) = (dt/rho0 G_x p, dt/rho0 G_y p);
// init: u^{-1/2} = dt/(2 rho0) G p0 first.  Writes the R2C of (u_x, u_y) into (A, B).
__global__ void __launch_bounds__(256) k_row_u(Geo g, float2* __restrict__ A, float2* __restrict__ B,
                                               float* __restrict__ ux, float* __restrict__ uy, int init, int R) {
    extern __shared__ float2 sm[];
    const int ng = g.ng, hc = g.hc;
    const int k = blockIdx.y;
    const int y0 = blockIdx.x * R;
    const int nr = min(R, ng - y0);
    float2* tw = sm;
    float2* z = sm + ng;
    float2* w = z + R * ng;
    load_twiddles(tw, g);
    for (int i = threadIdx.x; i < nr * hc; i += blockDim.x) {
        const int r = i / hc, kx = i - r * hc;
        const size_t gi = (size_t(k) * ng + y0 + r) * g.hp + kx;
        put_c2r(z + r * ng, ng, kx, A[gi], B[gi]);
    }
    __syncthreads();
    float2* res = fft_smem<true>(z, w, nr, ng, g.fft, tw);
    float2* oth = (res == z) ? w : z;
    const size_t kf = size_t(k) * ng * ng;
    for (int i = threadIdx.x; i < nr * ng; i += blockDim.x) {
        const int r = i / ng, x = i - r * ng, yy = y0 + r;
        const size_t o = kf + size_t(yy) * ng + x;
        const float2 gv = res[i];
        const float ax = g.a_stag[x], ay = g.a_stag[yy];
        const float uxo = init ? 0.5f * gv.x : ux[o];
        const float uyo = init ? 0.5f * gv.y : uy[o];
        const float uxn = ax * (ax * uxo - gv.x);
        const float uyn = ay * (ay * uyo - gv.y);
        ux[o] = uxn;
        uy[o] = uyn;
        res[i] = make_float2(uxn, uyn);
    }
    __syncthreads();
    float2* res2 = fft_smem<false>(res, oth, nr, ng, g.fft, tw);
    for (int i = threadIdx.x; i < nr * hc; i += blockDim.x) {
        const int r = i / hc, kx = i - r * hc;
        float2 a, b;
        get_r2c(res2 + r * ng, ng, kx, a, b);
        const size_t gi = (size_t(k) * ng + y0 + r) * g.hp + kx;
        A[gi] = a;
        B[gi] = b;
    }
}

// ---------------------------------------------------------------------------
// column pass: FFT along y of C spectral columns, k-space multipliers, IFFT.
//   op 0: G multipliers  i k kappa exp(+i k dx/2);  op 1: D multipliers i k kappa exp(-i k dx/2)
//   mode 0: A -> (MX A, MY A) into (A, B); mode 1: (A, B) -> (MX A, MY B); mode 2: MX A + MY B -> A
__global__ void __launch_bounds__(256) k_col(Geo g, float2* __restrict__ A, float2* __restrict__ B,
                                             int mode, int op, float scale, int C) {
    extern __shared__ float2 sm[];
    const int ng = g.ng, hc = g.hc;
    const int k = blockIdx.y;
    const int kx0 = blockIdx.x * C;
    float2* tw = sm;
    float2* b0 = sm + ng;
    float2* b1 = b0 + 2 * C * ng;
    load_twiddles(tw, g);
    const int nin = (mode == 0) ? 1 : 2;
    for (int i = threadIdx.x; i < nin * C * ng; i += blockDim.x) {
        const int c = i % C;
        const int rest = i / C;
        const int ky = rest % ng;
        const int src = rest / ng;
        const int kx = kx0 + c;
        float2 v = make_float2(0.f, 0.f);
        if (kx < hc) v = (src == 0 ? A : B)[(size_t(k) * ng + ky) * g.hp + kx];
        b0[(src * C + c) * ng + ky] = v;
    }
    __syncthreads();
    float2* res = fft_smem<false>(b0, b1, nin * C, ng, g.fft, tw);
    for (int i = threadIdx.x; i < C * ng; i += blockDim.x) {
        const int c = i / ng, ky = i - c * ng;
        const int kx = kx0 + c;
        if (kx >= hc) continue;
        const float kap = scale * g.kappa_t[size_t(kx) * ng + ky];
        float2 mx = g.fx[kx], my = g.fy[ky];
        if (op == 1) {  // -conj: D factor from the G factor
            mx.x = -mx.x;
            my.x = -my.x;
        }
        mx = cscale(mx, kap);
        my = cscale(my, kap);
        float2* s0 = res + c * ng + ky;
        float2* s1 = res + (C + c) * ng + ky;
        if (mode == 0) {
            const float2 X = *s0;
            *s0 = cmul(X, mx);
            *s1 = cmul(X, my);
        } else if (mode == 1) {
            *s0 = cmul(*s0, mx);
            *s1 = cmul(*s1, my);
        } else {
            *s0 = cadd(cmul(*s0, mx), cmul(*s1, my));
        }
    }
    __syncthreads();
    const int nout = (mode == 2) ? 1 : 2;
    float2* oth = (res == b0) ? b1 : b0;
    float2* res2 = fft_smem<true>(res, oth, nout * C, ng, g.fft, tw);
    for (int i = threadIdx.x; i < nout * C * ng; i += blockDim.x) {
        const int c = i % C;
        const int rest = i / C;
        const int ky = rest % ng;
        const int dst = rest / ng;
        const int kx = kx0 + c;
        if (kx < hc) (dst == 0 ? A : B)[(size_t(k) * ng + ky) * g.hp + kx] = res2[(dst * C + c) * ng + ky];
    }
}

// ---------------------------------------------------------------------------
// adjoint helpers: C2R of one spectrum for pairs of rows into real rows pb[nr][ng]
// (returns the free complex buffer); pb lives in the other buffer.
__device__ __forceinline__ float2* c2r_rows(const Geo& g, const float2* __restrict__ Q, int k, int y0, int nr,
                                            float2* z, float2* w, const float2* tw, float*& pb) {
    const int ng = g.ng, hc = g.hc;
    const int np = nr / 2;
    for (int i = threadIdx.x; i < np * hc; i += blockDim.x) {
        const int j = i / hc, kx = i - j * hc;
        const float2 a = Q[(size_t(k) * ng + y0 + 2 * j) * g.hp + kx];
        const float2 b = Q[(size_t(k) * ng + y0 + 2 * j + 1) * g.hp + kx];
        put_c2r(z + j * ng, ng, kx, a, b);
    }
    __syncthreads();
    float2* res = fft_smem<true>(z, w, np, ng, g.fft, tw);
    float2* oth = (res == z) ? w : z;
    pb = reinterpret_cast<float*>(oth);
    for (int i = threadIdx.x; i < np * ng; i += blockDim.x) {
        const int j = i / ng, x = i - j * ng;
        const float2 v = res[i];
        pb[(2 * j) * ng + x] = v.x;
        pb[(2 * j + 1) * ng + x] = v.y;
    }
    __syncthreads();
    return res;
}

// S^T r^tstep added into the real rows pb (one thread per row: fixed order).
__device__ __forceinline__ void scatter_rows(const Geo& g, float* pb, const float* __restrict__ resid, int k,
                                             int tstep, int y0, int nr) {
    if (threadIdx.x < nr) {
        const int r = threadIdx.x, yy = y0 + r;
        const float* rv = resid + (size_t(k) * g.nt + in_range_or_zero(tstep, g.nt, g.status)) * g.m;
        for (int e = g.srow[yy]; e < g.srow[yy + 1]; ++e) {
            const int2 se = g.sent[e];
            const float4 sw = g.sentw[e];
            if (!(in_range(se.x, g.m, g.status) && in_range(se.y + 1, g.ng, g.status))) continue;
            const float v = rv[se.x] * sw.z;
            pb[r * g.ng + se.y] += sw.x * v;
            pb[r * g.ng + se.y + 1] += sw.y * v;
        }
    }
    __syncthreads();
}

// adjoint of the density update at step n (n >= 1):
//   pb^n = C2R(Q) + S^T r^n;  rb += c^2 pb;  cbar += 2 c rho^n pb (= 2 p^n pb / c);
//   t = a rb;  rb <- a t;  (A2, B2) <- R2C(t_x, t_y)
__global__ void __launch_bounds__(256) k_row_adj_rho(Geo g, float2* __restrict__ A2, float2* __restrict__ B2,
                                                     float* __restrict__ rbx, float* __restrict__ rby,
                                                     float* __restrict__ cbar, const float* __restrict__ cg,
                                                     int first, const float* __restrict__ resid, int tstep,
                                                     const float* __restrict__ hist, int hist_slot, int R) {
    extern __shared__ float2 sm[];
    const int ng = g.ng, hc = g.hc;
    const int k = blockIdx.y;
    const int y0 = blockIdx.x * R;
    const int nr = min(R, ng - y0);
    float2* tw = sm;
    float2* z = sm + ng;
    float2* w = z + R * ng;
    load_twiddles(tw, g);
    float* pb;
    float2* freeb;
    if (!first) {
        freeb = c2r_rows(g, A2, k, y0, nr, z, w, tw, pb);
    } else {
        pb = reinterpret_cast<float*>(w);
        for (int i = threadIdx.x; i < nr * ng; i += blockDim.x) pb[i] = 0.f;
        freeb = z;
        __syncthreads();
    }
    scatter_rows(g, pb, resid, k, tstep, y0, nr);
    const size_t kf = size_t(k) * ng * ng;
    cg = medium_of(g, cg, k);
    const float* hp = hist + (size_t(k) * g.s_eff + in_range_or_zero(hist_slot, g.s_eff, g.status)) * ng * ng;
    for (int i = threadIdx.x; i < nr * ng; i += blockDim.x) {
        const int r = i / ng, x = i - r * ng, yy = y0 + r;
        const size_t o = kf + size_t(yy) * ng + x;
        const float p_b = pb[i];
        const float c = cg[size_t(yy) * ng + x];
        const float c2 = c * c;
        const float vbx = rbx[o] + c2 * p_b;
        const float vby = rby[o] + c2 * p_b;
        const int xd = x - g.P, yd = yy - g.P;
        if (xd >= 0 && xd < g.n && yd >= 0 && yd < g.n) {
            float* cb = cbar + (size_t(k) * g.n + yd) * g.n + xd;
            *cb += 2.f * hp[size_t(yy) * ng + x] * p_b / c;
        }
        const float acx = g.a_cell[x], acy = g.a_cell[yy];
        const float tx = acx * vbx, ty = acy * vby;
        rbx[o] = acx * tx;
        rby[o] = acy * ty;
        freeb[i] = make_float2(tx, ty);
    }
    __syncthreads();
    float2* res2 = fft_smem<false>(freeb, reinterpret_cast<float2*>(pb), nr, ng, g.fft, tw);
    for (int i = threadIdx.x; i < nr * hc; i += blockDim.x) {
        const int r = i / hc, kx = i - r * hc;
        float2 a, b;
        get_r2c(res2 + r * ng, ng, kx, a, b);
        const size_t gi = (size_t(k) * ng + y0 + r) * g.hp + kx;
        A2[gi] = a;
        B2[gi] = b;
    }
}

// adjoint of the velocity update: ub += C2R(A2, B2) (= dt rho0 G t);
//   t' = a' ub;  ub <- a' t';  (A2, B2) <- R2C(t'_x, t'_y)
__global__ void __launch_bounds__(256) k_row_adj_u(Geo g, float2* __restrict__ A2, float2* __restrict__ B2,
                                                   float* __restrict__ ubx, float* __restrict__ uby, int R) {
    extern __shared__ float2 sm[];
    const int ng = g.ng, hc = g.hc;
    const int k = blockIdx.y;
    const int y0 = blockIdx.x * R;
    const int nr = min(R, ng - y0);
    float2* tw = sm;
    float2* z = sm + ng;
    float2* w = z + R * ng;
    load_twiddles(tw, g);
    for (int i = threadIdx.x; i < nr * hc; i += blockDim.x) {
        const int r = i / hc, kx = i - r * hc;
        const size_t gi = (size_t(k) * ng + y0 + r) * g.hp + kx;
        put_c2r(z + r * ng, ng, kx, A2[gi], B2[gi]);
    }
    __syncthreads();
    float2* res = fft_smem<true>(z, w, nr, ng, g.fft, tw);
    float2* oth = (res == z) ? w : z;
    const size_t kf = size_t(k) * ng * ng;
    for (int i = threadIdx.x; i < nr * ng; i += blockDim.x) {
        const int r = i / ng, x = i - r * ng, yy = y0 + r;
        const size_t o = kf + size_t(yy) * ng + x;
        const float2 gv = res[i];
        const float ax = g.a_stag[x], ay = g.a_stag[yy];
        const float tpx = ax * (ubx[o] + gv.x);
        const float tpy = ay * (uby[o] + gv.y);
        ubx[o] = ax * tpx;
        uby[o] = ay * tpy;
        res[i] = make_float2(tpx, tpy);
    }
    __syncthreads();
    float2* res2 = fft_smem<false>(res, oth, nr, ng, g.fft, tw);
    for (int i = threadIdx.x; i < nr * hc; i += blockDim.x) {
        const int r = i / hc, kx = i - r * hc;
        float2 a, b;
        get_r2c(res2 + r * ng, ng, kx, a, b);
        const size_t gi = (size_t(k) * ng + y0 + r) * g.hp + kx;
        A2[gi] = a;
        B2[gi] = b;
    }
}

// n = 0, part 1: pb^0 = C2R(Q) + S^T r^0 written to grad_p0 (domain);
// (A2, B2) <- R2C(ub_x^{-1/2}, ub_y^{-1/2}) for the initial-velocity transpose.
__global__ void __launch_bounds__(256) k_row_adj_final1(Geo g, float2* __restrict__ A2, float2* __restrict__ B2,
                                                        const float* __restrict__ ubx, const float* __restrict__ uby,
                                                        int first, const float* __restrict__ resid,
                                                        float* __restrict__ grad_p0, int R) {
    extern __shared__ float2 sm[];
    const int ng = g.ng, hc = g.hc;
    const int k = blockIdx.y;
    const int y0 = blockIdx.x * R;
    const int nr = min(R, ng - y0);
    float2* tw = sm;
    float2* z = sm + ng;
    float2* w = z + R * ng;
    load_twiddles(tw, g);
    float* pb;
    float2* freeb;
    if (!first) {
        freeb = c2r_rows(g, A2, k, y0, nr, z, w, tw, pb);
    } else {
        pb = reinterpret_cast<float*>(w);
        for (int i = threadIdx.x; i < nr * ng; i += blockDim.x) pb[i] = 0.f;
        freeb = z;
        __syncthreads();
    }
    scatter_rows(g, pb, resid, k, 0, y0, nr);
    const size_t kf = size_t(k) * ng * ng;
    for (int i = threadIdx.x; i < nr * ng; i += blockDim.x) {
        const int r = i / ng, x = i - r * ng, yy = y0 + r;
        const int xd = x - g.P, yd = yy - g.P;
        if (xd >= 0 && xd < g.n && yd >= 0 && yd < g.n) grad_p0[(size_t(k) * g.n + yd) * g.n + xd] = pb[i];
        const size_t o = kf + size_t(yy) * ng + x;
        freeb[i] = make_float2(ubx[o], uby[o]);
    }
    __syncthreads();
    float2* res2 = fft_smem<false>(freeb, reinterpret_cast<float2*>(pb), nr, ng, g.fft, tw);
    for (int i = threadIdx.x; i < nr * hc; i += blockDim.x) {
        const int r = i / hc, kx = i - r * hc;
        float2 a, b;
        get_r2c(res2 + r * ng, ng, kx, a, b);
        const size_t gi = (size_t(k) * ng + y0 + r) * g.hp + kx;
        A2[gi] = a;
        B2[gi] = b;
    }
}

// n = 0, part 2: grad_p0 += C2R(A2) (= -dt/(2 rho0) D.ub^{-1/2}) + (rb_x + rb_y)/(2 c^2);
//                cbar -= (rb_x + rb_y) p0 / c^3   (domain cells)
__global__ void __launch_bounds__(256) k_row_adj_final2(Geo g, const float2* __restrict__ A2,
                                                        const float* __restrict__ rbx, const float* __restrict__ rby,
                                                        const float* __restrict__ cg, const float* __restrict__ p0,
                                                        float* __restrict__ grad_p0, float* __restrict__ cbar, int R) {
    extern __shared__ float2 sm[];
    const int ng = g.ng;
    const int k = blockIdx.y;
    const int y0 = blockIdx.x * R;
    const int nr = min(R, ng - y0);
    float2* tw = sm;
    float2* z = sm + ng;
    float2* w = z + R * ng;
    load_twiddles(tw, g);
    float* q;
    c2r_rows(g, A2, k, y0, nr, z, w, tw, q);
    const size_t kf = size_t(k) * ng * ng;
    cg = medium_of(g, cg, k);
    for (int i = threadIdx.x; i < nr * ng; i += blockDim.x) {
        const int r = i / ng, x = i - r * ng, yy = y0 + r;
        const int xd = x - g.P, yd = yy - g.P;
        if (xd < 0 || xd >= g.n || yd < 0 || yd >= g.n) continue;
        const size_t o = kf + size_t(yy) * ng + x;
        const size_t od = (size_t(k) * g.n + yd) * g.n + xd;
        const float c = cg[size_t(yy) * ng + x];
        const float c2 = c * c;
        const float rs = rbx[o] + rby[o];
        grad_p0[od] += q[i] + rs / (2.f * c2);
        cbar[od] -= rs * p0[od] / (c2 * c);
    }
}

// grad_c of each instance = sum of cbar_k over its data sets (fixed order)
__global__ void k_reduce_cbar(const float* __restrict__ cbar, float* __restrict__ gc, const int* __restrict__ kfirst,
                              int ninst, int nn) {
    const size_t total = size_t(ninst) * nn;
    for (size_t t = size_t(blockIdx.x) * blockDim.x + threadIdx.x; t < total; t += size_t(gridDim.x) * blockDim.x) {
        const int inst = int(t / nn);
        const size_t i = t - size_t(inst) * nn;
        float s = 0.f;
        for (int k = kfirst[inst]; k < kfirst[inst + 1]; ++k) s += cbar[size_t(k) * nn + i];
        gc[t] = s;
    }
}

// c on the whole grid of every instance: c_dom inside the domain, c_bg in the PML
__global__ void k_medium(const float* __restrict__ cd, float* __restrict__ cg, int n, int P, int ng, int ninst,
                         float cbg) {
    const size_t total = size_t(ninst) * ng * ng;
    for (size_t t = size_t(blockIdx.x) * blockDim.x + threadIdx.x; t < total; t += size_t(gridDim.x) * blockDim.x) {
        const int inst = int(t / (size_t(ng) * ng));
        const int i = int(t - size_t(inst) * ng * ng);
        const int yy = i / ng, x = i - yy * ng;
        const int xd = x - P, yd = yy - P;
        cg[t] = (xd >= 0 && xd < n && yd >= 0 && yd < n) ? cd[(size_t(inst) * n + yd) * n + xd] : cbg;
    }
}

// r = w_k (y_pred - y_meas); FP64 partial sums of w_k/2 (y_pred - y_meas)^2, kResidBlocks per
// data set (block (b, k) covers the samples b, b + kResidBlocks * 256, ... of data set k)
__global__ void __launch_bounds__(256) k_residual(const float* __restrict__ yp, const float* __restrict__ ym,
                                                  const float* __restrict__ wts, float* __restrict__ r,
                                                  int ntm, double* __restrict__ part, int* __restrict__ flag) {
    __shared__ double red[256];
    const int k = blockIdx.y;
    const size_t off = size_t(k) * ntm;
    const float wk = wts[k];
    double acc = 0.0;
    int bad = !isfinite(wk);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ntm; i += gridDim.x * blockDim.x) {
        const float d = yp[off + i] - ym[off + i];
        r[off + i] = wk * d;
        acc += 0.5 * double(wk) * double(d) * double(d);
        if (!isfinite(d)) bad = 1;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[size_t(k) * gridDim.x + blockIdx.x] = red[0];
    if (bad) atomicOr(flag, 1);
}

// J of each instance = sum of the partials of its data sets (fixed order)
__global__ void k_sum_partials(const double* __restrict__ part, const int* __restrict__ kfirst, int ninst,
                               double* __restrict__ J, int* __restrict__ flag) {
    for (int inst = threadIdx.x; inst < ninst; inst += blockDim.x) {
        double s = 0.0;
        for (int i = kfirst[inst] * kResidBlocks; i < kfirst[inst + 1] * kResidBlocks; ++i) s += part[i];
        J[inst] = s;
        if (!isfinite(s)) atomicOr(flag, 1);
    }
}

// ---------------------------------------------------------------------------
// launchers

int check_launch(const char* what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, what);
    return PAT_OK;
}

// The dynamic shared-memory limit is a per-kernel attribute shared by every plan
// of the process (and thread): it only ever grows, so that a plan of a smaller
// grid never lowers it below what a larger plan launches with.
static std::mutex g_smem_mu;
static int g_smem_row = 0, g_smem_col = 0;

int configure_kernels(pat_plan_s* p) {
    // keep rows per CTA even (pairs of real rows) and the shared memory in bounds
    int R = p->R;
    while (R > 2 && size_t(p->ng + 2 * R * p->ng) * sizeof(float2) > 200 * 1024) R -= 2;
    p->R = R;
    p->smem_row = size_t(p->ng + 2 * R * p->ng) * sizeof(float2);
    p->smem_col = size_t(p->ng + 4 * p->C * p->ng) * sizeof(float2);
    {
        std::lock_guard<std::mutex> lock(g_smem_mu);
        if (int(p->smem_row) > g_smem_row) {
            const void* row_kernels[] = {(const void*)k_row_rho, (const void*)k_row_u, (const void*)k_row_adj_rho,
                                         (const void*)k_row_adj_u, (const void*)k_row_adj_final1,
                                         (const void*)k_row_adj_final2};
            for (const void* f : row_kernels)
                PAT_CUDA(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, int(p->smem_row)));
            g_smem_row = int(p->smem_row);
        }
        if (int(p->smem_col) > g_smem_col) {
            PAT_CUDA(cudaFuncSetAttribute((const void*)k_col, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          int(p->smem_col)));
            g_smem_col = int(p->smem_col);
        }
    }
    return select_variant(p, fixed_variants(p->ng) > 0 ? 0 : -1);
}

int select_variant(pat_plan_s* p, int variant) {
    if (variant < 0) {
        p->fast = nullptr;
        p->variant = -1;
        return PAT_OK;
    }
    const FixedOps* f = fixed_ops_for(p->ng, variant);
    if (!f) {
        set_error("no fixed-size variant %d for grid side %d", variant, p->ng);
        return PAT_EINVAL;
    }
    int rc = f->configure();
    if (rc != PAT_OK) return rc;
    p->fast = f;
    p->variant = variant;
    return PAT_OK;
}

// plan constants plus the workspace's status word (second int of the flag region)
static Geo geo_ws(const pat_plan_s* p, const Ws& w) {
    Geo g = geo(p);
    g.status = w.flag + 1;
    return g;
}

static dim3 row_grid(const pat_plan_s* p) { return dim3((p->ng + p->R - 1) / p->R, p->K); }

int launch_medium(const Launch& L, const float* c_dom, float* cg) {
    const pat_plan_s* p = L.p;
    count_launch();
    const size_t tot = size_t(p->ninst) * p->ng * p->ng;
    k_medium<<<unsigned(std::min<size_t>((tot + 255) / 256, 4096)), 256, 0, L.st>>>(c_dom, cg, p->n, p->P, p->ng,
                                                                                 p->ninst, float(p->g.c_bg));
    return check_launch("k_medium");
}

int launch_row_rho(const Launch& L, const Ws& w, int mode, const float* p0, float* y, int tstep, float* hist,
                   int hist_slot) {
    const pat_plan_s* p = L.p;
    prof_begin(PAT_K_ROW_RHO, L.st);
    if (p->fast)
        ((L.recompute && p->fast->row_rho_rc) ? p->fast->row_rho_rc : p->fast->row_rho)(
            geo_ws(p, w), L.st, w.A, w.B, w.rx, w.ry, w.cg, mode, p0, y, tstep, hist, hist_slot);
    else
        k_row_rho<<<row_grid(p), 256, p->smem_row, L.st>>>(geo(p), w.A, w.B, w.rx, w.ry, w.cg, mode, p0, y,
                                                           tstep, hist, hist_slot, p->R);
    prof_end(PAT_K_ROW_RHO, L.st);
    return check_launch("k_row_rho");
}

int launch_forward_cluster(const Launch& L, const Ws& w, const float* p0, const float* state, int n0, int n1,
                           float* y, float* hist, int hist_base, float* ckpt, float* state_out) {
    const pat_plan_s* p = L.p;
    if (!p->clops) {
        set_error("no cluster-resident stepping for grid side %d", p->ng);
        return PAT_EINVAL;
    }
    const double nrm = double(p->ng) * p->ng;
    ClusterArgs a;
    a.cg = w.cg;
    a.p0 = p0;
    a.state = state;
    a.state_out = state_out;
    a.y = y;
    a.hist = hist;
    a.hist_base = hist_base;
    a.ckpt = ckpt;
    a.s = p->s_eff;
    a.n0 = n0;
    a.n1 = n1;
    a.init = state ? 0 : 1;
    a.sg = float(p->g.dt / p->g.rho0 / nrm);
    a.sd = float(p->g.dt * p->g.rho0 / nrm);
    count_launch();
    int rc = p->clops->forward(geo_ws(p, w), L.st, a);
    if (rc != PAT_OK) return rc;
    return check_launch("kc_forward");
}

int launch_forward_persistent(const Launch& L, const Ws& w, const float* p0, float* y, float* hist, int last0,
                              float* ckpt) {
    const pat_plan_s* p = L.p;
    if (!p->sweep) {
        set_error("no persistent sweep for grid side %d", p->ng);
        return PAT_EINVAL;
    }
    const double nrm = double(p->ng) * p->ng;
    SweepArgs a;
    a.A = w.A;
    a.B = w.B;
    a.ux = w.ux;
    a.uy = w.uy;
    a.rx = w.rx;
    a.ry = w.ry;
    a.cg = w.cg;
    a.p0 = p0;
    a.y = y;
    a.hist = hist;
    a.last0 = last0;
    a.ckpt = ckpt;
    a.s = p->s_eff;
    a.sg = float(p->g.dt / p->g.rho0 / nrm);
    a.sd = float(p->g.dt * p->g.rho0 / nrm);
    a.nsteps = p->nt - 1;
    a.queue = w.queue;
    a.wait_ns = kQueueWaitNs;
    const Geo g = geo_ws(p, w);
    if (double(p->sweep->items(g, a.nsteps)) >= 2147483647.0) {
        set_error("persistent sweep: too many work items (K * nt too large)");
        return PAT_EINVAL;
    }
    count_launch();
    PAT_CUDA(cudaMemsetAsync(w.queue, 0, (size_t(p->K) + 2) * sizeof(int), L.st));
    int rc = p->sweep->launch(g, L.st, a);
    if (rc != PAT_OK) return rc;
    return check_launch("kp_forward");
}

int launch_row_u(const Launch& L, const Ws& w, int init) {
    const pat_plan_s* p = L.p;
    prof_begin(PAT_K_ROW_U, L.st);
    if (p->fast)
        ((L.recompute && p->fast->row_u_rc) ? p->fast->row_u_rc : p->fast->row_u)(geo_ws(p, w), L.st, w.A, w.B,
                                                                                   w.ux, w.uy, 0, init);
    else
        k_row_u<<<row_grid(p), 256, p->smem_row, L.st>>>(geo(p), w.A, w.B, w.ux, w.uy, init, p->R);
    prof_end(PAT_K_ROW_U, L.st);
    return check_launch("k_row_u");
}

int launch_col(const Launch& L, float2* A, float2* B, int mode, int op, float scale) {
    const pat_plan_s* p = L.p;
    dim3 grid((p->hc + p->C - 1) / p->C, p->K);
    const int cls = mode == 0 ? PAT_K_COL_GRAD : (mode == 1 ? PAT_K_COL_PAIR : PAT_K_COL_SUM);
    prof_begin(cls, L.st);
    if (p->fast)
        ((L.solo && p->fast->col_solo) ? p->fast->col_solo : p->fast->col)(geo(p), L.st, A, B, mode, op, scale);
    else
        k_col<<<grid, 256, p->smem_col, L.st>>>(geo(p), A, B, mode, op, scale, p->C);
    prof_end(cls, L.st);
    return check_launch("k_col");
}

int launch_row_adj_rho(const Launch& L, const Ws& w, int first, const float* resid, int tstep, const float* hist,
                       int hist_slot) {
    const pat_plan_s* p = L.p;
    prof_begin(PAT_K_ROW_ADJ_RHO, L.st);
    if (p->fast)
        p->fast->row_adj_rho(geo_ws(p, w), L.st, w.A2, w.B2, w.rbx, w.rby, w.cbar, w.cg, first, resid, tstep, hist,
                             hist_slot);
    else
        k_row_adj_rho<<<row_grid(p), 256, p->smem_row, L.st>>>(geo(p), w.A2, w.B2, w.rbx, w.rby, w.cbar, w.cg,
                                                               first, resid, tstep, hist, hist_slot, p->R);
    prof_end(PAT_K_ROW_ADJ_RHO, L.st);
    return check_launch("k_row_adj_rho");
}

int launch_row_adj_u(const Launch& L, const Ws& w) {
    const pat_plan_s* p = L.p;
    prof_begin(PAT_K_ROW_ADJ_U, L.st);
    if (p->fast)
        p->fast->row_u(geo_ws(p, w), L.st, w.A2, w.B2, w.ubx, w.uby, 1, 0);
    else
        k_row_adj_u<<<row_grid(p), 256, p->smem_row, L.st>>>(geo(p), w.A2, w.B2, w.ubx, w.uby, p->R);
    prof_end(PAT_K_ROW_ADJ_U, L.st);
    return check_launch("k_row_adj_u");
}

int launch_row_adj_final1(const Launch& L, const Ws& w, int first, const float* resid, float* grad_p0) {
    const pat_plan_s* p = L.p;
    count_launch();
    k_row_adj_final1<<<row_grid(p), 256, p->smem_row, L.st>>>(geo(p), w.A2, w.B2, w.ubx, w.uby, first, resid,
                                                              grad_p0, p->R);
    return check_launch("k_row_adj_final1");
}

int launch_row_adj_final2(const Launch& L, const Ws& w, const float* p0, float* grad_p0) {
    const pat_plan_s* p = L.p;
    count_launch();
    k_row_adj_final2<<<row_grid(p), 256, p->smem_row, L.st>>>(geo(p), w.A2, w.rbx, w.rby, w.cg, p0, grad_p0,
                                                              w.cbar, p->R);
    return check_launch("k_row_adj_final2");
}

int launch_reduce_cbar(const Launch& L, const Ws& w, float* grad_c) {
    const pat_plan_s* p = L.p;
    const int nn = p->n * p->n;
    const size_t tot = size_t(p->ninst) * nn;
    count_launch();
    k_reduce_cbar<<<unsigned(std::min<size_t>((tot + 255) / 256, 4096)), 256, 0, L.st>>>(w.cbar, grad_c, p->t.kfirst,
                                                                                       p->ninst, nn);
    return check_launch("k_reduce_cbar");
}

int launch_residual(const Launch& L, const Ws& w, const float* ypred, const float* ymeas, const float* wts,
                    float* resid, double* J_out) {
    const pat_plan_s* p = L.p;
    PAT_CUDA(cudaMemsetAsync(w.flag, 0, sizeof(int), L.st));
    count_launch();
    k_residual<<<dim3(kResidBlocks, p->K), 256, 0, L.st>>>(ypred, ymeas, wts, resid, p->nt * p->m, w.part, w.flag);
    int rc = check_launch("k_residual");
    if (rc) return rc;
    count_launch();
    k_sum_partials<<<1, 128, 0, L.st>>>(w.part, p->t.kfirst, p->ninst, J_out ? J_out : w.J, w.flag);
    return check_launch("k_sum_partials");
}

}  // namespace pat
